"""CUDA path vs the CPU oracle: stage arrays element by element, heights bit-exact, full-size sampled checks.

Every test here calls libqfs through its C ABI (via the ctypes binding) on cuda:0.
"""
import numpy as np
import pytest
import torch

import oracle
from helpers import example_quartics
from paper_2502_12428_gb300 import inputs

pytestmark = pytest.mark.gpu

CORE_FORMS = ["int32", "dp4a", "int8tc"]


@pytest.fixture(scope="session")
def qfs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2502_12428_gb300 import build
    build.build()
    import paper_2502_12428_gb300.qfs as q
    return q


def dev_tensor(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0")


def gpu_heights(qfs, p, f, **kw):
    return qfs.heights(p, dev_tensor(f), **kw).cpu().numpy()


def find_rows(p, n, seed, want, count, gen=inputs.dense):
    f = gen(p, n, seed)
    h = oracle.heights(p, f)
    idx = [i for i in range(n) if want(h[i])][:count]
    return f[idx], h[idx]


# ------------------------------------------------------------------------------------- stage arrays
def check_stages(qfs, p, f, form, max_h=10):
    ref = oracle.stage_arrays_a(p, f, max_h=max_h)
    got = qfs.debug_stages(p, dev_tensor(f), max_h=max_h, form=form)
    assert got["h"] == ref["h"]
    assert np.array_equal(got["g"].cpu().numpy(), ref["g"]), "f^(p-1) mod p"
    if ref["h"] != 1:
        assert np.array_equal(got["G"].cpu().numpy(), ref["D"]), "lift(g)^p mod p^2"
        assert np.array_equal(got["delta"].cpu().numpy(), ref["delta"]), "Delta_1(f^(p-1))"
        rows = ref["iters"].shape[0]
        assert np.array_equal(got["iters"].cpu().numpy()[:rows], ref["iters"]), "theta iterates"
    return ref["h"]


@pytest.mark.parametrize("form", CORE_FORMS)
def test_stages_p3(qfs, form):
    f = np.concatenate([inputs.dense(3, 10, 301), inputs.sparse(3, 4, 302), inputs.fermat()[None]])
    hs = [check_stages(qfs, 3, row, form) for row in f]
    assert any(h != 1 for h in hs)


@pytest.mark.parametrize("form", CORE_FORMS)
def test_stages_p5(qfs, form):
    f, h = find_rows(5, 400, 501, lambda x: x >= 2 or x == 0, 5)
    ex = [r[3] for r in example_quartics() if r[0] == 5 and r[1] in (1, 3, 0)]
    for row in list(f) + ex:
        check_stages(qfs, 5, row, form)


def _route_a_parallel(p, rows):
    # route A releases the interpreter while it runs (ctypes), so one thread per quartic runs them side by side
    from concurrent.futures import ThreadPoolExecutor
    with ThreadPoolExecutor(max_workers=len(rows)) as ex:
        return list(ex.map(lambda r: oracle.stage_arrays_a(p, r), rows))


@pytest.mark.slow
def test_stages_p7(qfs):
    # Figure 5's rows of height 2, 3 and infinity and a sparse quartic of height >= 3, every form, every array
    ex = {r[1]: r[3] for r in example_quartics() if r[0] == 7}
    fs, hs = find_rows(7, 3000, 7070, lambda x: x >= 3, 1, gen=inputs.sparse)
    rows = [ex[2], ex[3], ex[0], fs[0]]
    refs = _route_a_parallel(7, rows)
    assert [r["h"] for r in refs[:3]] == [2, 3, 0] and refs[3]["h"] >= 3
    for row, ref in zip(rows, refs):
        for form in CORE_FORMS:
            got = qfs.debug_stages(7, dev_tensor(row), form=form)
            assert got["h"] == ref["h"]
            assert np.array_equal(got["g"].cpu().numpy(), ref["g"])
            assert np.array_equal(got["G"].cpu().numpy(), ref["D"])
            assert np.array_equal(got["delta"].cpu().numpy(), ref["delta"])
            n_it = ref["iters"].shape[0]
            assert n_it >= 1
            assert np.array_equal(got["iters"].cpu().numpy()[:n_it], ref["iters"])


@pytest.mark.slow
def test_stages_p11(qfs):
    # Figure 6's row of height 2 at p = 11 (per-CTA buffers above 15 MB): g, G and Delta against the oracle's stage
    # arrays with D formed by products with f (equal to route A's lift(g)^p, pinned on CPU), the iterate against
    # route R (equal to route A's iterates, pinned on CPU)
    row = next(r[3] for r in example_quartics() if r[0] == 11 and r[1] == 2)
    ref = oracle.stage_arrays_fchain(11, row)
    it = oracle.stage_arrays_r(11, row)
    assert not ref["h1"] and it["h"] == 2
    for form in CORE_FORMS:
        got = qfs.debug_stages(11, dev_tensor(row), form=form)
        assert got["h"] == 2
        assert np.array_equal(got["g"].cpu().numpy(), ref["g"])
        assert np.array_equal(got["G"].cpu().numpy(), ref["D"])
        assert np.array_equal(got["delta"].cpu().numpy(), ref["delta"])
        assert np.array_equal(got["iters"].cpu().numpy()[:1], it["iters"])


# ------------------------------------------------------------------------------------- heights, small sets
@pytest.mark.parametrize("form", CORE_FORMS)
def test_heights_p3_64_plus_fermat(qfs, form):
    f = np.concatenate([inputs.dense(3, 64, inputs.config_seed(1)), inputs.fermat()[None]])
    want = oracle.heights(3, f, route=oracle.ROUTE_A)
    got = gpu_heights(qfs, 3, f, form=form)
    assert np.array_equal(got, want)
    assert got[-1] == 0  # Fermat quartic at p = 3: infinity


@pytest.mark.parametrize("form", CORE_FORMS)
def test_heights_paper_examples(qfs, form):
    rows = example_quartics()
    for p in (5, 7, 11, 13):
        sel = [r for r in rows if r[0] == p]
        f = np.stack([r[3] for r in sel])
        want = np.array([r[1] for r in sel], np.int8)
        assert np.array_equal(gpu_heights(qfs, p, f, form=form), want), f"p={p}"


@pytest.mark.parametrize("p,n", [(3, 2000), (5, 4096), (7, 1024), (11, 48)])
def test_heights_random_dense_and_sparse(qfs, p, n):
    f = np.concatenate([inputs.dense(p, n, 900 + p), inputs.sparse(p, n, 950 + p)])
    want = oracle.heights(p, f)
    for form in CORE_FORMS:
        assert np.array_equal(gpu_heights(qfs, p, f, form=form), want), form


def test_route_a_subset_p5(qfs):
    f = inputs.dense(5, 300, 1234)
    want = oracle.heights(5, f, route=oracle.ROUTE_A)
    assert np.array_equal(gpu_heights(qfs, 5, f), want)


# ------------------------------------------------------------------------------------- mixed primes in one launch
def test_multi_group_mixed_and_pgl4(qfs):
    groups, wants, pairs = [], [], []
    for p, n in [(5, 2048), (7, 1024), (11, 32)]:
        f = inputs.dense(p, n, 7700 + p)
        A = inputs.pgl4_matrices(p, n, 7800 + p)
        g = inputs.substitute(f, A, p)
        both = np.concatenate([f, g])
        groups.append((p, dev_tensor(both), None))
        wants.append(oracle.heights(p, both))
        pairs.append(n)
    outs = [o.cpu().numpy() for o in qfs.heights_multi(groups)]
    for out, want, n in zip(outs, wants, pairs):
        assert np.array_equal(out, want)
        assert np.array_equal(out[:n], out[n:])  # PGL_4 invariance of the height
    # one launch equals separate launches
    for (p, t, _), out in zip(groups, outs):
        assert np.array_equal(qfs.heights(p, t).cpu().numpy(), out)


def test_multi_group_with_empty_groups(qfs):
    # empty groups take no part in the launch; a call whose groups are all empty enqueues nothing
    f = inputs.dense(7, 300, 7900)
    empty = torch.zeros(0, 35, dtype=torch.uint8, device="cuda:0")
    outs = qfs.heights_multi([(5, empty, None), (7, dev_tensor(f), None), (11, empty, None)])
    assert outs[0].numel() == 0 and outs[2].numel() == 0
    assert np.array_equal(outs[1].cpu().numpy(), oracle.heights(7, f))
    outs = qfs.heights_multi([(5, empty, None), (7, empty, None)])
    assert all(o.numel() == 0 for o in outs)


# ------------------------------------------------------------------------------------- edge cases and errors
def test_edge_cases(qfs):
    p = 5
    assert qfs.heights(p, torch.zeros(0, 35, dtype=torch.uint8, device="cuda:0")).numel() == 0
    f = inputs.dense(p, 1000, 4242)
    bad = f.copy()
    bad[3, 0] = p
    bad[500, 34] = 255
    got = gpu_heights(qfs, p, bad)
    want = oracle.heights(p, f)
    assert got[3] == -1 and got[500] == -1
    keep = np.ones(1000, bool)
    keep[[3, 500]] = False
    assert np.array_equal(got[keep], want[keep])
    for n in (1, 7, 153):
        assert np.array_equal(gpu_heights(qfs, p, f[:n]), want[:n])
    # max_h caps: with max_h = 1 only the Fedder test runs
    h1 = gpu_heights(qfs, p, f, max_h=1)
    assert np.array_equal(h1, np.where(want == 1, 1, 0).astype(np.int8))
    h3 = gpu_heights(qfs, p, f, max_h=3)
    assert np.array_equal(h3, np.where((want >= 1) & (want <= 3), want, 0).astype(np.int8))
    # the all-zero form: f^(p-1) = 0, every iterate is zero -> infinity
    assert gpu_heights(qfs, p, np.zeros((1, 35), np.uint8))[0] == oracle.height_a(p, np.zeros(35, np.uint8)) == 0


def test_error_codes(qfs):
    t = dev_tensor(inputs.dense(5, 4, 1))
    with pytest.raises(qfs.QfsError) as e:
        qfs.heights(4, t)
    assert e.value.status == 1
    with pytest.raises(qfs.QfsError) as e:
        qfs.heights(5, t, max_h=11)
    assert e.value.status == 2
    with pytest.raises(qfs.QfsError) as e:
        qfs.heights(5, t, form=9)
    assert e.value.status == 7


def test_determinism_across_cta_counts(qfs):
    p = 7
    f = inputs.dense(p, 3000, 5151)
    t = dev_tensor(f)
    ref = qfs.heights(p, t).cpu().numpy()
    for cap in (1, 3, 37):
        assert np.array_equal(qfs.heights(p, t, max_ctas=cap).cpu().numpy(), ref)
    assert np.array_equal(ref, oracle.heights(p, f))


def test_device_status_clean(qfs):
    assert qfs.read_status() == 0


# ------------------------------------------------------------------------------------- height-1 screen
def test_screen_settles_whole_batches(qfs):
    # a batch that the screen settles entirely leaves the persistent launch with no survivors
    p = 5
    f, h = find_rows(p, 600, 6100, lambda x: x == 1, 300)
    qfs.read_stats()
    assert np.array_equal(gpu_heights(qfs, p, f), h)
    assert qfs.read_stats()[0] == 0
    bad = f.copy()
    bad[:, 7] = p
    assert (gpu_heights(qfs, p, bad) == -1).all()
    assert qfs.read_stats()[0] == 0
    # and a batch with no height-1 row at all: every row reaches the persistent launch
    g, hg = find_rows(p, 2000, 6150, lambda x: x != 1, 120)
    assert np.array_equal(gpu_heights(qfs, p, g), hg)
    assert qfs.read_stats()[0] == len(g)


def test_screen_survivor_count_matches_oracle(qfs):
    p = 7
    f = inputs.dense(p, 1500, 6200)
    want = oracle.heights(p, f)
    qfs.read_stats()
    assert np.array_equal(gpu_heights(qfs, p, f), want)
    assert qfs.read_stats()[0] == int((want != 1).sum())


@pytest.mark.parametrize("p", [3, 11, 13])
def test_screen_fedder_decision(qfs, p):
    # with max_h = 1 only the height-1 test decides a row: F = f^((p-1)/2) takes 0, 4 and 5 products in the warp
    f = np.concatenate([inputs.dense(p, 1200, 6300 + p), inputs.sparse(p, 400, 6400 + p)])
    want = oracle.heights(p, f, max_h=1)
    assert np.array_equal(gpu_heights(qfs, p, f, max_h=1), want)


# ------------------------------------------------------------------------------------- staged engine
@pytest.mark.parametrize("p,n", [(3, 500), (5, 3000), (7, 600)])
def test_staged_engine_matches_fused_and_oracle(qfs, p, n):
    f = np.concatenate([inputs.dense(p, n, 9100 + p), inputs.sparse(p, n // 2, 9200 + p)])
    bad = f.copy()
    bad[1, 3] = p
    t = dev_tensor(bad)
    fused = qfs.heights(p, t).cpu().numpy()
    staged = qfs.heights(p, t, engine="staged").cpu().numpy()
    assert np.array_equal(staged, fused)
    want = oracle.heights(p, f)
    want[1] = -1
    assert np.array_equal(staged, want)
    for max_h in (1, 3):
        assert np.array_equal(qfs.heights(p, t, engine="staged", max_h=max_h).cpu().numpy(),
                              qfs.heights(p, t, max_h=max_h).cpu().numpy())
    assert qfs.read_status() == 0


def test_staged_engine_small_chunks_and_multi(qfs):
    # a tiny workspace budget forces many chunks (admission by memory)
    f5 = inputs.dense(5, 5000, 9300)
    f7 = inputs.dense(7, 400, 9301)
    t5, t7 = dev_tensor(f5), dev_tensor(f7)
    outs = qfs.heights_multi([(5, t5, None), (7, t7, None)], engine="staged", workspace_budget=64 << 20)
    assert np.array_equal(outs[0].cpu().numpy(), oracle.heights(5, f5))
    assert np.array_equal(outs[1].cpu().numpy(), oracle.heights(7, f7))
    assert qfs.read_status() == 0


# ------------------------------------------------------------------------------------- identity power mode
@pytest.mark.parametrize("p,n", [(3, 6), (5, 6)])
def test_identity_power_stage_arrays(qfs, p, n):
    # the identity mode forms the same Delta_1(f^(p-1)) array as Algorithm 1, element by element
    f, h = find_rows(p, 400, 700 + p, lambda x: x >= 2 or x == 0, n)
    for row in f:
        ref = oracle.stage_arrays_a(p, row)
        for form in CORE_FORMS:
            got = qfs.debug_stages(p, dev_tensor(row), form=form, power="identity")
            assert got["h"] == ref["h"]
            assert np.array_equal(got["delta"].cpu().numpy(), ref["delta"]), form
            rows = ref["iters"].shape[0]
            assert np.array_equal(got["iters"].cpu().numpy()[:rows], ref["iters"]), form


@pytest.mark.parametrize("p,n", [(3, 1500), (5, 3000), (7, 800), (11, 24), (13, 6)])
def test_identity_power_heights(qfs, p, n):
    f = np.concatenate([inputs.dense(p, n, 7500 + p), inputs.sparse(p, n, 7600 + p)])
    t = dev_tensor(f)
    want = oracle.heights(p, f)
    for form in CORE_FORMS:
        assert np.array_equal(qfs.heights(p, t, form=form, power="identity").cpu().numpy(), want), form
    assert qfs.read_status() == 0


def test_identity_power_paper_examples(qfs):
    for p in (5, 7, 11, 13):
        sel = [r for r in example_quartics() if r[0] == p]
        f = np.stack([r[3] for r in sel])
        want = np.array([r[1] for r in sel], np.int8)
        assert np.array_equal(qfs.heights(p, dev_tensor(f), power="identity").cpu().numpy(), want), p


# ------------------------------------------------------------------------------------- tile autotuner, graphs
def test_tile_shapes_do_not_change_heights(qfs):
    p = 7
    f = inputs.dense(p, 1200, 6600)
    t = dev_tensor(f)
    want = oracle.heights(p, f)
    saved = qfs.tune_get(p)
    try:
        for rc, ring in [(256, 48 << 10), (1024, 80 << 10), (64, 32 << 10)]:
            qfs.tune_set(p, rc, ring)
            assert qfs.tune_get(p)["round_chunks"] == rc
            assert np.array_equal(qfs.heights(p, t).cpu().numpy(), want)
        with pytest.raises(qfs.QfsError):
            qfs.tune_set(p, 8, 48 << 10)
        best = qfs.autotune(p, t[:400])
        assert best["round_chunks"] >= 32 and best["ms"] > 0
        assert np.array_equal(qfs.heights(p, t).cpu().numpy(), want)
    finally:
        qfs.tune_set(p, saved["round_chunks"], saved["ring_bytes"])


@pytest.mark.parametrize("form", ["dp4a", "int32"])
def test_sweep_shapes_do_not_change_heights(qfs, form):
    # the swept chain's dense threshold decides, per quartic, between the every-pair two-slice loop and the
    # zero-pair-skipping one-slice loop; mixed dense and sparse rows take both paths under every threshold
    p = 5
    f = np.concatenate([inputs.dense(p, 700, 6610), inputs.sparse(p, 1300, 6611)])
    t = dev_tensor(f)
    want = oracle.heights(p, f)
    saved = qfs.sweep_tune_get(form, p)
    try:
        for dm, ctas in [(0, 2), (16, 1), (8, 0), (12, 1)]:
            qfs.sweep_tune_set(form, p, dm, ctas)
            assert qfs.sweep_tune_get(form, p) == {"dense_min": dm if dm else 12, "ctas_per_sm": ctas}
            assert np.array_equal(qfs.heights(p, t, form=form).cpu().numpy(), want)
        with pytest.raises(qfs.QfsError):
            qfs.sweep_tune_set(form, p, 17, 0)
        with pytest.raises(qfs.QfsError):
            qfs.sweep_tune_set("int8tc", p, 8, 0)
        best = qfs.sweep_autotune(p, t[:600], form=form)
        assert 0 <= best["dense_min"] <= 16 and best["ctas_per_sm"] >= 0 and best["ms"] > 0
        assert qfs.sweep_tune_get(form, p)["ctas_per_sm"] == best["ctas_per_sm"]
        assert np.array_equal(qfs.heights(p, t, form=form).cpu().numpy(), want)
    finally:
        qfs.sweep_tune_set(form, p, saved["dense_min"], saved["ctas_per_sm"])


def test_cuda_graph_capture_and_replay(qfs):
    # the call is stream-ordered and allocation-free once the workspace exists, so it can be captured
    p = 5
    a = inputs.dense(p, 3000, 6700)
    want = oracle.heights(p, a)
    coeffs = dev_tensor(a)
    out = torch.empty(3000, dtype=torch.int8, device="cuda:0")
    qfs.heights(p, coeffs, out=out)              # sizes the workspace before capture
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    out.zero_()
    with torch.cuda.graph(g):
        qfs.heights(p, coeffs, out=out)
    for _ in range(2):
        out.fill_(-5)
        g.replay()
        torch.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy(), want)
    # new inputs in the same buffer replay through the same graph
    b = inputs.sparse(p, 3000, 6701)
    coeffs.copy_(torch.from_numpy(b))
    g.replay()
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), oracle.heights(p, b))


# ------------------------------------------------------------------------------------- reduced theta mode
@pytest.mark.parametrize("p,n", [(3, 6), (5, 6), (7, 2)])
def test_reduced_mode_iterates(qfs, p, n):
    # the reduced step gives the same iterates g_h as u(Delta_1(f^(p-1)) g) (route A), element by element
    f, h = find_rows(p, 300, 800 + p, lambda x: x >= 2 or x == 0, n)
    for row in f:
        ref = oracle.stage_arrays_r(p, row)
        for form in CORE_FORMS:
            got = qfs.debug_stages(p, dev_tensor(row), form=form, power="reduced")
            assert got["h"] == ref["h"]
            rows = ref["iters"].shape[0]
            assert np.array_equal(got["iters"].cpu().numpy()[:rows], ref["iters"]), form


@pytest.mark.parametrize("p,n", [(3, 1500), (5, 4000), (7, 2000), (11, 200), (13, 60)])
def test_reduced_mode_heights(qfs, p, n):
    f = np.concatenate([inputs.dense(p, n, 8500 + p), inputs.sparse(p, n, 8600 + p)])
    t = dev_tensor(f)
    want = oracle.heights(p, f)
    for form in CORE_FORMS:
        assert np.array_equal(qfs.heights(p, t, form=form, power="reduced").cpu().numpy(), want), form
    for max_h in (1, 2, 4):
        assert np.array_equal(qfs.heights(p, t, power="reduced", max_h=max_h).cpu().numpy(),
                              oracle.heights(p, f, max_h=max_h))
    assert qfs.read_status() == 0


def test_reduced_mode_paper_examples(qfs):
    for p in (5, 7, 11, 13):
        sel = [r for r in example_quartics() if r[0] == p]
        f = np.stack([r[3] for r in sel])
        want = np.array([r[1] for r in sel], np.int8)
        assert np.array_equal(qfs.heights(p, dev_tensor(f), power="reduced").cpu().numpy(), want), p


# ------------------------------------------------------------------------------------- theta matrix export
@pytest.mark.parametrize("p,n", [(3, 8), (5, 3), (7, 1)])
def test_theta_matrix_matches_oracle(qfs, p, n):
    # every entry of M equals the oracle's M from its definition; height-1 rows are exported too
    f = np.concatenate([inputs.dense(p, n, 8800 + p), inputs.sparse(p, 1, 8900 + p)])
    got = qfs.theta_matrix(p, dev_tensor(f)).cpu().numpy()
    for i in range(len(f)):
        assert np.array_equal(got[i], oracle.theta_matrix(p, f[i])), i
    assert qfs.read_status() == 0


def test_theta_matrix_applies_theta_and_rejects_bad_rows(qfs):
    # M g = theta(g): the device's first iterate, and an invalid row gives M = 0
    p = 5
    f, h = find_rows(p, 400, 8950, lambda x: x >= 2, 2)
    bad = f[:1].copy()
    bad[0, 7] = p
    rows = np.concatenate([f, bad])
    M = qfs.theta_matrix(p, dev_tensor(rows)).cpu().numpy().astype(np.int64)
    for i in range(len(f)):
        st = qfs.debug_stages(p, dev_tensor(f[i]))
        g = st["g"].cpu().numpy().astype(np.int64)
        assert np.array_equal(M[i] @ g % p, st["iters"].cpu().numpy()[0])
    assert not M[-1].any()
    with pytest.raises(qfs.QfsError):
        qfs.theta_matrix(4, dev_tensor(f))


# ------------------------------------------------------------------------------------- matrix multiplication mod p
@pytest.mark.parametrize("p,n,m,k", [(11, 1, 1, 1), (11, 17, 33, 65), (11, 300, 257, 129), (11, 128, 128, 64),
                                     (11, 513, 130, 1000), (2, 200, 300, 77), (251, 140, 70, 300), (256, 64, 64, 64)])
def test_matmul_mod_matches_oracle(qfs, p, n, m, k):
    rng = np.random.default_rng(p * 1000 + n + m + k)
    A = rng.integers(0, p, (n, k), dtype=np.uint8)
    B = rng.integers(0, p, (k, m), dtype=np.uint8)
    got = qfs.matmul_mod(p, dev_tensor(A), dev_tensor(B)).cpu().numpy()
    assert np.array_equal(got, oracle.matmul_mod(p, A, B))


def test_matmul_mod_long_k_reduces_between_tiles(qfs):
    # k (p-1)^2 above 2^31 at p = 251: the accumulators are reduced between K tiles
    p, n, m, k = 251, 16, 24, 40000
    rng = np.random.default_rng(9)
    A = rng.integers(p - 20, p, (n, k), dtype=np.uint8)
    B = rng.integers(p - 20, p, (k, m), dtype=np.uint8)
    got = qfs.matmul_mod(p, dev_tensor(A), dev_tensor(B)).cpu().numpy()
    assert np.array_equal(got, oracle.matmul_mod(p, A, B))


def test_matmul_mod_full_size_sampled(qfs):
    # the paper's smallest size (5,000 x 5,000 mod 11); 256 entries checked one by one
    p, n = 11, 5000
    g = torch.Generator(device="cuda").manual_seed(11)
    A = torch.randint(0, p, (n, n), dtype=torch.uint8, device="cuda", generator=g)
    B = torch.randint(0, p, (n, n), dtype=torch.uint8, device="cuda", generator=g)
    C = qfs.matmul_mod(p, A, B).cpu().numpy()
    An, Bn = A.cpu().numpy(), B.cpu().numpy()
    rng = np.random.default_rng(3)
    for i, j in zip(rng.integers(0, n, 256), rng.integers(0, n, 256)):
        assert C[i, j] == oracle.matmul_mod(p, An[i:i + 1], Bn[:, j:j + 1])[0, 0]


def test_matmul_mod_edges(qfs):
    z = torch.zeros(0, 5, dtype=torch.uint8, device="cuda")
    assert qfs.matmul_mod(11, z, torch.zeros(5, 3, dtype=torch.uint8, device="cuda")).shape == (0, 3)
    A = torch.ones(4, 0, dtype=torch.uint8, device="cuda")
    C = qfs.matmul_mod(11, A, torch.ones(0, 6, dtype=torch.uint8, device="cuda"))
    assert C.shape == (4, 6) and not C.any()
    with pytest.raises(qfs.QfsError):
        qfs.matmul_mod(1, torch.ones(2, 2, dtype=torch.uint8, device="cuda"), torch.ones(2, 2, dtype=torch.uint8,
                                                                                         device="cuda"))


# ------------------------------------------------------------------------------------- exact powering over Z
def _multinomial(es):
    from math import factorial
    out = factorial(sum(es))
    for e in es:
        out //= factorial(e)
    return out


def _eval_mod(cs, deg, pt, mod):
    pw = [[pow(x, k, mod) for k in range(deg + 1)] for x in pt]
    acc = 0
    for c, e in zip(cs, oracle.form_monomials(deg)):
        acc = (acc + c * pw[0][e[0]] * pw[1][e[1]] * pw[2][e[2]] * pw[3][e[3]]) % mod
    return acc


@pytest.mark.parametrize("d,n", [(1, 100), (16, 6)])
def test_poly_power_multinomial_closed_form(qfs, d, n):
    # (x1+x2+x3+x4)^d to the n-th power: every coefficient is a multinomial coefficient (up to 200 bits)
    f = [_multinomial(e) for e in oracle.form_monomials(d)]
    got = qfs.poly_power(d, f, n)
    assert got == [_multinomial(e) for e in oracle.form_monomials(d * n)]


# (d, n) chosen so that the transform length puts every pass size on the device: (1, 7) a one-stage column pass
# (the shared-memory stage loop), (1, 9) two, (2, 5) three, (4, 3) four, (16, 1) five, (4, 5) six, (5, 6) seven,
# (16, 2) eight; transforms of 2^13 words or more ((16, 1), (16, 2), (4, 5), (5, 6)) run the register-phase inner
# pass, the shorter ones the shared-memory one
@pytest.mark.parametrize("d,n", [(4, 3), (16, 2), (16, 1), (1, 7), (1, 9), (2, 5), (4, 5), (5, 6)])
def test_poly_power_matches_definition(qfs, d, n):
    rng = np.random.default_rng(d * 100 + n)
    f = [int(x) for x in rng.integers(0, 5, len(oracle.form_monomials(d)))]
    assert qfs.poly_power(d, f, n) == oracle.poly_power(d, f, n)


@pytest.mark.parametrize("n", [5, 15])
def test_poly_power_paper_workload_evaluation(qfs, n):
    # degree 16, coefficients in {0..4}: f^n(pt) = f(pt)^n at an integer point, modulo 2^127 - 1
    rng = np.random.default_rng(16 + n)
    f = [int(x) for x in rng.integers(0, 5, len(oracle.form_monomials(16)))]
    P = qfs.poly_power(16, f, n)
    mod = (1 << 127) - 1
    pt = (3, 5, 7, 11)
    assert _eval_mod(P, 16 * n, pt, mod) == pow(_eval_mod(f, 16, pt, mod), n, mod)


def test_poly_power_errors(qfs):
    with pytest.raises(qfs.QfsError):
        qfs.poly_power(16, [1] * 969, 16)   # degree 256
    with pytest.raises(qfs.QfsError):
        qfs.poly_power(1, [2 ** 31] * 4, 8)   # coefficients too large for 256 bits
