"""Python binding of libqfs (include/qfs.h): argument marshalling only, every step runs in the CUDA library.

Tensors are PyTorch CUDA tensors; the binding passes their data pointers and the current CUDA stream.  There is
no CPU fallback: if the library is not built, or no CUDA device is present, every call raises.
"""
import ctypes
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libqfs.so")

OK = 0
FORM_INT32, FORM_DP4A, FORM_INT8TC = 0, 1, 2
ENGINE_FUSED, ENGINE_STAGED = 0, 1
FORMS = {"int32": FORM_INT32, "dp4a": FORM_DP4A, "int8tc": FORM_INT8TC}
ENGINES = {"fused": ENGINE_FUSED, "staged": ENGINE_STAGED}
POWER_CHAIN, POWER_IDENTITY, POWER_REDUCED = 0, 1, 2
POWERS = {"chain": POWER_CHAIN, "identity": POWER_IDENTITY, "reduced": POWER_REDUCED}
MAX_GROUPS = 8
PRIMES = (3, 5, 7, 11, 13)


class QfsError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        msg = _lib().qfs_strerror(status).decode() if _LIB is not None else f"status {status}"
        if status == 6 and _LIB is not None:
            msg += f" (cudaError {_LIB.qfs_last_cuda_error()})"
        super().__init__(f"{where}: {msg}")


class Group(ctypes.Structure):
    _fields_ = [("p", ctypes.c_int), ("n", ctypes.c_int64), ("coeffs", ctypes.c_void_p),
                ("heights_out", ctypes.c_void_p)]


class Options(ctypes.Structure):
    _fields_ = [("form", ctypes.c_int), ("engine", ctypes.c_int), ("ctas_per_sm", ctypes.c_int),
                ("max_ctas", ctypes.c_int), ("workspace_budget", ctypes.c_size_t), ("power", ctypes.c_int)]


_LIB = None


def _lib():
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libqfs is not built ({LIB_PATH} missing): run __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        vp, i64, c_int = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
        L.qfs_heights.argtypes = [c_int, i64, vp, c_int, vp, vp]
        L.qfs_heights_multi.argtypes = [c_int, ctypes.POINTER(Group), c_int, vp]
        L.qfs_heights_multi_ex.argtypes = [c_int, ctypes.POINTER(Group), c_int, ctypes.POINTER(Options), vp]
        L.qfs_set_default_form.argtypes = [c_int]
        L.qfs_plan_prepare.argtypes = [c_int, i64]
        L.qfs_shutdown.argtypes = []
        L.qfs_read_status.argtypes = [ctypes.POINTER(ctypes.c_uint32)]
        L.qfs_read_stats.argtypes = [ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64)]
        L.qfs_strerror.argtypes = [c_int]
        L.qfs_strerror.restype = ctypes.c_char_p
        L.qfs_last_cuda_error.argtypes = []
        L.qfs_debug_stages.argtypes = [c_int, vp, c_int, c_int, vp, vp, vp, vp, vp]
        L.qfs_heights_noalloc.argtypes = [c_int, i64, vp, c_int, vp, vp]
        L.qfs_theta_matrix.argtypes = [c_int, i64, vp, vp, vp]
        L.qfs_matmul_mod.argtypes = [c_int, c_int, c_int, c_int, vp, vp, vp, vp]
        L.qfs_poly_power.argtypes = [c_int, vp, c_int, vp, vp]
        L.qfs_int_peaks.argtypes = [ctypes.POINTER(ctypes.c_double), ctypes.POINTER(c_int), ctypes.POINTER(c_int)]
        L.qfs_poly_power_info.argtypes = [c_int, vp, c_int, ctypes.POINTER(c_int), ctypes.POINTER(ctypes.c_uint64),
                                          ctypes.POINTER(ctypes.c_uint64)]
        L.qfs_tune_set.argtypes = [c_int, c_int, ctypes.c_size_t]
        L.qfs_tune_get.argtypes = [c_int, ctypes.POINTER(c_int), ctypes.POINTER(ctypes.c_size_t),
                                   ctypes.POINTER(ctypes.c_size_t)]
        L.qfs_autotune.argtypes = [c_int, i64, vp, c_int, ctypes.POINTER(c_int), ctypes.POINTER(ctypes.c_size_t),
                                   ctypes.POINTER(ctypes.c_float)]
        L.qfs_sweep_tune_set.argtypes = [c_int, c_int, c_int, c_int]
        L.qfs_sweep_tune_get.argtypes = [c_int, c_int, ctypes.POINTER(c_int), ctypes.POINTER(c_int)]
        L.qfs_sweep_autotune.argtypes = [c_int, c_int, i64, vp, ctypes.POINTER(c_int), ctypes.POINTER(c_int),
                                         ctypes.POINTER(ctypes.c_float)]
        for name in ("qfs_heights", "qfs_heights_multi", "qfs_heights_multi_ex", "qfs_set_default_form",
                     "qfs_plan_prepare", "qfs_shutdown", "qfs_read_status", "qfs_read_stats", "qfs_last_cuda_error",
                     "qfs_debug_stages", "qfs_heights_noalloc", "qfs_tune_set", "qfs_tune_get", "qfs_autotune",
                     "qfs_sweep_tune_set", "qfs_sweep_tune_get", "qfs_sweep_autotune",
                     "qfs_theta_matrix", "qfs_matmul_mod", "qfs_poly_power", "qfs_poly_power_info",
                     "qfs_int_peaks"):
            getattr(L, name).restype = c_int
        _LIB = L
        load_tile_table()
    return _LIB


def lib():
    """The loaded ctypes library (loads it on first use)."""
    return _lib()


def _check(rc, where):
    if rc != OK:
        raise QfsError(rc, where)


def _need_cuda(t, dtype, name):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must have dtype {dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _options(form, engine, ctas_per_sm, max_ctas, workspace_budget, power=None):
    o = Options()
    o.power = POWERS[power] if isinstance(power, str) else (-1 if power is None else int(power))
    o.form = FORMS[form] if isinstance(form, str) else (-1 if form is None else int(form))
    o.engine = ENGINES[engine] if isinstance(engine, str) else (-1 if engine is None else int(engine))
    o.ctas_per_sm = int(ctas_per_sm)
    o.max_ctas = int(max_ctas)
    o.workspace_budget = int(workspace_budget)
    return o


def heights(p, coeffs, max_h=10, out=None, stream=None, form=None, engine=None, ctas_per_sm=0, max_ctas=0,
            workspace_budget=0, power=None):
    """Heights of the quartics in `coeffs` (CUDA uint8 tensor, n x 35, descending lex) over F_p.

    Returns an int8 CUDA tensor of n codes (1..max_h height, 0 infinity, -1 invalid row).  Asynchronous on the
    current stream (or `stream`).
    """
    _need_cuda(coeffs, torch.uint8, "coeffs")
    if coeffs.dim() != 2 or coeffs.shape[1] != 35:
        raise ValueError("coeffs must have shape (n, 35)")
    n = coeffs.shape[0]
    if out is None:
        out = torch.empty(n, dtype=torch.int8, device=coeffs.device)
    _need_cuda(out, torch.int8, "out")
    return heights_multi([(p, coeffs, out)], max_h, stream, form, engine, ctas_per_sm, max_ctas,
                         workspace_budget, power)[0]


def heights_multi(groups, max_h=10, stream=None, form=None, engine=None, ctas_per_sm=0, max_ctas=0,
                  workspace_budget=0, power=None):
    """One launch over several (p, coeffs, out) batches; `out` may be None.  Returns the list of outputs."""
    if not 1 <= len(groups) <= MAX_GROUPS:
        raise ValueError(f"between 1 and {MAX_GROUPS} groups")
    arr = (Group * len(groups))()
    outs = []
    for i, (p, coeffs, out) in enumerate(groups):
        _need_cuda(coeffs, torch.uint8, "coeffs")
        if coeffs.dim() != 2 or coeffs.shape[1] != 35:
            raise ValueError("coeffs must have shape (n, 35)")
        if out is None:
            out = torch.empty(coeffs.shape[0], dtype=torch.int8, device=coeffs.device)
        _need_cuda(out, torch.int8, "out")
        if out.numel() != coeffs.shape[0]:
            raise ValueError("out must have one entry per quartic")
        if out.device != coeffs.device:
            raise ValueError("out and coeffs must be on the same device")
        arr[i].p, arr[i].n = int(p), int(coeffs.shape[0])
        arr[i].coeffs, arr[i].heights_out = coeffs.data_ptr(), out.data_ptr()
        outs.append(out)
    opts = _options(form, engine, ctas_per_sm, max_ctas, workspace_budget, power)
    rc = _lib().qfs_heights_multi_ex(len(groups), arr, int(max_h), ctypes.byref(opts), _stream(stream))
    _check(rc, "qfs_heights_multi_ex")
    return outs


def heights_noalloc(p, coeffs, max_h=10, out=None, stream=None):
    """qfs_heights_noalloc: the same heights, computed in the library's fixed 64 MiB device scratch array, with no
    device allocation inside the call (for callers that cannot allocate then, e.g. during a global-mode stream
    capture or under another allocator that owns the device).  Make the first call on a device before any capture.
    Calls that overlap on the GPU share the scratch and race."""
    _need_cuda(coeffs, torch.uint8, "coeffs")
    if coeffs.dim() != 2 or coeffs.shape[1] != 35:
        raise ValueError("coeffs must have shape (n, 35)")
    if out is None:
        out = torch.empty(coeffs.shape[0], dtype=torch.int8, device=coeffs.device)
    _need_cuda(out, torch.int8, "out")
    if out.numel() != coeffs.shape[0]:
        raise ValueError("out must have one entry per quartic")
    if out.device != coeffs.device:
        raise ValueError("out and coeffs must be on the same device")
    rc = _lib().qfs_heights_noalloc(int(p), int(coeffs.shape[0]), coeffs.data_ptr(), int(max_h), out.data_ptr(),
                                    _stream(stream))
    _check(rc, "qfs_heights_noalloc")
    return out


def theta_matrix(p, coeffs, out=None, stream=None):
    """qfs_theta_matrix: the theta matrix M of each quartic (coeffs: CUDA uint8 (n, 35) or (35,)), as a CUDA uint8
    tensor (n, ld, ld) or (ld, ld), ld = C(4p-1, 3): M[r][c] = Delta_1(f^(p-1))[p r + (p-1)1 - c] mod p, so that
    theta(g) = M g mod p."""
    _need_cuda(coeffs, torch.uint8, "coeffs")
    single = coeffs.dim() == 1
    c2 = coeffs.reshape(-1, 35).contiguous()
    ld = (4 * p - 1) * (4 * p - 2) * (4 * p - 3) // 6
    if out is None:
        out = torch.empty(c2.shape[0], ld, ld, dtype=torch.uint8, device=coeffs.device)
    _need_cuda(out, torch.uint8, "out")
    rc = _lib().qfs_theta_matrix(int(p), int(c2.shape[0]), c2.data_ptr(), out.data_ptr(), _stream(stream))
    _check(rc, "qfs_theta_matrix")
    return out[0] if single else out


def matmul_mod(p, A, B, out=None, stream=None):
    """qfs_matmul_mod: C = A B mod p for CUDA uint8 matrices A (n, k) and B (k, m) with values in [0, p)."""
    _need_cuda(A, torch.uint8, "A")
    _need_cuda(B, torch.uint8, "B")
    if A.dim() != 2 or B.dim() != 2 or A.shape[1] != B.shape[0]:
        raise ValueError("A (n, k) and B (k, m) required")
    A, B = A.contiguous(), B.contiguous()
    n, k = A.shape
    m = B.shape[1]
    if out is None:
        out = torch.empty(n, m, dtype=torch.uint8, device=A.device)
    _need_cuda(out, torch.uint8, "out")
    _check(_lib().qfs_matmul_mod(int(p), int(n), int(m), int(k), A.data_ptr(), B.data_ptr(), out.data_ptr(),
                                 _stream(stream)), "qfs_matmul_mod")
    return out


def poly_power_limbs(d, coeffs, n, out=None, stream=None, device=None):
    """qfs_poly_power: the n-th power over Z of the degree-d form with nonnegative integer coefficients `coeffs`
    (host sequence, descending lex).  Returns a CUDA int64 tensor (C(d n + 3, 3), 8) of 32-bit limbs (little endian)
    holding each 256-bit coefficient; poly_power() turns them into Python integers."""
    c = np.ascontiguousarray(np.asarray(coeffs, dtype=np.uint32).reshape(-1))
    n_out = (d * n + 3) * (d * n + 2) * (d * n + 1) // 6
    if out is None:
        out = torch.empty(n_out, 8, dtype=torch.int32, device=device or "cuda")
    _need_cuda(out, torch.int32, "out")
    _check(_lib().qfs_poly_power(int(d), c.ctypes.data, int(n), out.data_ptr(), _stream(stream)), "qfs_poly_power")
    return out


def poly_power_info(d, coeffs, n):
    """qfs_poly_power_info: {nprimes, transform_len, hbm_bytes} of one poly_power_limbs call (host only)."""
    c = np.ascontiguousarray(np.asarray(coeffs, dtype=np.uint32).reshape(-1))
    npr, tl, hb = ctypes.c_int(0), ctypes.c_uint64(0), ctypes.c_uint64(0)
    _check(_lib().qfs_poly_power_info(int(d), c.ctypes.data, int(n), ctypes.byref(npr), ctypes.byref(tl),
                                      ctypes.byref(hb)), "qfs_poly_power_info")
    return dict(nprimes=npr.value, transform_len=tl.value, hbm_bytes=hb.value)


def poly_power(d, coeffs, n, stream=None):
    """The coefficients of f^n as Python integers (descending lex order)."""
    limbs = poly_power_limbs(d, coeffs, n, stream=stream).cpu().numpy().astype(np.uint32).astype(object)
    out = limbs[:, 0].copy()
    for l in range(1, 8):
        out = out + (limbs[:, l] << (32 * l))
    return list(out)


TILE_TABLE = os.path.join(_HERE, "tile_table.json")


def tune_set(p, round_chunks, ring_bytes):
    _check(_lib().qfs_tune_set(int(p), int(round_chunks), int(ring_bytes)), "qfs_tune_set")


def tune_get(p):
    r, ring, smem = ctypes.c_int(0), ctypes.c_size_t(0), ctypes.c_size_t(0)
    _check(_lib().qfs_tune_get(int(p), ctypes.byref(r), ctypes.byref(ring), ctypes.byref(smem)), "qfs_tune_get")
    return dict(round_chunks=r.value, ring_bytes=ring.value, smem_bytes=smem.value)


def autotune(p, sample, form="dp4a"):
    """Times every candidate chain tile shape on `sample` (CUDA uint8 n x 35) and keeps the fastest for p."""
    _need_cuda(sample, torch.uint8, "sample")
    r, ring, ms = ctypes.c_int(0), ctypes.c_size_t(0), ctypes.c_float(0)
    rc = _lib().qfs_autotune(int(p), int(sample.shape[0]), sample.data_ptr(),
                             FORMS[form] if isinstance(form, str) else int(form), ctypes.byref(r), ctypes.byref(ring),
                             ctypes.byref(ms))
    _check(rc, "qfs_autotune")
    return dict(p=int(p), round_chunks=r.value, ring_bytes=ring.value, ms=ms.value)


def save_tile_table(entries, path=TILE_TABLE):
    """Persists autotuner results ({p: {round_chunks, ring_bytes, ...}}) as JSON."""
    import json
    with open(path, "w") as fh:
        json.dump({str(k): v for k, v in entries.items()}, fh, indent=1, sort_keys=True)


def _form_id(form):
    return FORMS[form] if isinstance(form, str) else int(form)


def sweep_tune_set(form, p, dense_min, ctas_per_sm):
    """qfs_sweep_tune_set: swept-chain shape of (form, p); (0, 0) restores the defaults."""
    _check(_lib().qfs_sweep_tune_set(_form_id(form), int(p), int(dense_min), int(ctas_per_sm)), "qfs_sweep_tune_set")


def sweep_tune_get(form, p):
    dm, c = ctypes.c_int(0), ctypes.c_int(0)
    _check(_lib().qfs_sweep_tune_get(_form_id(form), int(p), ctypes.byref(dm), ctypes.byref(c)), "qfs_sweep_tune_get")
    return dict(dense_min=dm.value, ctas_per_sm=c.value)


def sweep_autotune(p, sample, form="dp4a"):
    """Times every candidate swept-chain shape (dense threshold x CTAs per SM) on `sample` (CUDA uint8 n x 35) and
    keeps the fastest for (form, p)."""
    _need_cuda(sample, torch.uint8, "sample")
    dm, c, ms = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_float(0)
    _check(_lib().qfs_sweep_autotune(_form_id(form), int(p), int(sample.shape[0]), sample.data_ptr(),
                                     ctypes.byref(dm), ctypes.byref(c), ctypes.byref(ms)), "qfs_sweep_autotune")
    return dict(dense_min=dm.value, ctas_per_sm=c.value, ms=ms.value)


def load_tile_table(path=TILE_TABLE):
    """Applies a persisted tile table (missing file: nothing to do): per prime the ring tile of the int8 tensor
    form, and under "sweep" the swept-chain shape of each of the dp4a and int32 forms.  Returns the entries."""
    import json
    if not os.path.exists(path):
        return {}
    with open(path) as fh:
        table = json.load(fh)
    for p, v in table.items():
        if "round_chunks" in v:
            tune_set(int(p), v["round_chunks"], v["ring_bytes"])
        for form, sw in v.get("sweep", {}).items():
            sweep_tune_set(form, int(p), sw["dense_min"], sw["ctas_per_sm"])
    return table


def set_default_form(form):
    _check(_lib().qfs_set_default_form(FORMS[form] if isinstance(form, str) else int(form)), "qfs_set_default_form")


def plan_prepare(p, n_hint=0):
    _check(_lib().qfs_plan_prepare(int(p), int(n_hint)), "qfs_plan_prepare")


def shutdown():
    _check(_lib().qfs_shutdown(), "qfs_shutdown")


def int_peaks():
    """Measured integer multiply-add rates of the current device (qfs_int_peaks): dict with MACs/s of IMAD, IDP4A
    and mma.sync s8, the SM count and the maximum SM clock in MHz."""
    rates = (ctypes.c_double * 3)()
    sms, khz = ctypes.c_int(0), ctypes.c_int(0)
    _check(_lib().qfs_int_peaks(rates, ctypes.byref(sms), ctypes.byref(khz)), "qfs_int_peaks")
    return dict(imad=rates[0], dp4a=rates[1], mma_s8=rates[2], sms=sms.value, max_mhz=khz.value / 1e3)


def read_status():
    v = ctypes.c_uint32(0)
    _check(_lib().qfs_read_status(ctypes.byref(v)), "qfs_read_status")
    return v.value


def read_stats():
    """(survivors, theta_steps) counted by the device since the last call (synchronises)."""
    a, b = ctypes.c_uint64(0), ctypes.c_uint64(0)
    _check(_lib().qfs_read_stats(ctypes.byref(a), ctypes.byref(b)), "qfs_read_stats")
    return a.value, b.value


def debug_stages(p, coeffs, max_h=10, form="dp4a", power="chain"):
    """Runs the device pipeline on one quartic and returns every intermediate array (int32 CUDA tensors,
    descending lex): dict(h, g, G, delta, iters).  Synchronous; for parity tests."""
    _need_cuda(coeffs, torch.uint8, "coeffs")
    coeffs = coeffs.reshape(35).contiguous()
    dev = coeffs.device
    ld = (4 * p - 1) * (4 * p - 2) * (4 * p - 3) // 6
    D = 4 * p * (p - 1)
    lD = (D + 3) * (D + 2) * (D + 1) // 6
    g = torch.zeros(ld, dtype=torch.int32, device=dev)
    G = torch.zeros(lD, dtype=torch.int32, device=dev)
    delta = torch.zeros(lD, dtype=torch.int32, device=dev)
    iters = torch.zeros(max(max_h - 1, 1), ld, dtype=torch.int32, device=dev)
    h = torch.zeros(1, dtype=torch.int8, device=dev)
    torch.cuda.synchronize(dev)
    fcode = (FORMS[form] if isinstance(form, str) else int(form)) | (POWERS[power] << 8)
    rc = _lib().qfs_debug_stages(int(p), coeffs.data_ptr(), int(max_h), fcode, g.data_ptr(), G.data_ptr(),
                                 delta.data_ptr(), iters.data_ptr(), h.data_ptr())
    _check(rc, "qfs_debug_stages")
    return dict(h=int(h.item()), g=g, G=G, delta=delta, iters=iters)
