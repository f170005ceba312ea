#!/usr/bin/env python3
"""Throughput of quasi-F-split height classification on GB300: quartics per second, bit-exact.

One step = one pass of the whole hot path (f^(p-1), Fedder test, power chain to f^(p(p-1)) mod p^2, Delta_1,
theta iterations with early exit) over one batch of seeded random quartics, the paper's own workload (Sec. 7.1):
coefficients uniform in F_p^35.  The headline workload is p = 7, 262,144 quartics; the same run also times
p = 5, 65,536 quartics and every arithmetic form.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--form dp4a|int32|int8tc]

Multi-GPU (one rank per GPU): every rank classifies its own n quartics (rows rank*n .. rank*n+n-1 of the same
generator); there is no data-path collective, the ranks only meet for the barrier and the max-time reduction
("scaling": "weak").  Launched by torchrun, the ranks come from its environment; `--gpus N` without it re-runs this
script under torch.distributed.run with N ranks (N at most the visible GPU count).  --impl reference times the CPU
oracle (the literal Algorithms 1-3) on the host.

Parity: while the GPU is timed, a separate process runs the oracle (route R, every host core but one) over every
row of every workload the run launches, and the line's "parity" entries count the rows checked and the mismatches
per workload, form and mode.
"""
import argparse
import hashlib
import json
import multiprocessing
import os
import socket
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2502_12428_gb300 import inputs  # noqa: E402

METRIC = "quartics/sec height-classified at p=5,7 (1 GB300), bit-exact; int8-TC vs int32 form"
HEADLINE_CFG = 4        # p = 7, 262,144 dense quartics
SECOND_CFG = 2          # p = 5, 65,536 dense quartics
PAPER_P7_RATE = 185.0   # surfaces/s at p = 7, paper Sec. 7.2 (2080 Ti; context, other hardware)
# integer MAC lanes per SM per clock of each form's instruction (4 SMSPs x 16 lanes; an IDP4A lane does 4 MACs;
# mma.sync m16n8k32 s8 is rated like IDP4A); SM count and maximum clock are read from the device
LANES = {"int32": 64, "dp4a": 64 * 4, "int8tc": 64 * 4}
# which measured rate of qfs_int_peaks bounds each form
PEAK_KIND = {"int32": "imad", "dp4a": "dp4a", "int8tc": "mma_s8"}
CPU_SAMPLE_A = 1024     # route-A quartics of the CPU baseline (about half a minute on 16 cores at p = 7)

def hbm_peak():
    """The measured HBM copy rate of this machine's GB300 (MEASURED_PEAKS.json, driver-written), else the fallback."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            return {"gbs": float(json.load(fh)["hbm_gbs"]), "basis": "measured copy rate (MEASURED_PEAKS.json)"}
    except (OSError, KeyError, ValueError):
        return {"gbs": 6800.0, "basis": "fallback 6.8 TB/s (no measured copy rate present)"}


HBM_PEAK = hbm_peak()


# ----------------------------------------------------------------------------------------------- work counts
def n_mon(d):
    return (d + 3) * (d + 2) * (d + 1) // 6 if d >= 0 else 0


def chain_macs(p, k_from, k_to):
    """MACs of f^(k+1) = f^k * f for k in [k_from, k_to]: every term of f^k meets each of f's 35 terms once."""
    return sum(n_mon(4 * k) * 35 for k in range(k_from, k_to + 1))


def theta_nnz(p):
    """Nonzero entries of the matrix of g -> u(Delta g) on degree-4(p-1) forms: pairs (r, c) whose Delta index
    p r + (p-1) - c has no negative exponent (Sec. 4, matching monomials)."""
    d = 4 * (p - 1)
    mons = np.array([(e1, e2, e3, d - e1 - e2 - e3) for e1 in range(d, -1, -1) for e2 in range(d - e1, -1, -1)
                     for e3 in range(d - e1 - e2, -1, -1)], np.int64)
    total = 0
    for chunk in np.array_split(np.arange(len(mons)), max(1, len(mons) // 256)):
        e = p * mons[chunk][:, None, :] + (p - 1) - mons[None, :, :]
        total += int((e >= 0).all(axis=2).sum())
    return total


def algorithmic_macs(p, n, survivors, theta_steps):
    a2 = chain_macs(p, 1, p - 2)
    a4 = chain_macs(p, p - 1, p * (p - 1) - 1)
    return n * a2 + survivors * a4 + theta_steps * theta_nnz(p)


def tc_tiles(m_out):
    """mma.sync tiles of one chain product of the int8 tensor form (ring_chain_step): per 32-column block and output
    slice u, each 16-column group runs one tile per word pair (8 outputs) of its longest existing column."""
    t = 0
    for s0 in range(0, m_out + 1, 32):
        s_last = min(s0 + 31, m_out)
        for u in range(s0, m_out + 1):
            hi = min(s_last, u)
            for grp in (0, 1):
                sg = s0 + 16 * grp
                if sg <= hi:
                    t += min(hi, sg + 15) // 8 + 1
    return t


def tc_executed_macs_per_survivor(p):
    """MACs the int8 tensor form's mma.sync tiles execute for one quartic past the height-1 screen: every chain
    product f~^(k+1) = f~^k f~, k = 1 .. p(p-1)-1, at 8 x m16n8k32 (8 x 4096 MACs) per tile."""
    return sum(tc_tiles(4 * k + 4) for k in range(1, p * (p - 1))) * 8 * 4096


# ----------------------------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        mhz = [float(r[1]) for r in self.rows if len(r) >= 9 and r[1].replace(".", "").isdigit()]
        if not mhz:
            return None
        maxmhz = max(float(r[2]) for r in self.rows if len(r) >= 9 and r[2].replace(".", "").isdigit())
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows if len(r) >= 9 for i in range(4) if r[5 + i] == "Active"})
        return {"sm_mhz": statistics.median(mhz), "sm_max_mhz": maxmhz, "reasons": reasons, "samples": len(mhz)}


# ----------------------------------------------------------------------------------------------- helpers
# the sources the fused dp4a kernel is compiled from (its launch shape comes from qfs_api.cu's occupancy query)
FUSED_KERNEL_SOURCES = ("qfs_layout.cuh", "qfs_common.cuh", "qfs_sweep.cuh", "qfs_engine.cuh", "qfs_kernels.cuh",
                        "qfs_form_dp4a.cu")


def kernel_source_hash():
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2502_12428_gb300", "csrc")
    for f in FUSED_KERNEL_SOURCES:
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic(form, workload):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on the current kernel sources."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as fh:
        data = json.load(fh)
    ent = data.get(form, {}).get(workload)
    if not ent or ent.get("kernel_hash") != kernel_source_hash():
        return None
    return ent.get("dram_bytes_per_launch")


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def init_ranks(backend, world):
    """One process group over the launch's ranks (none for a single rank)."""
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group(backend, init_method="env://")


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world, device="cpu"):
    """The largest value of x over the ranks (every rank gets it): step times are the slowest rank's."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def free_port():
    with socket.socket() as so:
        so.bind(("127.0.0.1", 0))
        return so.getsockname()[1]


def torchrun_argv(n, argv, port):
    """The command that runs this script with n ranks on this node (one per GPU), rendezvous on 127.0.0.1."""
    return [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={n}",
            "--master-addr", "127.0.0.1", f"--master-port={port}", os.path.abspath(__file__), *argv]


def config_batch(cfg, rank=0):
    (p, n, kind), = inputs.CONFIG_SIZES[cfg]
    seed = inputs.config_seed(cfg)
    if kind == "dense+fermat":
        f = np.concatenate([inputs.dense(p, n, seed, row0=rank * n), inputs.fermat()[None]])
        return p, n + 1, kind, f
    gen = inputs.sparse if kind == "sparse" else inputs.dense
    return p, n, kind, gen(p, n, seed, row0=rank * n)


def mixed_batch(rank=0):
    """Mixed-prime workload: 131,072 quartics at p = 5, 131,072 at p = 7 and 4,096 at p = 11, each followed by its
    image under a random PGL_4(F_p) change of variables (so every group holds 2n rows)."""
    groups, total = [], 0
    seed = inputs.config_seed(5)
    for p, n, kind in inputs.CONFIG_SIZES[5]:
        f = inputs.dense(p, n, seed + p, row0=rank * n)
        A = inputs.pgl4_matrices(p, n, seed + 100 + p, row0=rank * n)
        groups.append((p, np.concatenate([f, inputs.substitute(f, A, p)])))
        total += 2 * n
    return groups, total


def workload_name(cfg):
    (p, n, kind), = inputs.CONFIG_SIZES[cfg]
    return f"p{p}-{kind}-{n}"


# ----------------------------------------------------------------------------------------------- oracle parity
def parity_workloads(rank):
    """Every batch the GPU arm launches, by name: (p, rows, oracle route)."""
    out = {}
    p, n, kind, f = config_batch(1, rank)
    out[workload_name(1)] = (p, f, "A")
    for cfg in (2, 3, 4):
        p, n, kind, f = config_batch(cfg, rank)
        out[workload_name(cfg)] = (p, f, "R")
    groups, _ = mixed_batch(rank)
    for p, f in groups:
        out[f"mixed-pgl4 p{p}"] = (p, f, "R")
    return out


def oracle_job(rank, threads, path):
    """Oracle heights of every parity workload (runs in its own process, started with spawn)."""
    import oracle
    oracle.build()
    res, secs = {}, {}
    for name, (p, f, route) in parity_workloads(rank).items():
        t0 = time.perf_counter()
        res[name] = oracle.heights(p, f, route=oracle.ROUTE_A if route == "A" else oracle.ROUTE_R, threads=threads)
        secs[name] = time.perf_counter() - t0
    tmp = path + ".tmp.npz"
    np.savez(tmp, **{k.replace(" ", "__"): v for k, v in res.items()})
    os.replace(tmp, path)
    with open(path + ".json", "w") as fh:
        json.dump({"seconds": secs, "threads": threads}, fh)


def parity_entries(gpu_outputs, oracle_path):
    """[{workload, form, mode, checked, mismatches}] for every GPU output kept, against the oracle's heights."""
    want = dict(np.load(oracle_path))
    want = {k.replace("__", " "): v for k, v in want.items()}
    out = []
    for (name, form, mode), got in gpu_outputs:
        w = want[name]
        out.append({"workload": name, "form": form, "mode": mode, "checked": int(w.size),
                    "mismatches": int((got != w).sum()) if got.shape == w.shape else int(w.size)})
    return out


# ----------------------------------------------------------------------------------------------- GPU arm
def run_ours(args):
    import torch
    import paper_2502_12428_gb300.qfs as qfs
    from paper_2502_12428_gb300 import build as qbuild

    world, rank, local = dist_setup()
    # the oracle process starts before this process touches CUDA (spawn: it shares nothing with it)
    oracle_proc, oracle_path, tmpdir = None, None, None
    if rank == 0 and not args.no_parity:
        tmpdir = tempfile.mkdtemp(prefix="qfs_parity_")
        oracle_path = os.path.join(tmpdir, "oracle.npz")
        threads = max(1, (os.cpu_count() or 2) - 1)
        oracle_proc = multiprocessing.get_context("spawn").Process(target=oracle_job,
                                                                   args=(rank, threads, oracle_path))
        oracle_proc.start()
    if world > 1:
        torch.cuda.set_device(local)
    init_ranks("nccl", world)
    dev = torch.device("cuda", torch.cuda.current_device())
    if rank == 0:
        qbuild.build()
    barrier(world)
    qfs.lib()
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)  # > L2 (129 MB)
    peaks = qfs.int_peaks()     # measured IMAD / IDP4A / mma.sync s8 rates, SM count, maximum SM clock
    sms, max_mhz = peaks["sms"], peaks["max_mhz"]
    keep = []                   # (workload, form, mode) -> heights, for the parity check

    def mx(x):
        return max_over_ranks(x, world, dev)

    def timed_steps(p, coeffs, form, steps, warmup, engine=None, power=None):
        out = torch.empty(coeffs.shape[0], dtype=torch.int8, device=dev)
        for _ in range(warmup):
            qfs.heights(p, coeffs, out=out, form=form, engine=engine, power=power)
        torch.cuda.synchronize()
        qfs.read_stats()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        barrier(world)
        torch.cuda.synchronize()
        for i in range(steps):
            flush.fill_(i & 0xFF)                # L2 flush between timed steps, outside the events
            ev[i][0].record(stream)
            qfs.heights(p, coeffs, out=out, form=form, engine=engine, power=power)
            ev[i][1].record(stream)
        torch.cuda.synchronize()
        barrier(world)
        per = [a.elapsed_time(b) for a, b in ev]
        survivors, theta = qfs.read_stats()
        return out, per, survivors / steps, theta / steps

    def nominal_peak(form):
        return sms * LANES[form] * max_mhz * 1e6 * 2 / 1e12

    def measured_peak(form):
        return 2 * peaks[PEAK_KIND[form]] / 1e12

    result = {}
    forms = [args.form] + [f for f in ("int32", "dp4a", "int8tc") if f != args.form and f in args.forms]
    # headline: timed with the clock sampler running
    p, n, kind, f_np = config_batch(HEADLINE_CFG, rank)
    coeffs = torch.from_numpy(f_np).to(dev)
    hname = workload_name(HEADLINE_CFG)
    sampler = ClockSampler(dev.index) if rank == 0 else None
    if sampler:
        sampler.start()
    out, per, surv, theta = timed_steps(p, coeffs, args.form, args.steps, args.warmup)
    clocks = sampler.stop() if sampler else None
    ms_step = mx(statistics.mean(per))
    heights_np = out.cpu().numpy()
    keep.append(((hname, args.form, "chain"), heights_np))
    value = world * n / (ms_step / 1e3)
    macs = algorithmic_macs(p, n, surv, theta)
    achieved = 2 * macs / (statistics.mean(per) / 1e3) / 1e12
    peak = nominal_peak(args.form)
    traffic = profiled_traffic(args.form, hname)
    roofline = {"bound": "alu", "achieved": round(achieved, 3), "peak": round(peak, 1), "unit": "TOP/s",
                "frac": round(achieved / peak, 4), "traffic": traffic,
                "kernel": f"qfs::fused_kernel<{ {'int32': 0, 'dp4a': 1, 'int8tc': 2}[args.form]}>",
                "ops_per_launch": 2 * macs,
                "duration_basis": "CUDA events around the call on its stream: the height-1 screen (about 0.5 % "
                                  "of the launch list) and the persistent kernel",
                "peak_basis": f"{sms} SMs x {LANES[args.form]} int MAC lanes x {max_mhz:.0f} MHz x 2 ops (nominal; "
                              f"SM count and maximum clock read from the device; 1 MAC = 2 ops)",
                "peak_measured": round(measured_peak(args.form), 1),
                "frac_of_measured": round(achieved / measured_peak(args.form), 4),
                "peak_measured_basis": f"qfs_int_peaks in this run: independent {PEAK_KIND[args.form]} chains, "
                                       f"8 CTAs x 256 threads per SM, best of 3"}

    forms_out = {args.form: {"value": round(value, 1), "ms_per_step": round(ms_step, 3),
                             "frac_of_alu_peak": roofline["frac"],
                             "frac_of_measured_peak": roofline["frac_of_measured"]}}
    for form in forms[1:]:
        try:
            o2, per2, s2, t2 = timed_steps(p, coeffs, form, max(2, args.steps // 2), args.warmup)
        except qfs.QfsError as e:
            forms_out[form] = {"unavailable": str(e)}
            continue
        ms2 = mx(statistics.mean(per2))
        sec2 = statistics.mean(per2) / 1e3
        alg2 = algorithmic_macs(p, n, s2, t2)
        o2np = o2.cpu().numpy()
        keep.append(((hname, form, "chain"), o2np))
        ent = {"value": round(world * n / (ms2 / 1e3), 1), "ms_per_step": round(ms2, 3),
               "frac_of_alu_peak": round(2 * alg2 / sec2 / 1e12 / nominal_peak(form), 4),
               "frac_of_measured_peak": round(2 * alg2 / sec2 / 1e12 / measured_peak(form), 4),
               "bit_exact_vs_headline_form": bool(np.array_equal(o2np, heights_np))}
        if form == "int8tc":
            # the tensor pipe's own work: every chain product of every quartic past the screen, as mma.sync tiles
            ex = s2 * tc_executed_macs_per_survivor(p)
            ent.update({"algorithmic_macs": alg2, "tensor_executed_macs": ex,
                        "tensor_executed_frac_of_measured_mma": round(2 * ex / sec2 / 1e12 / measured_peak(form), 4),
                        "useful_fraction_of_tensor_macs": round(s2 * chain_macs(p, 1, p * (p - 1) - 1) / ex, 4)})
        forms_out[form] = ent

    # second workload (p = 5)
    p5, n5, kind5, f5 = config_batch(SECOND_CFG, rank)
    c5 = torch.from_numpy(f5).to(dev)
    second = {"workload": workload_name(SECOND_CFG)}
    for form in forms:
        try:
            o5, per5, s5, t5 = timed_steps(p5, c5, form, args.steps, args.warmup)
        except qfs.QfsError as e:
            second[form] = {"unavailable": str(e)}
            continue
        keep.append(((workload_name(SECOND_CFG), form, "chain"), o5.cpu().numpy()))
        ms5 = mx(statistics.mean(per5))
        second[form] = {"value": round(world * n5 / (ms5 / 1e3), 1), "ms_per_step": round(ms5, 3)}

    # the 65-quartic p = 3 workload (the oracle's route A checks it): every form, untimed
    p1, n1, kind1, f1 = config_batch(1, rank)
    c1 = torch.from_numpy(f1).to(dev)
    for form in forms:
        keep.append(((workload_name(1), form, "chain"), qfs.heights(p1, c1, form=form).cpu().numpy()))

    # the other workloads, each timed in the headline form: sparse p = 5 (uneven work) and the mixed-prime batch
    # with PGL_4 images in one launch; and the staged engine on the headline workload
    extra = {}
    if not args.no_extra:
        p3, n3, kind3, f3 = config_batch(3, rank)
        c3 = torch.from_numpy(f3).to(dev)
        o3, per3, s3, t3 = timed_steps(p3, c3, args.form, max(2, args.steps // 2), args.warmup)
        ms3 = mx(statistics.mean(per3))
        keep.append(((workload_name(3), args.form, "chain"), o3.cpu().numpy()))
        extra[workload_name(3)] = {"value": round(world * n3 / (ms3 / 1e3), 1), "ms_per_step": round(ms3, 3),
                                   "past_height_1": s3, "theta_steps": t3}
        for form in forms[1:]:      # the other forms once each, for the parity check (the tensor form timed)
            if form == "int8tc":
                o3t, per3t, _, _ = timed_steps(p3, c3, form, max(2, args.steps // 2), args.warmup)
                ms3t = mx(statistics.mean(per3t))
                keep.append(((workload_name(3), form, "chain"), o3t.cpu().numpy()))
                extra[workload_name(3) + " form=int8tc"] = {"value": round(world * n3 / (ms3t / 1e3), 1),
                                                             "ms_per_step": round(ms3t, 3)}
            else:
                keep.append(((workload_name(3), form, "chain"), qfs.heights(p3, c3, form=form).cpu().numpy()))
        # the same workload replayed from a captured CUDA graph (the height-1 screen and the persistent launch);
        # the call allocates nothing once the workspace exists, so it captures as it is
        out3g = torch.empty(n3, dtype=torch.int8, device=dev)
        qfs.heights(p3, c3, out=out3g, form=args.form)
        torch.cuda.synchronize()
        g3 = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g3):
            qfs.heights(p3, c3, out=out3g, form=args.form)
        for _ in range(args.warmup):
            g3.replay()
        torch.cuda.synchronize()
        barrier(world)
        evg = []
        for i in range(max(2, args.steps // 2)):
            flush.fill_(i & 0xFF)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            g3.replay()
            b.record(stream)
            evg.append((a, b))
        torch.cuda.synchronize()
        msg = mx(statistics.mean(a.elapsed_time(b) for a, b in evg))
        extra[workload_name(3) + " cuda graph"] = {
            "value": round(world * n3 / (msg / 1e3), 1), "ms_per_step": round(msg, 3),
            "bit_exact_vs_launch": bool(np.array_equal(out3g.cpu().numpy(), o3.cpu().numpy()))}
        del g3
        groups5, n5tot = mixed_batch(rank)
        dev_groups = [(p_, torch.from_numpy(f_).to(dev), None) for p_, f_ in groups5]
        for _ in range(args.warmup):
            qfs.heights_multi(dev_groups, form=args.form)
        torch.cuda.synchronize()
        barrier(world)
        ev5 = []
        for i in range(max(2, args.steps // 2)):
            flush.fill_(i & 0xFF)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            outs5 = qfs.heights_multi(dev_groups, form=args.form)
            b.record(stream)
            ev5.append((a, b))
        torch.cuda.synchronize()
        ms5 = mx(statistics.mean(a.elapsed_time(b) for a, b in ev5))
        invariant = all(np.array_equal(o.cpu().numpy()[:len(f_) // 2], o.cpu().numpy()[len(f_) // 2:])
                        for o, (p_, f_) in zip(outs5, groups5))
        for o, (p_, f_) in zip(outs5, groups5):
            keep.append(((f"mixed-pgl4 p{p_}", args.form, "chain"), o.cpu().numpy()))
        for form in forms[1:]:
            for o, (p_, f_) in zip(qfs.heights_multi(dev_groups, form=form), groups5):
                keep.append(((f"mixed-pgl4 p{p_}", form, "chain"), o.cpu().numpy()))
        extra["mixed-p5-p7-p11-pgl4"] = {"value": round(world * n5tot / (ms5 / 1e3), 1), "ms_per_step": round(ms5, 3),
                                         "quartics": n5tot, "pgl4_invariant": bool(invariant)}
        # the other power modes on the headline workload (bit-identical heights; the reduced mode never forms
        # Delta_1(f^(p-1)), see include/qfs.h)
        for power in ("identity", "reduced"):
            om, per_m, sm_, tm_ = timed_steps(p, coeffs, args.form, max(2, args.steps // 2), args.warmup,
                                              power=power)
            msm = mx(statistics.mean(per_m))
            omnp = om.cpu().numpy()
            keep.append(((hname, args.form, power), omnp))
            extra[hname + f" power={power}"] = {
                "value": round(world * n / (msm / 1e3), 1), "ms_per_step": round(msm, 3),
                "bit_exact_vs_chain": bool(np.array_equal(omnp, heights_np))}
        o3r, per3r, _, _ = timed_steps(p3, c3, args.form, max(2, args.steps // 2), args.warmup, power="reduced")
        ms3r = mx(statistics.mean(per3r))
        keep.append(((workload_name(3), args.form, "reduced"), o3r.cpu().numpy()))
        extra[workload_name(3) + " power=reduced"] = {"value": round(world * n3 / (ms3r / 1e3), 1),
                                                      "ms_per_step": round(ms3r, 3),
                                                      "bit_exact_vs_chain": bool(np.array_equal(o3r.cpu().numpy(),
                                                                                                o3.cpu().numpy()))}
        os_, per_s, ss, ts = timed_steps(p, coeffs, "dp4a", 2, args.warmup, engine="staged")
        keep.append(((hname, "dp4a", "staged engine"), os_.cpu().numpy()))
        extra[hname + " staged engine"] = {
            "value": round(world * n / (mx(statistics.mean(per_s)) / 1e3), 1),
            "ms_per_step": round(mx(statistics.mean(per_s)), 3),
            "bit_exact_vs_fused": bool(np.array_equal(os_.cpu().numpy(), heights_np))}
        # theta-matrix export (Sec. 3.4's M, every quartic): the first 2 x SMs quartics of the headline workload
        nm = 2 * sms
        sub = coeffs[:nm].contiguous()
        ld = (4 * p - 1) * (4 * p - 2) * (4 * p - 3) // 6
        mbuf = torch.empty(nm, ld, ld, dtype=torch.uint8, device=dev)
        qfs.theta_matrix(p, sub, out=mbuf)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        qfs.theta_matrix(p, sub, out=mbuf)
        e1.record(stream)
        torch.cuda.synchronize()
        msm = mx(e0.elapsed_time(e1))
        extra[hname + " theta-matrix export"] = {
            "value": round(world * nm / (msm / 1e3), 1), "unit": "matrices/s", "ms": round(msm, 3),
            "quartics": nm, "matrix_bytes": ld * ld}
        del mbuf
        # matrix multiplication mod 11 (Sec. 5 sizes): one warm-up and one timed product per size
        for nmm in (5000, 10000, 20000):
            g = torch.Generator(device=dev).manual_seed(nmm)
            A = torch.randint(0, 11, (nmm, nmm), dtype=torch.uint8, device=dev, generator=g)
            B = torch.randint(0, 11, (nmm, nmm), dtype=torch.uint8, device=dev, generator=g)
            Cm = torch.empty(nmm, nmm, dtype=torch.uint8, device=dev)
            qfs.matmul_mod(11, A, B, out=Cm)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            qfs.matmul_mod(11, A, B, out=Cm)
            e1.record(stream)
            torch.cuda.synchronize()
            msm = mx(e0.elapsed_time(e1))
            extra[f"matmul-mod11-{nmm}"] = {"seconds": round(msm / 1e3, 5), "unit": "s per product",
                                            "tops": round(2.0 * nmm ** 3 / (msm / 1e3) / 1e12, 2),
                                            "frac_of_measured_mma": round(nmm ** 3 / (msm / 1e3) / peaks["mma_s8"],
                                                                          4)}
            del A, B, Cm
        # exact powering over Z (Sec. 4 workload): degree-16 form, coefficients in {0..4}, powers 5, 10, 15
        rng = np.random.default_rng(16)
        f16 = rng.integers(0, 5, 969).astype(np.uint32)
        for npow in (5, 10, 15):
            n_out = (16 * npow + 3) * (16 * npow + 2) * (16 * npow + 1) // 6
            limbs = torch.empty(n_out, 8, dtype=torch.int32, device=dev)
            qfs.poly_power_limbs(16, f16, npow, out=limbs)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            qfs.poly_power_limbs(16, f16, npow, out=limbs)
            e1.record(stream)
            torch.cuda.synchronize()
            sec = mx(e0.elapsed_time(e1)) / 1e3
            plan = qfs.poly_power_info(16, f16, npow)
            gbs = plan["hbm_bytes"] / sec / 1e9
            extra[f"poly-power-deg16-n{npow}"] = {
                "seconds": round(sec, 5), "unit": "s per power", "output_terms": n_out, "primes": plan["nprimes"],
                "transform_len": plan["transform_len"],
                "roofline": {"bound": "hbm", "achieved": round(gbs, 1), "unit": "GB/s",
                             "peak": HBM_PEAK["gbs"], "peak_basis": HBM_PEAK["basis"],
                             "frac": round(gbs / HBM_PEAK["gbs"], 4), "traffic": None,
                             "bytes_per_call": plan["hbm_bytes"],
                             "bytes_basis": "qfs_poly_power_info: reads + writes of every kernel as launched"}}
            del limbs

    # end to end through the public API: pinned host input -> H2D -> heights -> D2H, every step
    host_in = torch.from_numpy(f_np).pin_memory()
    host_out = torch.empty(n, dtype=torch.int8).pin_memory()
    dev_in = torch.empty_like(coeffs)
    dev_out = torch.empty(n, dtype=torch.int8, device=dev)
    for _ in range(args.warmup):
        dev_in.copy_(host_in, non_blocking=True)
        qfs.heights(p, dev_in, out=dev_out, form=args.form)
        host_out.copy_(dev_out, non_blocking=True)
    torch.cuda.synchronize()
    barrier(world)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        dev_in.copy_(host_in, non_blocking=True)
        qfs.heights(p, dev_in, out=dev_out, form=args.form)
        host_out.copy_(dev_out, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    e2e_ms = mx(e0.elapsed_time(e1) / args.steps)
    assert np.array_equal(host_out.numpy(), heights_np)

    if rank == 0:
        parity, parity_basis, oracle_secs = None, None, None
        if oracle_proc is not None:
            oracle_proc.join()
            if oracle_proc.exitcode == 0 and os.path.exists(oracle_path):
                parity = parity_entries(keep, oracle_path)
                with open(oracle_path + ".json") as fh:
                    oracle_secs = json.load(fh)
                parity_basis = (f"every row of every workload this run launched, against the CPU oracle (route A for "
                                f"{workload_name(1)}, route R for the others) on {oracle_secs['threads']} host "
                                f"threads, run in a separate process while the GPU was timed")
            else:
                parity_basis = f"oracle process failed (exit code {oracle_proc.exitcode})"
        hist = np.bincount(heights_np.astype(np.int64) + 1, minlength=12)
        result = {
            "metric": METRIC, "value": round(value, 1), "unit": "quartics/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_step, 3),
            "higher_is_better": True, "scaling": "weak",
            "vs_baseline": round(value / PAPER_P7_RATE, 1),
            "vs_baseline_basis": "paper Sec. 7.2: about 185 surfaces/s at p=7 on 2080 Ti GPUs (other hardware)",
            "dtype": "int8" if args.form != "int32" else "int32", "data": "synthetic",
            "config": {"workload": hname, "p": p, "quartics_per_gpu": n,
                       "coefficients": "uniform in F_7, splitmix64 seed 0x5EED0004", "max_h": 10,
                       "form": args.form, "engine": "fused persistent", "l2": "flushed between timed steps",
                       "parallelism": f"replicas x{world}"},
            "forms": forms_out, "second_workload": second, "other_workloads": extra,
            "heights_histogram": {"invalid": int(hist[0]), "inf": int(hist[1]),
                                  **{str(h): int(hist[h + 1]) for h in range(1, 11)}},
            "work_per_step": {"past_height_1": surv, "theta_steps": theta, "algorithmic_macs": macs},
            "roofline": roofline,
            "measured_int_peaks": {"imad_tmac_s": round(peaks["imad"] / 1e12, 2),
                                   "dp4a_tmac_s": round(peaks["dp4a"] / 1e12, 2),
                                   "mma_s8_tmac_s": round(peaks["mma_s8"] / 1e12, 2), "sms": sms,
                                   "max_sm_mhz": max_mhz},
            "parity": parity, "parity_basis": parity_basis,
            "parity_mismatches_total": None if parity is None else sum(e["mismatches"] for e in parity),
            "e2e": {"value": round(world * n / (e2e_ms / 1e3), 1), "unit": "quartics/s",
                    "h2d_bytes_per_step": int(n * 35), "d2h_bytes_per_step": int(n)},
            "gpu_launches": 2 * args.steps,   # per step: the height-1 screen and the persistent fused kernel
            "clocks": clocks,
        }
        if not args.no_cpu_baseline:
            result["cpu_baseline"] = cpu_baseline(p, f_np, args.cpu_sample or CPU_SAMPLE_A, oracle_secs, hname, n)
        if tmpdir:
            for fn in os.listdir(tmpdir):
                os.remove(os.path.join(tmpdir, fn))
            os.rmdir(tmpdir)
        print(json.dumps(result), flush=True)
    barrier(world)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


# ----------------------------------------------------------------------------------------------- CPU oracle
def cpu_baseline(p, f_np, sample, oracle_secs, hname, n):
    """Route A (the literal Algorithms 1-3) on the first `sample` quartics of the headline workload, on every host
    core; plus the rate of route R over the whole workload, taken from the parity run."""
    import oracle
    cores = os.cpu_count() or 1
    rows = f_np[:sample]
    t0 = time.perf_counter()
    oracle.heights(p, rows, route=oracle.ROUTE_A, threads=cores)
    dt = time.perf_counter() - t0
    out = {"value": round(sample / dt, 3), "unit": "quartics/s", "cores": cores, "kind": "oracle",
           "sample": f"first {sample} quartics of the same workload, route A (literal Algorithms 1-3), "
                     f"{cores} threads, {dt:.1f} s"}
    if oracle_secs and hname in oracle_secs["seconds"]:
        sec = oracle_secs["seconds"][hname]
        out["route_r_full_set"] = {"value": round(n / sec, 1), "unit": "quartics/s", "cores": oracle_secs["threads"],
                                   "kind": "oracle", "sample": f"all {n} quartics of the workload, route R (reduced "
                                   f"derivation), {sec:.1f} s, while the GPU arm ran"}
    return out


def run_reference(args):
    world, rank, local = dist_setup()
    init_ranks("gloo", world)
    if rank == 0:
        import oracle
        oracle.build()
        p, n, kind, f_np = config_batch(HEADLINE_CFG, 0)
        cores = os.cpu_count() or 1
        sample = args.cpu_sample or 128
        per = []
        for i in range(args.warmup + args.steps):
            rows = f_np[(i * sample) % n:][:sample]
            t0 = time.perf_counter()
            oracle.heights(p, rows, route=oracle.ROUTE_A, threads=cores)
            if i >= args.warmup:
                per.append(time.perf_counter() - t0)
        ms = 1e3 * statistics.mean(per)
        value = sample / (ms / 1e3)
        print(json.dumps({
            "impl": "reference", "metric": METRIC, "value": round(value, 3), "unit": "quartics/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 1), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": {"workload": workload_name(HEADLINE_CFG), "p": p, "max_h": 10, "sample_per_step": sample},
            "cpu_baseline": {"value": round(value, 3), "unit": "quartics/s", "cores": cores, "kind": "oracle",
                             "sample": f"{sample} quartics of the workload per step, route A"},
            "e2e": {"value": round(value, 3), "unit": "quartics/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0},
        }), flush=True)
    # the other ranks do no work; every rank leaves together
    barrier(world)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_ncu_case(args):
    """A small fixed launch for profilers: p = 7, the first --ncu-quartics quartics of the headline workload,
    one warm-up launch and one profiled launch of the fused kernel."""
    import torch
    import paper_2502_12428_gb300.qfs as qfs
    from paper_2502_12428_gb300 import build as qbuild
    qbuild.build()
    p, n, kind, f_np = config_batch(HEADLINE_CFG, 0)
    coeffs = torch.from_numpy(f_np[:args.ncu_quartics]).cuda()
    for _ in range(2):
        h = qfs.heights(p, coeffs, form=args.form, max_ctas=args.ncu_ctas, engine=args.engine, power=args.power)
    torch.cuda.synchronize()
    print(json.dumps({"ncu_case": workload_name(HEADLINE_CFG), "quartics": args.ncu_quartics, "form": args.form,
                      "engine": args.engine or "fused", "power": args.power or "chain",
                      "past_height_1": int((h.cpu().numpy() != 1).sum())}))


def run_powering_case(args):
    """A small fixed launch sequence for profilers: two calls of the exact powering f^n (the bench's degree-16 form
    with coefficients in {0..4}), n = --ncu-powering."""
    import torch
    import paper_2502_12428_gb300.qfs as qfs
    from paper_2502_12428_gb300 import build as qbuild
    qbuild.build()
    rng = np.random.default_rng(16)
    f16 = rng.integers(0, 5, 969).astype(np.uint32)
    npow = args.ncu_powering
    n_out = (16 * npow + 3) * (16 * npow + 2) * (16 * npow + 1) // 6
    limbs = torch.empty(n_out, 8, dtype=torch.int32, device="cuda")
    for _ in range(2):
        qfs.poly_power_limbs(16, f16, npow, out=limbs)
    torch.cuda.synchronize()
    print(json.dumps({"powering_case": f"deg16-n{npow}", "calls": 2, "output_terms": n_out}))


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--form", choices=["dp4a", "int32", "int8tc"], default="dp4a")
    ap.add_argument("--forms", default="int32,dp4a,int8tc", help="forms timed besides the headline one")
    ap.add_argument("--cpu-sample", type=int, default=None,
                    help=f"quartics per oracle run (default {CPU_SAMPLE_A} for the baseline leg, 128 per reference step)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-parity", action="store_true", help="skip the oracle run over every row")
    ap.add_argument("--no-extra", action="store_true", help="skip the sparse, mixed-prime and staged-engine lines")
    ap.add_argument("--ncu-case", action="store_true", help="run the small profiling case and exit")
    ap.add_argument("--ncu-quartics", type=int, default=8192)
    ap.add_argument("--ncu-powering", type=int, default=0,
                    help="run two exact powerings f^n of the degree-16 bench form (the profiling case) and exit")
    ap.add_argument("--ncu-ctas", type=int, default=0)
    ap.add_argument("--engine", choices=["fused", "staged"], default=None, help="engine of the --ncu-case launch")
    ap.add_argument("--power", choices=["chain", "identity", "reduced"], default=None,
                    help="power mode of the --ncu-case launch")
    args = ap.parse_args()
    args.forms = args.forms.split(",")
    if args.warmup < 3:
        ap.error("--warmup must be at least 3")
    if args.gpus < 1:
        ap.error("--gpus must be at least 1")
    if args.gpus > 1 and "WORLD_SIZE" not in os.environ and not args.ncu_case and not args.ncu_powering:
        # not launched by torchrun: start the N ranks here, one per GPU
        if args.impl == "ours":
            import torch
            visible = torch.cuda.device_count()
            if args.gpus > visible:
                ap.error(f"--gpus {args.gpus} asks for more GPUs than the {visible} visible")
        sys.exit(subprocess.call(torchrun_argv(args.gpus, sys.argv[1:], free_port())))
    if "WORLD_SIZE" in os.environ and int(os.environ["WORLD_SIZE"]) != args.gpus:
        ap.error(f"--gpus {args.gpus} does not match the launcher's WORLD_SIZE {os.environ['WORLD_SIZE']}")
    if args.ncu_powering:
        run_powering_case(args)
    elif args.ncu_case:
        run_ncu_case(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
