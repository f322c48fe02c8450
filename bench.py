#!/usr/bin/env python
"""Benchmark of the GB300 Flip-Flop SRQR library: rank-k approximations per second.

Workload (default): A = U_r diag(sigma) V_r^T + E, m = n = 20000, r = 2000,
sigma_j = j^-1.5 (slow decay), E ~ N(0, 1e-6^2), FP32, target rank k = 200,
oversampling p = 10, FFSRQR_MIXED_BF16X3 arithmetic.  A (1.6 GB) is larger than the
129 MB L2, so no flush is needed between steps.  One step = one call of
ffsrqr_run (all pipeline steps: sketch, QRCP, panel QR, R12 pass, SRQR test,
QR of (R11 R12)^T, A Pi Qhat1 pass, small SVD, U and V).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

The default line runs FFSRQR_MIXED_BF16X3; "modes" beside it times all three
arithmetic modes (plain FP32, TF32x3, BF16x3) on the same matrix and states
each one's singular-value and residual errors against the FP64 oracle run on
the same array.  That oracle run (about 25 s on 16 host cores) is also the
cpu_baseline: the whole workload, measured, no scaling.  --impl reference
times the same oracle run on its own (one step: the runs that happened).
With more than one GPU the replicas run independently (the method has no
data-path exchange).  Prints one JSON line on rank 0.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "rank-k approx/s"
UNIT = "approx/s"
def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--mode", choices=["mixed", "bf16x3", "plain"], default="bf16x3",
                    help="mixed: TF32 sketch and three-product TF32 passes; bf16x3: BF16 sketch and "
                         "three-product split-BF16 passes; plain: FP32 on the CUDA cores")
    ap.add_argument("--decay", choices=["slow", "fast", "geo95"], default="slow",
                    help="sigma_j = j^-1.5 (slow), 0.97^j (fast) or 0.95^j (geo95, the 50000x8000 case)")
    ap.add_argument("--m", type=int, default=20000)
    ap.add_argument("--n", type=int, default=20000)
    ap.add_argument("--k", type=int, default=200)
    ap.add_argument("--p", type=int, default=10)
    ap.add_argument("--e2e-steps", type=int, default=24)
    ap.add_argument("--block", type=int, default=0,
                    help="TRQRCP block size b < k (Alg. 2; the sketch has b + p rows); 0: one block")
    ap.add_argument("--g2-rows", type=int, default=0,
                    help="SRQR test: 0 exact g2, d >= 1 Alg. 4's d-row random estimate")
    ap.add_argument("--no-cpu", action="store_true",
                    help="skip the FP64 oracle run (cpu_baseline and the modes' errors against it)")
    ap.add_argument("--no-modes", action="store_true", help="skip the comparison of the three modes")
    ap.add_argument("--workload", choices=["single", "batch", "hosvd", "sthosvd", "hosvd-core", "rpca", "rsisvd",
                                           "serving"],
                    default="single",
                    help="single: one 20000x20000 problem (default); batch: 256 uneven matrices in one graph; "
                         "hosvd: the three unfoldings of a 400^3 tensor; sthosvd: sequentially truncated HOSVD "
                         "of that tensor; hosvd-core: its HOSVD with the core; rpca: IALM robust PCA of an "
                         "--m x --m matrix; rsisvd: randomized subspace iteration against FFSRQR on the default "
                         "matrix; serving: Poisson request stream")
    ap.add_argument("--duration", type=float, default=10.0, help="serving: seconds of arrivals")
    ap.add_argument("--rate", type=float, default=200.0, help="serving: mean arrivals per second")
    ap.add_argument("--phase-batch", action="store_true",
                    help="serving: batch the small SVDs of requests admitted together")
    return ap.parse_args()


def workload_name(a):
    d = {"slow": "sigma_j=j^-1.5", "fast": "sigma_j=0.97^j", "geo95": "sigma_j=0.95^j"}[a.decay]
    return f"FFSRQR rank-{a.k} of {a.m}x{a.n} FP32, r=2000, {d}, E~N(0,1e-6^2)"


def spectrum(a, r):
    from paper_1803_01982_gb300 import synth
    if a.decay == "slow":
        return synth.slow_decay(r)
    return synth.fast_decay(r, 0.97 if a.decay == "fast" else 0.95)


# --------------------------------------------------------------------------
# CPU oracle baselines of the other workloads
# --------------------------------------------------------------------------
def tucker_cpu_baseline(X_host, ranks, st_method: bool):
    """The FP64 oracle's Tucker decomposition of the same tensor on the host
    cores: (seconds, sample text).  Only the benchmark calls it."""
    import oracle
    from oracle import tucker as otk
    oracle.build()
    t0 = time.perf_counter()
    if st_method:
        otk.sthosvd(X_host, ranks, None, p=5)
    else:
        otk.hosvd(X_host, ranks, p=5)
    return time.perf_counter() - t0, "FP64 oracle on the same tensor, whole decomposition"


def rpca_cpu_baseline(m_full: int):
    """The FP64 oracle's IALM solve (Alg. 9 as the SVD) of a 1000 x 1000 matrix
    of the same recipe, scaled to m_full x m_full by m n rank (the passes over
    the matrix at the rank it converges to): (seconds at m_full, sample text)."""
    import oracle
    from oracle import rpca as orp
    from paper_1803_01982_gb300 import synth
    oracle.build()
    ms = min(1000, m_full)
    M, _, _ = synth.rpca_problem(ms, ms, ms // 10, int(0.05 * ms * ms), seed=1)
    t0 = time.perf_counter()
    orp.rpca(M, kmax=224, tol=1e-6)
    dt = time.perf_counter() - t0
    scale = (m_full / ms) ** 3
    return dt * scale, (f"FP64 oracle IALM solve of the {ms}x{ms} matrix of the same recipe (tol 1e-6), "
                        f"time scaled by m n rank to {m_full}x{m_full}")


def cores_used():
    env = os.environ.get("OMP_NUM_THREADS")
    return int(env) if env else (os.cpu_count() or 1)


# --------------------------------------------------------------------------
# clocks
# --------------------------------------------------------------------------
def clocks_start(dev_index):
    fd, path = tempfile.mkstemp(suffix=".csv")
    os.close(fd)
    q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    try:
        p = subprocess.Popen(["nvidia-smi", f"--id={dev_index}", f"--query-gpu={q}",
                              "--format=csv,noheader,nounits", "-lms", "200"],
                             stdout=open(path, "w"), stderr=subprocess.DEVNULL)
    except OSError:
        p = None
    return p, path


def clocks_stop(p, path):
    if p is None:
        return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
    p.terminate()
    try:
        p.wait(timeout=5)
    except subprocess.TimeoutExpired:
        p.kill()
    sm, smax, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in open(path):
        f = [x.strip() for x in line.split(",")]
        if len(f) < 9:
            continue
        try:
            sm.append(float(f[1]))
            smax.append(float(f[2]))
        except ValueError:
            continue
        for nm, v in zip(names, f[5:9]):
            if v.lower().startswith("active"):
                reasons.add(nm)
    os.unlink(path)
    return {"sm_mhz": statistics.median(sm) if sm else None,
            "sm_max_mhz": max(smax) if smax else None,
            "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------------------
# roofline inputs
# --------------------------------------------------------------------------
def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return d["hbm_gbs"], "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def ncu_traffic(kernel_key, mode):
    """DRAM bytes per launch from the committed ncu summary of this mode's
    tensor-core passes, if it was taken on the current source of the kernel
    (else None)."""
    if mode not in ("mixed", "bf16x3"):
        return None
    path = os.path.join(ROOT, "profiles", "tc_pass_traffic.json" if mode == "mixed" else
                        "tc_pass_bf16_traffic.json")
    src = os.path.join(ROOT, "paper_1803_01982_gb300", "csrc", "tc_gemm.cuh")
    try:
        with open(path) as f:
            d = json.load(f)
        sha = hashlib.sha256(open(src, "rb").read()).hexdigest()
        if d.get("source_sha256") != sha:
            return None
        return d.get("traffic_bytes_per_launch", {}).get(kernel_key)
    except (OSError, ValueError):
        return None


# --------------------------------------------------------------------------
def run_reference(a, rank, world):
    """The FP64 oracle on the whole workload: the same matrix as our arm's
    (generated by the same recipe and seed), one timed run on the host cores.
    A run of the full problem takes minutes, so --steps / --warmup are not
    repeated: the line reports the one step that ran (no warm-up is needed by
    a CPU program whose first touch of its inputs is inside the run)."""
    if rank != 0:
        return
    import numpy as np
    import torch

    import oracle
    from paper_1803_01982_gb300 import synth
    oracle.build()
    r = min(2000, a.m, a.n)
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    A = synth.decayed_torch(a.m, a.n, spectrum(a, r), 1e-6, seed=replica_seed(0), device=dev)
    A64 = A.cpu().numpy().astype(np.float64)
    del A
    t0 = time.perf_counter()
    oracle.ffsrqr(A64, a.k, a.p, seed=0)
    dt = time.perf_counter() - t0
    val = 1.0 / dt
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": a.gpus,
            "steps": 1, "warmup": 0, "ms_per_step": dt * 1e3,
            "requested": {"steps": a.steps, "warmup": a.warmup},
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config(a),
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores_used(), "kind": "oracle",
                             "sample": f"the whole workload ({a.m}x{a.n}, k={a.k}, p={a.p}), one run, "
                                       "no scaling"},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def config(a):
    gb = a.m * a.n * 4 / 1e9
    l2 = (f"inputs larger than L2 (A is {gb:.2f} GB), no flush" if gb > 0.129
          else f"A ({gb * 1e3:.0f} MB) fits in L2; steps run back to back without a flush")
    cfg = {"workload": workload_name(a), "m": a.m, "n": a.n, "k": a.k, "p": a.p,
           "mode": a.mode, "l2": l2, "parallelism": f"replicas x{a.gpus}"}
    if getattr(a, "g2_rows", 0):
        cfg["g2"] = f"d-row estimate, d = {a.g2_rows}"
    if getattr(a, "block", 0):
        cfg["block"] = a.block
    return cfg


def max_over_ranks(x: float, device) -> float:
    """The contract's timing rule across replicas: the max of a per-rank
    scalar over all ranks (x itself on a single rank).  device: where the
    collective's tensor lives (a CUDA device for NCCL, "cpu" for gloo)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return x
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def parse_cpulist(text: str) -> set:
    """The CPUs of a sysfs cpulist such as "0-7,16,18-19"."""
    cpus = set()
    for part in text.strip().split(","):
        part = part.strip()
        if "-" in part:
            lo, hi = part.split("-")
            cpus.update(range(int(lo), int(hi) + 1))
        elif part:
            cpus.add(int(part))
    return cpus


def gpu_local_cpus(index: int):
    """The CPUs of the host memory node that sysfs lists for GPU `index` (via
    nvidia-smi's PCI bus id), or None when that is not known."""
    try:
        bus = subprocess.run(["nvidia-smi", "--query-gpu=pci.bus_id", "--format=csv,noheader", "-i", str(index)],
                             capture_output=True, text=True, timeout=20).stdout.strip().lower()
        if not bus:
            return None
        dom, rest = bus.split(":", 1)
        dev = f"{int(dom, 16):04x}:{rest}"
        with open(f"/sys/bus/pci/devices/{dev}/numa_node") as f:
            node = int(f.read().strip())
        if node < 0:
            return None
        with open(f"/sys/devices/system/node/node{node}/cpulist") as f:
            cpus = parse_cpulist(f.read()) & os.sched_getaffinity(0)
        return cpus or None
    except (OSError, ValueError, subprocess.SubprocessError):
        return None


def replica_seed(rank: int) -> int:
    """Each replica factors its own matrix of the same recipe."""
    return 1 + rank


def run_ours(a, rank, world, local_rank):
    import torch
    import torch.distributed as dist

    from paper_1803_01982_gb300 import ffsrqr, synth
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    mode = {"mixed": ffsrqr.MIXED_TF32X3, "bf16x3": ffsrqr.MIXED_BF16X3, "plain": ffsrqr.PLAIN_FP32}[a.mode]
    r = min(2000, a.m, a.n)
    A = synth.decayed_torch(a.m, a.n, spectrum(a, r), 1e-6, seed=replica_seed(rank), device=str(dev))
    plan = ffsrqr.Plan(a.m, a.n, a.k, a.p, mode, flags=ffsrqr.FLAG_PHASE_TIMES, device=dev,
                       g2_rows=a.g2_rows, b=(a.block or None))
    out = plan.outputs()
    st = torch.cuda.current_stream(dev)
    for _ in range(a.warmup):
        plan.run(A, 0, out)
    torch.cuda.synchronize(dev)
    launches_per_step = ffsrqr.ffsrqr_launch_count(plan._h)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    clk, clk_path = clocks_start(dev.index if dev.index is not None else 0)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    phase_sum = None
    ev0.record(st)
    for i in range(a.steps):
        plan.run(A, 0, out)
        # the plan records alternate runs into alternate event sets: read the
        # previous step's kernel times while this step is already queued, so
        # the device never waits for the host inside the timed region
        if i >= 1:
            ph = ffsrqr.phase_times(plan, back=1)
            phase_sum = ph if phase_sum is None else {k: phase_sum[k] + v for k, v in ph.items()}
    ev1.record(st)
    torch.cuda.synchronize(dev)
    ph = ffsrqr.phase_times(plan, back=0)
    phase_sum = ph if phase_sum is None else {k: phase_sum[k] + v for k, v in ph.items()}
    if world > 1:
        dist.barrier()
    clocks = clocks_stop(clk, clk_path)
    ms = max_over_ranks(ev0.elapsed_time(ev1) / a.steps, dev)
    info = plan.info()
    qrcp_barriers = int(plan.item("ctl")[0, 38].item())  # grid barriers of the sketch QRCP
    value = world * 1000.0 / ms
    phases = {k: v / a.steps for k, v in phase_sum.items()}

    # roofline: the dominant pass kernel (one read of A per launch)
    bytes_per_launch = float(a.m) * a.n * 4
    if mode in (ffsrqr.MIXED_TF32X3, ffsrqr.MIXED_BF16X3):
        keys = ["tc_pass1_kernel", "tc_pass2_kernel", "tc_pass3_kernel"]
    else:
        keys = ["pass1_sketch", "pass2_r12", "pass3_tmp"]
    dom = max(keys, key=lambda k: phases[k])
    peak, peak_src = peaks()
    achieved = bytes_per_launch / (phases[dom] * 1e-3) / 1e9
    roof = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "peak_source": peak_src,
            # the committed counters are scaled to the 20000 x 20000 workload
            "traffic": ncu_traffic(dom, a.mode) if (a.m == 20000 and a.n == 20000) else None,
            "algorithmic_bytes_per_launch": bytes_per_launch}
    three_pass_ms = 3 * bytes_per_launch / (peak * 1e9) * 1e3

    # end to end through the C ABI with host buffers: ffsrqr_pipe_run copies
    # each step's A from pinned host memory (overlapping the previous step's
    # computation) and each step's U, S, V, piv back to pinned host memory
    e2e = None
    if a.e2e_steps > 0:
        # the pinned host buffers are placed on the GPU's own host memory node
        # when sysfs names one (the allocating thread's CPUs decide where the
        # pages go); the affinity is restored afterwards
        local = gpu_local_cpus(local_rank)
        saved = os.sched_getaffinity(0) if local else None
        if local:
            os.sched_setaffinity(0, local)
        try:
            Ah = A.cpu().pin_memory()
            pipe = ffsrqr.Pipe(plan)
            host_out = [pipe.host_outputs() for _ in range(2)]
        finally:
            if saved:
                os.sched_setaffinity(0, saved)
        pipe.run([Ah], [host_out[0]], stream=st)  # warm-up
        torch.cuda.synchronize(dev)
        if world > 1:
            dist.barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        pipe.run([Ah] * a.e2e_steps, [host_out[i % 2] for i in range(a.e2e_steps)], stream=st)
        e1.record(st)
        torch.cuda.synchronize(dev)
        ems = max_over_ranks(e0.elapsed_time(e1) / a.e2e_steps, dev)
        d2h = sum(t.numel() * t.element_size() for t in out)
        e2e = {"value": world * 1000.0 / ems, "unit": UNIT, "h2d_bytes_per_step": A.numel() * 4,
               "d2h_bytes_per_step": d2h, "ms_per_step": ems,
               "host_buffers": (f"pinned on the GPU's node (CPUs {min(local)}-{max(local)})" if local
                                else "pinned, node not pinned (sysfs names none)")}

    # the three arithmetic modes on the same matrix (a few steps each) and
    # their errors against the FP64 oracle run on the same array, which is
    # also the CPU baseline (the whole workload, about 25 s on 16 cores)
    modes, cpu = None, None
    if rank == 0 and world == 1:
        modes = compare_modes(a, A, dev) if not a.no_modes else None
        if not a.no_cpu:
            cpu, ref = oracle_full(a, A)
            if modes:
                mode_errors(a, A, modes, ref)
            cpu.pop("ref", None)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
                "warmup": a.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": config(a),
                "roofline": roof,
                "three_pass_roofline": {"ms": three_pass_ms, "frac_of_step": three_pass_ms / ms},
                "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches_per_step * a.steps,
                "modes": {k: {kk: vv for kk, vv in v.items() if kk != "out"} for k, v in modes.items()}
                if modes else None,
                "clocks": clocks, "phases_ms": {k: round(v, 4) for k, v in phases.items()},
                "status": info["status"], "swaps": info["swaps"], "g2": info["g2_first"],
                "qrcp_barriers": qrcp_barriers}
        print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------
# the three modes side by side, with their errors against the FP64 oracle
# --------------------------------------------------------------------------
MODE_IDS = {"plain": 0, "mixed": 1, "bf16x3": 2}


def compare_modes(a, A, dev, steps=3, warm=2):
    """Each arithmetic mode on the same device matrix: ms per step (CUDA
    events over `steps` back-to-back runs after `warm` warm-up runs) and the
    outputs of one run (kept for mode_errors)."""
    import torch

    from paper_1803_01982_gb300 import ffsrqr
    out = {}
    for name, mid in MODE_IDS.items():
        plan = ffsrqr.Plan(a.m, a.n, a.k, a.p, mid, device=dev)
        res = plan.outputs()
        for _ in range(warm):
            plan.run(A, 0, res)
        torch.cuda.synchronize(dev)
        st = torch.cuda.current_stream(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(steps):
            plan.run(A, 0, res)
        e1.record(st)
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1) / steps
        out[name] = {"ms_per_step": ms, "value": 1000.0 / ms, "status": plan.info()["status"],
                     "out": [t.clone() for t in res]}
        del plan
    return out


def residual_fro_device(A, U, S, V, rows=2048):
    """||A - U diag(S) V^T||_F in FP64 on the device, by row blocks
    (measurement arithmetic, not the factorisation path)."""
    import torch
    U, S, V = U.double(), S.double(), V.double()
    US = U * S
    tot = 0.0
    for r0 in range(0, A.shape[0], rows):
        blk = A[r0:r0 + rows].double() - US[r0:r0 + rows] @ V.T
        tot += float((blk * blk).sum())
    return tot ** 0.5


def oracle_full(a, A):
    """The FP64 oracle on the same array (upcast), timed on the host cores:
    the CPU baseline on the whole workload, no scaling."""
    import numpy as np

    import oracle
    oracle.build()
    A64 = A.cpu().numpy().astype(np.float64)
    t0 = time.perf_counter()
    ref = oracle.ffsrqr(A64, a.k, a.p, seed=0)
    dt = time.perf_counter() - t0
    del A64
    cpu = {"value": 1.0 / dt, "unit": UNIT, "cores": cores_used(), "kind": "oracle",
           "sample": f"the whole workload ({a.m}x{a.n}, k={a.k}, p={a.p}), one run on the same array, no scaling",
           "seconds": dt}
    return cpu, ref


def mode_errors(a, A, modes, ref):
    """Each mode's singular values and Frobenius residual against the FP64
    oracle's (relative), and how much of its column set it shares."""
    import numpy as np
    import torch
    So = ref.S
    head = So >= 0.1 * So[0]
    Ud, Sd, Vd = (torch.from_numpy(x).to(A.device) for x in (ref.U, ref.S, ref.V))
    res_o = residual_fro_device(A, Ud, Sd, Vd)
    for name, m in modes.items():
        U, S, V, piv = m.pop("out")
        Sg = S.double().cpu().numpy()
        rel = np.abs(Sg - So) / So
        res = residual_fro_device(A, U, S, V)
        J = set(piv[:a.k].cpu().numpy().tolist())
        m.update({"sigma_rel_err_head_max": float(rel[head].max()), "sigma_rel_err_max": float(rel.max()),
                  "residual_rel_err": (res - res_o) / res_o,
                  "pivot_set_shared": len(J & set(ref.piv[:a.k].tolist())) / a.k})
    return modes


# --------------------------------------------------------------------------
# batched and serving workloads (one GPU; not the default line)
# --------------------------------------------------------------------------
def _batch_line(a, name, count, ms, roof_bytes, extra):
    from paper_1803_01982_gb300 import ffsrqr  # noqa: F401
    peak, src = peaks()
    t_roof = roof_bytes / (peak * 1e9) * 1e3
    line = {"metric": METRIC, "value": count * 1000.0 / ms, "unit": UNIT, "n_gpus": 1, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": name, "problems_per_step": count},
            "roofline": {"bound": "hbm", "achieved": roof_bytes / (ms * 1e-3) / 1e9, "peak": peak,
                         "unit": "GB/s", "frac": t_roof / ms, "peak_source": src,
                         "algorithmic_bytes_per_step": roof_bytes, "note": "three reads of every A"}}
    line.update(extra)
    print(json.dumps(line), flush=True)


def _time_batch(a, b, mats, outs):
    import torch
    st = torch.cuda.current_stream()
    for _ in range(a.warmup):
        b.run(mats, outs)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(a.steps):
        b.run(mats, outs)
    e1.record(st)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / a.steps


def run_batch(a):
    """256 FP32 matrices, m, n log-uniform in [256, 4096] (n rounded to a
    multiple of 4), k uniform in [8, 64], p = 10, sigma_j = 0.9^j (rank
    min(m, n, 256) plus N(0, 1e-6^2) noise): one graph launch per step."""
    import numpy as np
    import torch

    from paper_1803_01982_gb300 import ffsrqr, synth
    rng = np.random.default_rng(4)
    sizes, mats = [], []
    for i in range(256):
        m, n = (int(round(np.exp(rng.uniform(np.log(256), np.log(4096))))) for _ in range(2))
        n += (-n) % 4
        k = int(rng.integers(8, 65))
        r = min(m, n, 256)
        mats.append(synth.decayed_torch(m, n, 0.9 ** np.arange(r), 1e-6, seed=1000 + i))
        sizes.append((m, n, k, 10))
    mode = {"mixed": ffsrqr.MIXED_TF32X3, "bf16x3": ffsrqr.MIXED_BF16X3, "plain": ffsrqr.PLAIN_FP32}[a.mode]
    b = ffsrqr.Batch(sizes, mode, streams=4)
    outs = b.outputs()
    chosen, tune_ms = b.tune(mats, outs)
    ms = _time_batch(a, b, mats, outs)
    roof = sum(12.0 * m * n for m, n, _, _ in sizes)
    _batch_line(a, f"256 uneven FP32 matrices (m, n in [256, 4096], k in [8, 64], p = 10, sigma_j = 0.9^j), {a.mode}",
                256, ms, roof, {"autotune": {"streams": chosen, "phase_batched": b.phased, "ms": tune_ms,
                                             "small_svd_launches": b.small_svd_launches()}})


def run_hosvd(a):
    """Tucker/HOSVD factors of a 400^3 FP32 tensor (core 40^3 N(0,1) times
    three orthonormal 400 x 40 factors, plus N(0, 1e-4^2) noise): rank-40
    approximations (p = 5) of its three 400 x 160000 unfoldings in one graph.
    The mode-2 and mode-3 unfoldings are materialised as permuted copies."""
    import numpy as np
    import torch

    from paper_1803_01982_gb300 import ffsrqr, synth
    rng = np.random.default_rng(5)
    Us = [torch.as_tensor(synth.orthonormal(rng, 400, 40), device="cuda") for _ in range(3)]
    G = torch.as_tensor(rng.standard_normal((40, 40, 40)), device="cuda")
    T = torch.einsum("abc,ia,jb,kc->ijk", G, Us[0], Us[1], Us[2])
    T = T + 1e-4 * torch.randn(T.shape, dtype=T.dtype, device="cuda", generator=torch.Generator("cuda").manual_seed(5))
    T = T.float()
    unf = [T.reshape(400, 160000).contiguous(), T.permute(1, 0, 2).reshape(400, 160000).contiguous(),
           T.permute(2, 0, 1).reshape(400, 160000).contiguous()]
    del T
    mode = {"mixed": ffsrqr.MIXED_TF32X3, "bf16x3": ffsrqr.MIXED_BF16X3, "plain": ffsrqr.PLAIN_FP32}[a.mode]
    b = ffsrqr.Batch([(400, 160000, 40, 5)] * 3, mode, streams=3)
    outs = b.outputs()
    ms = _time_batch(a, b, unf, outs)
    _batch_line(a, f"HOSVD factors of a 400^3 FP32 tensor (3 unfoldings 400x160000, k = 40, p = 5), {a.mode}",
                3, ms, 3 * 12.0 * 400 * 160000, {})


def run_tucker(a):
    """Tucker approximation of the 400^3 FP32 tensor of the HOSVD workload
    (multilinear rank 40 + N(0, 1e-4^2) noise) to ranks (40, 40, 40), p = 5,
    one ffsrqr_tucker_run per step.
    sthosvd (Alg. 6, order 1-2-3): Flip-Flop SRQR of the 400 x 160000,
      400 x 16000 and 400 x 1600 unfoldings, with the permutes between them;
      only the first unfolding (256 MB) exceeds the L2.
    hosvd-core (Alg. 5): Flip-Flop SRQR of the three 400 x 160000 unfoldings
      (two of them permuted copies), then the core G = X x_r U_r^T mode by mode."""
    import torch

    from paper_1803_01982_gb300 import ffsrqr, synth
    dims, ranks = (400, 400, 400), (40, 40, 40)
    X = synth.tucker_torch(dims, ranks, 1e-4, seed=5)
    mode = {"mixed": ffsrqr.MIXED_TF32X3, "bf16x3": ffsrqr.MIXED_BF16X3, "plain": ffsrqr.PLAIN_FP32}[a.mode]
    st_method = a.workload == "sthosvd"
    t = ffsrqr.Tucker(dims, ranks, None, 5, mode, ffsrqr.TUCKER_STHOSVD if st_method else ffsrqr.TUCKER_HOSVD)
    out = t.outputs()
    st = torch.cuda.current_stream()
    for _ in range(a.warmup):
        t.run(X, out=out)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(a.steps):
        t.run(X, out=out)
    e1.record(st)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / a.steps
    if st_method:
        roof = 12.0 * 400 * (160000 + 16000 + 1600)   # three reads of each unfolding
        name = "ST-HOSVD (Alg. 6) of a 400^3 FP32 tensor to ranks (40, 40, 40), p = 5, order 1-2-3"
    else:
        roof = 3 * 12.0 * 400 * 160000 + 4.0 * 400 * (160000 + 16000 + 1600)  # + one read per core product
        name = "HOSVD (Alg. 5, factors and core) of a 400^3 FP32 tensor to ranks (40, 40, 40), p = 5"
    extra = {"metric": "Tucker decompositions/s", "unit": "decompositions/s",
             "gpu_launches": t.launch_count() * a.steps, "statuses": [i["status"] for i in t.infos()]}
    if not a.no_cpu:
        secs, sample = tucker_cpu_baseline(X.double().cpu().numpy(), ranks, st_method)
        extra["cpu_baseline"] = {"value": 1.0 / secs, "unit": "decompositions/s", "cores": cores_used(),
                                 "kind": "oracle", "sample": sample, "sample_seconds": secs}
    _batch_line(a, f"{name}, {a.mode}", 1, ms, roof, extra)


def run_rpca(a):
    """Robust PCA by IALM (Alg. 7) with Flip-Flop SRQR as the SVD, on the
    paper's synthetic test matrices (Sec. 4.3.1): M = X_L X_R^T + E*, rank
    0.1 m, 0.05 m^2 corruptions uniform in [-500, 500], m = n = --m (1000 or
    2000 here).  One step = one solve (blocking: the iteration reads the
    singular values back every iteration)."""
    import numpy as np
    import torch

    from paper_1803_01982_gb300 import ffsrqr, synth
    m = a.m if a.m <= 4000 else 2000
    M, Xs, _ = synth.rpca_problem(m, m, m // 10, int(0.05 * m * m), seed=1)
    Md = torch.as_tensor(M).cuda()
    mode = {"mixed": ffsrqr.MIXED_TF32X3, "bf16x3": ffsrqr.MIXED_BF16X3, "plain": ffsrqr.PLAIN_FP32}[a.mode]
    s = ffsrqr.RPCA(m, m, mode)
    X = torch.empty_like(Md)
    E = torch.empty_like(Md)
    for _ in range(a.warmup):
        s.run(Md, X, E)
    torch.cuda.synchronize()
    times, info = [], None
    for _ in range(a.steps):
        t0 = time.perf_counter()
        _, _, info = s.run(Md, X, E)
        torch.cuda.synchronize()
        times.append((time.perf_counter() - t0) * 1e3)
    ms = statistics.median(times)
    err = float(np.linalg.norm(X.double().cpu().numpy() - Xs) / np.linalg.norm(Xs))
    it = info["iters"]
    # per iteration: Alg. 9 reads Z three times; the update reads M, X, Y and
    # writes E, Y, Z; the product writes X
    roof = 10.0 * 4 * m * m * it
    line = {"metric": "RPCA solves/s", "value": 1000.0 / ms, "unit": "solves/s", "n_gpus": 1, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"IALM robust PCA, {m}x{m}, rank {m // 10}, {int(0.05 * m * m)} corruptions "
                                   f"in [-500, 500], lambda = 1/sqrt({m}), {a.mode}"},
            "iters": it, "ms_per_iter": ms / it, "rank": info["rank"], "nnz_e": info["nnz_e"],
            "rel_error_vs_truth": err, "rel_residual": info["rel_residual"],
            "gpu_launches": s.launch_count() * a.steps,
            "roofline": {"bound": "hbm", "algorithmic_bytes_per_step": roof,
                         "achieved": roof / (ms * 1e-3) / 1e9, "peak": peaks()[0], "unit": "GB/s",
                         "frac": roof / (ms * 1e-3) / 1e9 / peaks()[0]},
            "paper_context": {"1000": "IALM_FFSRQR 1.02 s, 25 iterations, error 2.79e-7 (CPU, Sec. 4.3.1)",
                              "2000": "IALM_FFSRQR 6.93 s, 25 iterations, error 1.82e-7 (CPU, Sec. 4.3.1)"}}
    if not a.no_cpu:
        secs, sample = rpca_cpu_baseline(m)
        line["cpu_baseline"] = {"value": 1.0 / secs, "unit": "solves/s", "cores": cores_used(), "kind": "oracle",
                                "sample": sample, "seconds_at_full_size": secs}
    print(json.dumps(line), flush=True)


def run_rsisvd(a):
    """Randomized subspace iteration (the paper's appendix algorithm; p = 5,
    q = 1, its parameters in Sec. 4.1) against Flip-Flop SRQR on the default
    workload (20000 x 20000, sigma_j = j^-1.5, k = 200), both on this library's
    kernels in --mode.  One step = one approximation.  The accuracy of both is
    measured after the timed region as ||A - U S V^T||_F / ||A||_F (a torch
    product, verification only)."""
    import torch

    from paper_1803_01982_gb300 import ffsrqr, synth
    mode = {"mixed": ffsrqr.MIXED_TF32X3, "bf16x3": ffsrqr.MIXED_BF16X3, "plain": ffsrqr.PLAIN_FP32}[a.mode]
    r = min(2000, a.m, a.n)
    A = synth.decayed_torch(a.m, a.n, spectrum(a, r), 1e-6, seed=1)
    st = torch.cuda.current_stream()
    res = {}
    for name, plan in (("rsisvd", ffsrqr.Plan(a.m, a.n, a.k, 5, mode, rsi_q=1)),
                       ("ffsrqr", ffsrqr.Plan(a.m, a.n, a.k, a.p, mode))):
        out = plan.outputs()
        for _ in range(a.warmup):
            plan.run(A, 0, out)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(a.steps):
            plan.run(A, 0, out)
        e1.record(st)
        torch.cuda.synchronize()
        U, S, V, _ = out
        err = float(torch.linalg.norm(A - (U * S) @ V.T) / torch.linalg.norm(A))
        res[name] = {"ms": e0.elapsed_time(e1) / a.steps, "rel_error_fro": err,
                     "launches": ffsrqr.ffsrqr_launch_count(plan._h), "status": plan.info()["status"],
                     "sigma_1": float(S[0]), "sigma_k": float(S[-1])}
    ms = res["rsisvd"]["ms"]
    peak, src = peaks()
    roof_bytes = 4.0 * a.m * a.n * 4  # q = 1: four reads of A
    line = {"metric": METRIC, "value": 1000.0 / ms, "unit": UNIT, "n_gpus": 1, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"RSISVD (p = 5, q = 1) of {a.m}x{a.n} FP32, r=2000, "
                                   f"{'sigma_j=j^-1.5' if a.decay == 'slow' else 'sigma_j=0.97^j'}, k={a.k}, "
                                   f"{a.mode}"},
            "roofline": {"bound": "hbm", "achieved": roof_bytes / (ms * 1e-3) / 1e9, "peak": peak, "unit": "GB/s",
                         "frac": roof_bytes / (peak * 1e9) / (ms * 1e-3), "peak_source": src,
                         "algorithmic_bytes_per_step": roof_bytes, "note": "four reads of A"},
            "gpu_launches": res["rsisvd"]["launches"] * a.steps, "comparison": res}
    print(json.dumps(line), flush=True)


def run_serving(a):
    """Poisson arrivals (mean a.rate per second, a.duration seconds) of
    truncated-SVD requests like singular-value-thresholding iterates:
    A = X_L X_R^T + N(0, 1e-3^2), X_L, X_R Gaussian of rank r uniform in
    [10, 100], m, n log-uniform in [500, 8000] (n a multiple of 4),
    k = r + 10, p = 10, served under a 120 GB budget with 8 slots.  The
    matrices come from a pool of 64 generated up front."""
    import numpy as np
    import torch

    from paper_1803_01982_gb300 import ffsrqr
    rng = np.random.default_rng(6)
    pool = []
    gen = torch.Generator("cuda").manual_seed(6)
    for i in range(64):
        m, n = (int(round(np.exp(rng.uniform(np.log(500), np.log(8000))))) for _ in range(2))
        n += (-n) % 4
        r = int(rng.integers(10, 101))
        XL = torch.randn(m, r, device="cuda", generator=gen)
        XR = torch.randn(n, r, device="cuda", generator=gen)
        A = XL @ XR.T + 1e-3 * torch.randn(m, n, device="cuda", generator=gen)
        pool.append((A, r + 10))
    mode = {"mixed": ffsrqr.MIXED_TF32X3, "bf16x3": ffsrqr.MIXED_BF16X3, "plain": ffsrqr.PLAIN_FP32}[a.mode]
    srv = ffsrqr.Server(120 * (1 << 30), slots=8)
    if a.phase_batch:
        srv.set_phase_batch(True)
    # warm the plan cache and the kernels
    for A, k in pool[:4]:
        o = (torch.empty(A.shape[0], k, device="cuda"), torch.empty(k, device="cuda"),
             torch.empty(A.shape[1], k, device="cuda"), torch.empty(A.shape[1], dtype=torch.int32, device="cuda"))
        srv.wait(srv.submit(A, k, 10, mode, o))
    gaps = rng.exponential(1.0 / a.rate, size=int(a.rate * a.duration * 1.5) + 10)
    arrivals = np.cumsum(gaps)
    arrivals = arrivals[arrivals < a.duration]
    lat, pending = [], []
    t0 = time.perf_counter()
    for i, ta in enumerate(arrivals):
        while time.perf_counter() - t0 < ta:
            # collect finished requests while waiting for the next arrival
            still = []
            for t in pending:
                r = srv.poll(t)
                if r is None:
                    still.append(t)
                else:
                    lat.append(r[1])
            pending = still
            time.sleep(0.0002)
        A, k = pool[i % len(pool)]
        o = (torch.empty(A.shape[0], k, device="cuda"), torch.empty(k, device="cuda"),
             torch.empty(A.shape[1], k, device="cuda"), torch.empty(A.shape[1], dtype=torch.int32, device="cuda"))
        pending.append(srv.submit(A, k, 10, mode, o))
    for t in pending:
        lat.append(srv.wait(t)[1])
    wall = time.perf_counter() - t0
    ph = srv.phase_stats()
    srv.close()
    lat = np.array(lat) * 1e3
    line = {"metric": "serving latency p50/p99 (ms) and throughput", "value": len(lat) / wall,
            "unit": "req/s", "n_gpus": 1, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"Poisson {a.rate:g} req/s for {a.duration:g} s, m, n in [500, 8000], "
                                   f"rank 10..100 + noise, k = r + 10, p = 10, 120 GB budget, 8 slots, {a.mode}",
                       "same_phase_batching": bool(a.phase_batch)},
            "offered_req_s": float(len(arrivals) / a.duration), "phase_stats": ph,
            "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                           "mean": float(lat.mean()), "max": float(lat.max())},
            "requests": int(len(lat)), "wall_s": wall}
    print(json.dumps(line), flush=True)


def main():
    a = parse()
    if a.workload != "single" and a.impl == "ours":
        {"batch": run_batch, "hosvd": run_hosvd, "sthosvd": run_tucker, "hosvd-core": run_tucker,
         "rpca": run_rpca, "rsisvd": run_rsisvd, "serving": run_serving}[a.workload](a)
        return
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if a.impl == "reference":
        run_reference(a, rank, world)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    try:
        run_ours(a, rank, world, local_rank)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
