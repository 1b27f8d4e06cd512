"""Benchmark: time to true relative residual 1e-10, forward + adjoint, of the
dense-banded SaP solver on one GB300 (and N independent replicas under
torchrun).

Workload (default): dense banded N = 200,000, K = 50, d = 1.0, P = 50,
off-diagonals U(-1,1), x_true ~ U(-1,1), b = A x_true, adjoint right-hand
side g-bar ~ U(-1,1).  One step = refactor of the SaP preconditioner (FP32
factors) + BiCGStab(2) solve of A x = b + adjoint solve of A^T lambda = g-bar,
each to relres <= 1e-10 (the FP64 SaP is timed the same way for comparison).
Inputs are resident in HBM before timing; L2 (129 MB) is flushed before
every timed step by writing a 512 MB buffer.

`python bench.py --impl reference` times the FP64 CPU oracle (the
repository's plain C reference) on the host cores instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "time to rel.res 1e-10 & HBM GB/s: FP32-precond vs FP64 SaP, fwd+adjoint"
# DRAM bytes (read + write) of the sweep launches of one FP32 SaP-D preconditioner
# apply on the N=200000, K=50, P=50 workload (automatic segment count), from one
# ncu capture of dram__bytes_read.sum + dram__bytes_write.sum of those launches
TRAFFIC_SWEEPS = 232656896
# DRAM bytes (read + write) of one k_band_lu launch (FP32), by (N, K, P), from an
# ncu capture of the current kernel; a workload without a capture reports null
TRAFFIC_LU = {(200000, 50, 50): 118135552}
# P=None: picked by sap_autotune (measured refactor + solve over N / {16000 .. 1000}, 152, 304)
# before the timed region; P_ref is the oracle's partition count in that case
# (the autotuner's pick on GB300 when this table was written).
WORKLOADS = {
    "n200k_k50": dict(N=200000, K=50, d=1.0, P=50, seed_cfg=2),
    "n10k_k10": dict(N=10000, K=10, d=1.2, P=8, seed_cfg=1),
    "n200k_k100": dict(N=200000, K=100, d=1.0, P=None, P_ref=304, seed_cfg=3),
    "n200k_k200": dict(N=200000, K=200, d=1.0, P=None, P_ref=152, seed_cfg=3),
    "n200k_k400": dict(N=200000, K=400, d=1.0, P=None, P_ref=304, seed_cfg=3),
    "convdiff_400x250": dict(N=100000, K=250, d=None, P=32, seed_cfg=4, grid=(400, 250), variant="C"),
    # the symmetric positive definite band at the C2 sizes, CG outer iteration (Sec. 3)
    "n200k_k50_spd_cg": dict(N=200000, K=50, d=1.0, P=50, seed_cfg=2, spd=True, krylov="CG"),
}
# oracle work (multiply-adds of the factorisations, forward + adjoint) above
# which the CPU baseline times a leading sample of the blocks and scales by rows
ORACLE_FULL_LIMIT = 1.5e10


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="n200k_k50", choices=sorted(WORKLOADS) + ["batch64"],
                    help="batch64: 64 systems N ~ U{1e4..1e5}, K ~ U{8..64} through the batched API")
    ap.add_argument("--variant", default=None, choices=["C", "D"],
                    help="SaP variant (default: the workload's, else D)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-compare", action="store_true", help="skip the FP64 / other-variant comparison runs")
    ap.add_argument("--blocks", action="store_true",
                    help="SaP with per-block bandwidths (third-stage reordering) against SaP on the whole band")
    ap.add_argument("--blocks-k", type=int, default=100, help="half-bandwidth K of the --blocks workload")
    ap.add_argument("--sparse", action="store_true",
                    help="time the sparse front end (Sec. 2.2) and the solve of the reordered band")
    ap.add_argument("--sweep", default=None, choices=["P", "d"],
                    help="the sensitivity study of Sec. 4.1.1 (P) or 4.1.2 (d) instead of the benchmark line")
    a = ap.parse_args()
    if a.variant is None:
        a.variant = WORKLOADS.get(a.workload, {}).get("variant", "D")
    return a


def max_over_ranks(ms: float) -> float:
    """Job time of one step: the slowest rank's (all ranks call this after
    their timed region; NCCL reduces on the device, gloo on the host)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return ms
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([ms], device=dev, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


# ----------------------------------------------------------------- inputs --

def make_inputs(w):
    import sap_inputs as G
    seed = G.config_seed(w["seed_cfg"])
    if "grid" in w:
        band, N, K = G.convection_diffusion(*w["grid"])
        assert (N, K) == (w["N"], w["K"])
    elif w.get("spd"):
        band = G.dense_banded_spd(w["N"], w["K"], w["d"], seed)
    else:
        band = G.dense_banded(w["N"], w["K"], w["d"], seed)
    xt = G.x_true(w["N"], seed)
    g = G.adjoint_seed(w["N"], seed)
    return band, xt, g


# ------------------------------------------------------------- CPU oracle --

def oracle_P(w):
    return w["P"] if w["P"] is not None else w["P_ref"]


def oracle_sample(w, variant, band, xt, g):
    """The oracle's inputs: the whole workload, or (too much work for a bounded
    CPU run) the leading principal sub-system of its first m blocks, with
    b = A_s x_true_s; returns (w_s, band_s, b_s, g_s, rows scale, description)."""
    import numpy as np
    import oracle as O
    N, K, P = w["N"], w["K"], oracle_P(w)
    per_row = (2 if variant == "C" else 1) * 2 * K * K
    if per_row * N <= ORACLE_FULL_LIMIT:
        return dict(w, P=P), band, O.spmv(band, N, K, xt), g, 1.0, "the full workload"
    n = N // P
    m = max(2 if variant == "C" else 1, int(ORACLE_FULL_LIMIT // (per_row * n)))
    Ns = m * n
    band_s = np.ascontiguousarray(band.reshape(2 * K + 1, N)[:, :Ns]).reshape(-1)
    ws = dict(w, N=Ns, P=m)
    return (ws, band_s, O.spmv(band_s, Ns, K, xt[:Ns]), np.ascontiguousarray(g[:Ns]), N / Ns,
            f"the leading {m} of {P} blocks ({Ns} of {N} rows, the principal sub-system), time scaled by "
            f"rows x{N / Ns:.2f}")


def oracle_step(band, b, g, w, variant, omp=False):
    """One fwd + adjoint time-to-solution with the FP64 CPU oracle."""
    import oracle as O
    N, K, P = w["N"], w["K"], oracle_P(w)
    var = O.SAP_C if variant == "C" else O.SAP_D
    s = O.Sap(band, N, K, P, var, omp=omp)
    if w.get("krylov") == "CG":     # symmetric A: the adjoint is the same system
        x, i1 = s.solve_cg(b)
        lam, i2 = s.solve_cg(g)
    else:
        x, i1 = s.solve(b)
        sa = O.Sap(O.transpose_band(band, N, K), N, K, P, var, omp=omp)
        lam, i2 = sa.solve(g)
    assert i1.status == O.OK and i2.status == O.OK
    return i1, i2


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for ln in open("/proc/cpuinfo"):
            if ln.lower().startswith(("model name", "cpu part", "hardware")):
                return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def cpu_baseline(w, variant, band, xt, g, reps=3):
    """The FP64 C oracle on the host cores: (i) single-threaded, the median of
    reps runs; (ii) the same oracle built with OpenMP over the independent
    blocks (bit-identical results), median of reps runs."""
    import oracle as O
    ws, band_s, b_s, g_s, scale, what = oracle_sample(w, variant, band, xt, g)
    ts = []
    for _ in range(reps):
        t0 = time.perf_counter()
        oracle_step(band_s, b_s, g_s, ws, variant)
        ts.append((time.perf_counter() - t0) * 1e3 * scale)
    out = {"value": statistics.median(ts), "unit": "ms", "cores": 1, "kind": "oracle",
           "sample": f"{what}, median of {reps} runs of factor + solve + adjoint solve "
                     f"(single-threaded FP64 C oracle, SaP-{variant}, P = {oracle_P(w)} for the workload)",
           "host_cpus": os.cpu_count(), "cpu_model": cpu_model()}
    try:
        tm = []
        for _ in range(reps):
            t0 = time.perf_counter()
            oracle_step(band_s, b_s, g_s, ws, variant, omp=True)
            tm.append((time.perf_counter() - t0) * 1e3 * scale)
        out["openmp"] = {"value": statistics.median(tm), "unit": "ms", "cores": O.omp_threads(),
                         "sample": "the same runs with the oracle built with -fopenmp (per-block loops of the "
                                   "factorisation and the applies in parallel; results bit-identical)"}
    except Exception as e:  # noqa: BLE001
        out["openmp"] = {"unavailable": str(e)[:200]}
    return out


def run_reference_batch(args):
    """Oracle arm of the 64-system batch: each step runs the FP64 oracle (factor,
    solve, adjoint solve) on the three smallest systems and scales the time by
    rows to the whole batch (a bounded sample)."""
    import numpy as np
    import oracle as O
    import sap_inputs as G
    specs = G.batch_specs(64)
    Ns = [n for n, _, _ in specs]
    idx = list(np.argsort(Ns)[:3])
    total = sum(Ns)
    rows = sum(Ns[i] for i in idx)
    sample = []
    for i in idx:
        n, k, sd = specs[i]
        band = G.dense_banded(n, k, 1.0, sd)
        P = max(1, round(2 * 152 * n / total))
        sample.append((band, n, k, O.spmv(band, n, k, G.x_true(n, sd)), G.adjoint_seed(n, sd), P))

    def step():
        for band, n, k, b, g, P in sample:
            O.solve(band, n, k, b, P, O.SAP_D)
            O.solve_adjoint(band, n, k, g, P, O.SAP_D)

    for _ in range(args.warmup):
        step()
    ts = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        step()
        ts.append((time.perf_counter() - t0) * 1e3 * total / rows)
    v = statistics.mean(ts)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "ms", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": v, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "batch of 64 dense banded systems, N ~ U{10000..100000}, K ~ U{8..64}, d=1.0, "
                                   "SaP-D, FP32 preconditioner + FP64 BiCGStab(2), fwd + adjoint to relres 1e-10 "
                                   "(solved concurrently; the adjoint right-hand sides are given)",
                       "systems": 64, "rows": int(total)},
            "cpu_baseline": {"value": v, "unit": "ms", "cores": 1, "kind": "oracle",
                             "sample": f"each step: the 3 smallest systems ({rows} rows), factor + solve + adjoint "
                                       f"solve, scaled by rows to {total}"},
            "e2e": {"value": v, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    if args.workload == "batch64":
        run_reference_batch(args)
        return
    w = WORKLOADS[args.workload]
    band, xt, g = make_inputs(w)
    ws, band_s, b_s, g_s, scale, what = oracle_sample(w, args.variant, band, xt, g)
    for _ in range(args.warmup):
        oracle_step(band_s, b_s, g_s, ws, args.variant)
    ts = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle_step(band_s, b_s, g_s, ws, args.variant)
        ts.append((time.perf_counter() - t0) * 1e3 * scale)
    v = statistics.mean(ts)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "ms", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": v, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(args, w),
            "cpu_baseline": {"value": v, "unit": "ms", "cores": 1, "kind": "oracle",
                             "sample": f"each step: {what}, factor + solve + adjoint solve "
                                       f"(single-threaded FP64 C oracle, P = {oracle_P(w)} for the workload)"},
            "e2e": {"value": v, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def workload_config(args, w):
    Ptxt = "autotuned" if w["P"] is None else w["P"]
    if "grid" in w:
        kind = (f"2-D convection-diffusion {w['grid'][0]}x{w['grid'][1]} (5-point upwind, Peclet 10) as a dense "
                f"band N={w['N']} K={w['K']}")
    elif w.get("spd"):
        kind = f"symmetric positive definite dense banded N={w['N']} K={w['K']} d={w['d']}"
    else:
        kind = f"dense banded N={w['N']} K={w['K']} d={w['d']}"
    if w.get("krylov") == "CG":
        how = ("FP32 preconditioner + FP64 preconditioned CG, fwd + adjoint to relres 1e-10 "
               "(the two solved concurrently; the adjoint right-hand side is given)")
    else:
        how = ("FP32 preconditioner + FP64 BiCGStab(2), fwd + adjoint to relres 1e-10 "
               "(the two solved concurrently; the adjoint right-hand side is given)")
    return {"workload": f"{kind} P={Ptxt} SaP-{args.variant}, {how}",
            "N": w["N"], "K": w["K"], "P": Ptxt, "d": w["d"], "variant": f"SaP-{args.variant}",
            "l2": "flushed (512 MB write) before every timed step"}


# ------------------------------------------------------------------- GPU --

class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, gpu_index):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={gpu_index}", f"--query-gpu={q}",
                                       "--format=csv,noheader,nounits", "-lms", "100"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        self.p.wait()
        self.f.flush()
        rows = [r.split(",") for r in open(self.f.name).read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm = [float(r[1]) for r in rows if len(r) >= 9 and r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if len(r) >= 9 and r[2].strip().replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            if len(r) < 9:
                continue
            for k, name in enumerate(names):
                if r[5 + k].strip().lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def run_gpu(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    import paper_1509_07919_gb300 as S

    w = WORKLOADS[args.workload]
    N, K, P = w["N"], w["K"], w["P"]
    variant = S.SAP_C if args.variant == "C" else S.SAP_D
    band_np, xt_np, g_np = make_inputs(w)
    band = torch.from_numpy(band_np).cuda()
    xt = torch.from_numpy(xt_np).cuda()
    g = torch.from_numpy(g_np).cuda()
    b = S.sap_spmv(band, N, K, xt)
    stream = torch.cuda.current_stream()
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    autotune = None
    if P is None:       # measured choice, outside the timed region
        P, _, table = S.sap_autotune(band, N, K, b=b, variant=variant, precision=S.SAP_FP32)
        autotune = {"P": P, "ms_by_P_segments": {f"{p},{sg}": v for (p, sg), v in sorted(table.items())}}

    krylov = S.SAP_KRYLOV_CG if w.get("krylov") == "CG" else S.SAP_KRYLOV_BICGSTAB2

    def make_handle(prec, var):
        return S.sap_factor(band, N, K, P=P, variant=var, precision=prec, krylov=krylov)

    # one step: refactor, then the forward and adjoint solves run concurrently
    # (sap_solve_pair; the adjoint right-hand side is given, independent of x);
    # sequential=True times sap_solve followed by sap_solve_adjoint instead
    def step(h, x, lam, sequential=False):
        S.sap_refactor(h)
        if sequential:
            _, i1, _ = S.sap_solve(h, b, x)
            _, i2, _ = S.sap_solve_adjoint(h, g, lam)
        else:
            _, _, i1, i2, _ = S.sap_solve_pair(h, b, g, x, lam)
        return i1, i2

    def timed(h, steps, warmup, clocks=False, sequential=False):
        x = torch.empty_like(b)
        lam = torch.empty_like(b)
        for _ in range(warmup):
            step(h, x, lam, sequential)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        ck = Clocks(local) if clocks else None
        l0 = S.sap_kernel_launches()
        times, infos = [], []
        for _ in range(steps):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            i1, i2 = step(h, x, lam, sequential)
            e1.record(stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
            infos.append((i1, i2))
        launches = S.sap_kernel_launches() - l0
        ckd = ck.stop() if ck else None
        return times, infos, launches, ckd, x, lam

    h = make_handle(S.SAP_FP32, variant)
    times, infos, launches, clocks, x, lam = timed(h, args.steps, args.warmup, clocks=True)
    ms = max_over_ranks(statistics.mean(times))
    i1, i2 = infos[-1]
    # the same step with the two solves one after the other (sap_solve, then sap_solve_adjoint)
    seq_times, _, _, _, _, _ = timed(h, args.steps, args.warmup, sequential=True)
    seq_ms = statistics.mean(seq_times)
    # accuracy against the generating solution
    err_x = float(torch.linalg.norm(x - xt) / torch.linalg.norm(xt))

    # ---- phase split and the dominant kernel's live duration ----
    t_lu = statistics.mean([a.t_lu_ms for a, _ in infos])          # the block LU kernel alone
    t_prep = statistics.mean([a.t_prep_ms for a, _ in infos])
    t_ul = statistics.mean([a.t_ul_ms for a, _ in infos])
    t_spk = statistics.mean([a.t_spk_ms for a, _ in infos])
    t_fwd = statistics.mean([a.t_solve_ms for a, _ in infos])
    t_adj = statistics.mean([b_.t_solve_ms for _, b_ in infos])

    # per-kernel timing with events on the launching stream (inside this run)
    def kernel_ms(fn, reps=20):
        for _ in range(3):
            fn()
        flush.fill_(2.0)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    y = torch.empty_like(b)
    z = torch.empty_like(b)
    t_spmv = kernel_ms(lambda: S.sap_spmv(band, N, K, xt, y))
    # the sweep kernels alone: one SaP-D apply is exactly their launches (one
    # fused launch unsegmented; with segments, per sweep kind the zero-history
    # sweep, the history chain (more than two segments) and the correction)
    hd = h if variant == S.SAP_D else make_handle(S.SAP_FP32, S.SAP_D)
    segs = i1.segments
    # one fused launch unsegmented; with segments per sweep kind the sweep and the
    # correction (which runs short history chains itself), plus the chain kernel
    # when its transfer matrices exceed the correction's 96 KB of shared memory
    kh = (K + 3) // 4 * 4
    fused_chain = segs > 2 and ((segs - 2) * kh * kh + (segs - 1) * kh) * 4 <= 96 * 1024
    sweep_launches = 1 if segs == 1 else (4 if segs == 2 or fused_chain else 6)
    t_sweep = kernel_ms(lambda: S.sap_apply_preconditioner(hd, b, z))
    t_apply = kernel_ms(lambda: S.sap_apply_preconditioner(h, b, z))
    W = 2 * K + 1
    hbm_peak, peak_kind = load_peaks()
    lu_bytes = 4 * N * W + 4 * N * W               # read the FP32 band copy, write FP32 factors
    spmv_bytes = 8 * N * W + 16 * N
    sweep_bytes = 4 * N * W + 16 * N               # SaP-D apply: FP32 factors once + r, z
    apply_bytes = sweep_bytes * (2 if variant == S.SAP_C else 1)
    kernels = {
        "band_lu": {"ms": t_lu, "bytes": lu_bytes, "GBs": lu_bytes / (t_lu * 1e6),
                    "TFLOPs_fp32": 2.0 * N * K * K / (t_lu * 1e9)},
        "spmv_fp64": {"ms": t_spmv, "bytes": spmv_bytes, "GBs": spmv_bytes / (t_spmv * 1e6),
                      "fp64_TFLOPs": 2 * N * W / (t_spmv * 1e9)},
        "block_solve_fp32": {"ms": t_sweep, "bytes": sweep_bytes, "GBs": sweep_bytes / (t_sweep * 1e6)},
        "apply_fp32": {"ms": t_apply, "bytes": apply_bytes, "GBs": apply_bytes / (t_apply * 1e6)},
    }
    ach_s = kernels["block_solve_fp32"]["GBs"]
    sweep_line = {"bound": "hbm",
                "kernel": ("k_block_solve (both triangular sweeps of every block, FP32)" if segs == 1 else
                           f"k_sweep + k_seg_correct{'' if sweep_launches == 4 else ' + k_seg_chain'} (both "
                           f"triangular sweeps of every block in {segs} segments, FP32; {sweep_launches} launches "
                           f"per apply)"),
                "achieved": ach_s, "peak": hbm_peak, "unit": "GB/s", "frac": ach_s / hbm_peak,
                "peak_kind": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured" else
                "fallback 6.8 TB/s",
                # dram__bytes_read.sum + dram__bytes_write.sum of the sweep launches of one
                # apply (one ncu capture); above the algorithmic bytes
                # because the sweeps stream the per-chunk inverse/coupling matrices
                "traffic": TRAFFIC_SWEEPS if (N, K, P) == (200000, 50, 50) else None,
                "algorithmic_bytes_per_launch": sweep_bytes,
                "unit_of_launch": f"one preconditioner apply = {sweep_launches} sweep launch(es)",
                "note": f"{segs} segment(s) per block, {segs * P} CTAs per pass; the 32-row chunk "
                        "recurrence is latency-bound"}
    # the dominant kernel of the step: the block LU (largest share of the launch list)
    ach = kernels["band_lu"]["GBs"]
    roofline = {"bound": "hbm", "kernel": "k_band_lu (FP32 block LU of every block, one CTA per block)",
                "achieved": ach, "peak": hbm_peak, "unit": "GB/s", "frac": ach / hbm_peak,
                "peak_kind": sweep_line["peak_kind"],
                "traffic": TRAFFIC_LU.get((N, K, P)),
                "algorithmic_bytes_per_launch": lu_bytes,
                "unit_of_launch": f"one factorisation: read the FP32 band copy (4 N (2K+1) B), write the FP32 "
                                  f"factors (4 N (2K+1) B); {2.0 * N * K * K:.3g} FP32 flops",
                "duration_ms": t_lu,
                "note": f"live duration from CUDA events around the k_band_lu launch on its stream, mean over the "
                        f"timed steps; {P} CTAs (one per block) of a serial chain of {-(-(N // P) // 16)} "
                        f"16-column panel steps: latency-bound, not bandwidth-bound"}

    # ---- end to end through the C ABI with host buffers: every step copies the band, b
    # and g-bar in from page-locked host memory and x, lambda back, inside the library
    # calls (sap_refactor_host, sap_solve_pair_host) ----
    band_h = torch.from_numpy(band_np).pin_memory()
    b_h = b.cpu().pin_memory()
    g_h = g.cpu().pin_memory()
    x_h = torch.empty_like(b_h).pin_memory()
    l_h = torch.empty_like(b_h).pin_memory()
    h2 = S.sap_factor_host(band_h, N, K, P=P, variant=variant, precision=S.SAP_FP32, krylov=krylov)
    e2e_times = []
    for k in range(args.warmup + args.steps):
        flush.fill_(3.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        S.sap_refactor_host(h2, band_h)
        S.sap_solve_pair_host(h2, b_h, g_h, x_h, l_h)
        if k >= args.warmup:
            e2e_times.append((time.perf_counter() - t0) * 1e3)
    e2e_ms = statistics.mean(e2e_times)
    e2e_err = float(np.linalg.norm(x_h.numpy() - xt_np) / np.linalg.norm(xt_np))
    del h2

    # ---- comparison: FP64 SaP and the other variant (same protocol, fewer steps) ----
    compare = {}
    if not args.no_compare:
        runs = [("sapc_fp64", S.SAP_FP64, S.SAP_C), ("sapd_fp64", S.SAP_FP64, S.SAP_D),
                ("sapc_fp32", S.SAP_FP32, S.SAP_C), ("sapd_fp32", S.SAP_FP32, S.SAP_D)]
        if K >= 64:     # the tensor-core (BF16 operand) trailing update of the block LU
            runs.append(("sapd_bf16tu", S.SAP_FP32_BF16TU, S.SAP_D))
            if variant == S.SAP_C:
                runs.append(("sapc_bf16tu", S.SAP_FP32_BF16TU, S.SAP_C))
        for name, prec, var in runs:
            try:
                hh = make_handle(prec, var)
            except S.SapError as e:
                compare[name] = {"unavailable": str(e)}
                continue
            tt, inf, _, _, _, _ = timed(hh, max(3, args.steps // 2), 2)
            a, c = inf[-1]
            compare[name] = {"ms": statistics.mean(tt), "iters_fwd": a.iters, "iters_adj": c.iters,
                             "t_lu_ms": a.t_lu_ms,
                             "relres_fwd": a.relres, "relres_adj": c.relres,
                             "t_factor_ms": a.t_factor_ms, "t_fwd_ms": a.t_solve_ms, "t_adj_ms": c.t_solve_ms,
                             "segments": a.segments}
            del hh

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(w, args.variant, band_np, xt_np, g_np)

    if rank == 0:
        # replicas: every rank solves its own system; job-level time per system
        line = {
            "metric": METRIC, "value": ms / world, "unit": "ms",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64", "data": "synthetic",
            "config": workload_config(args, w),
            "clocks": clocks,
            "e2e": {"value": e2e_ms, "unit": "ms",
                    "h2d_bytes_per_step": int(band_h.numel() * 8 + b_h.numel() * 8 + g_h.numel() * 8),
                    "d2h_bytes_per_step": int(x_h.numel() * 8 + l_h.numel() * 8),
                    "api": "sap_refactor_host + sap_solve_pair_host (C ABI, host buffers, copies inside)",
                    "err_x_vs_x_true": e2e_err},
            "gpu_launches": int(launches),
            "roofline": roofline,
            "cpu_baseline": cpu,
            "detail": {"P": P, "autotune": autotune, "solves": "forward and adjoint concurrent (sap_solve_pair)",
                       "sequential_solves_ms": seq_ms,
                       "sweep_segments_per_block": i1.segments, "krylov_graph": bool(i1.graphed),
                       "iters_fwd": i1.iters, "iters_adj": i2.iters, "matvecs_fwd": i1.n_matvec,
                       "matvecs_adj": i2.n_matvec, "restarts_fwd": i1.n_restarts,
                       "restarts_adj": i2.n_restarts, "relres_fwd": i1.relres,
                       "relres_adj": i2.relres, "err_x_vs_x_true": err_x, "n_boosted": i1.n_boosted,
                       "t_lu_ms": t_lu, "t_prep_ms": t_prep, "t_ul_ms": t_ul, "t_spk_ms": t_spk,
                       "t_fwd_solve_ms": t_fwd, "sweep_roofline": sweep_line,
                       "t_adj_solve_ms": t_adj, "kernels": kernels, "compare": compare,
                       "paper_context_ms_k20x": {"SaP-D": 187.717, "SaP-C": 186.756,
                                                 "note": "fwd only, K20X, precision unstated"}},
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_gpu_batch(args):
    """The 64-system batch (uneven N and K, d = 1), FP32 preconditioner + FP64
    BiCGStab(2): a step is one batched refactor, forward solve and adjoint
    solve of all systems; value = ms per step."""
    import numpy as np
    import torch
    import paper_1509_07919_gb300 as S
    import sap_inputs as G
    import oracle as O

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    specs = G.batch_specs(64)
    Ns = [n for n, _, _ in specs]
    Ks = [k for _, k, _ in specs]
    bands_np = [G.dense_banded(n, k, 1.0, sd) for n, k, sd in specs]
    bands = [torch.from_numpy(b).cuda() for b in bands_np]
    xts = [torch.from_numpy(G.x_true(n, sd)).cuda() for n, _, sd in specs]
    gs = [torch.from_numpy(G.adjoint_seed(n, sd)).cuda() for n, _, sd in specs]
    bs = [S.sap_spmv(bd, n, k, xt) for bd, n, k, xt in zip(bands, Ns, Ks, xts)]
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    bh = S.sap_factor_batched(bands, Ns, Ks, precision=S.SAP_FP32, variant=S.SAP_D)
    xs = [torch.empty_like(b) for b in bs]
    ls = [torch.empty_like(b) for b in bs]

    # refactor, then every system's forward and adjoint solves concurrently
    # (sap_solve_pair_batched); sequential=True: all forward, then all adjoint
    def step(sequential=False):
        S.sap_refactor_batched(bh)
        if sequential:
            _, i1, _, _ = S.sap_solve_batched(bh, bs, xs)
            _, i2, _, _ = S.sap_solve_adjoint_batched(bh, gs, ls)
        else:
            _, _, i1, i2, _, _ = S.sap_solve_pair_batched(bh, bs, gs, xs, ls)
        return i1, i2

    def seq_ms():
        ts = []
        for k in range(args.warmup + args.steps):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            a0 = torch.cuda.Event(enable_timing=True)
            a1 = torch.cuda.Event(enable_timing=True)
            a0.record()
            step(True)
            a1.record()
            torch.cuda.synchronize()
            if k >= args.warmup:
                ts.append(a0.elapsed_time(a1))
        return statistics.mean(ts)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ck = Clocks(local)
    l0 = S.sap_kernel_launches()
    times = []
    for _ in range(args.steps):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        i1, i2 = step()
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    launches = S.sap_kernel_launches() - l0
    clocks = ck.stop()
    ms = max_over_ranks(statistics.mean(times))
    err = max(float(torch.linalg.norm(x - xt) / torch.linalg.norm(xt)) for x, xt in zip(xs, xts))
    sequential = seq_ms()
    # end to end: bands, rhs and adjoint seeds from pinned host memory, results back
    hb = [torch.from_numpy(b).pin_memory() for b in bands_np]
    hr = [b.cpu().pin_memory() for b in bs]
    hg = [g.cpu().pin_memory() for g in gs]
    hx = [torch.empty_like(b).pin_memory() for b in hr]
    hl = [torch.empty_like(b).pin_memory() for b in hr]
    dr = [torch.empty_like(b) for b in bs]
    dg = [torch.empty_like(b) for b in bs]
    e2e = []
    for k in range(args.warmup + args.steps):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for a, b_ in zip(bands, hb):
            a.copy_(b_, non_blocking=True)
        for a, b_ in zip(dr, hr):
            a.copy_(b_, non_blocking=True)
        for a, b_ in zip(dg, hg):
            a.copy_(b_, non_blocking=True)
        S.sap_refactor_batched(bh)
        S.sap_solve_pair_batched(bh, dr, dg, xs, ls)
        for a, b_ in zip(hx, xs):
            a.copy_(b_, non_blocking=True)
        for a, b_ in zip(hl, ls):
            a.copy_(b_, non_blocking=True)
        torch.cuda.synchronize()
        if k >= args.warmup:
            e2e.append((time.perf_counter() - t0) * 1e3)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # oracle on the three smallest systems (bounded sample), scaled by rows
        idx = list(np.argsort(Ns)[:3])
        t0 = time.perf_counter()
        for i in idx:
            bnp = bs[i].cpu().numpy()
            O.solve(bands_np[i], Ns[i], Ks[i], bnp, S.sap_batch_partitions(bh)[i], O.SAP_D)
            O.solve_adjoint(bands_np[i], Ns[i], Ks[i], gs[i].cpu().numpy(), S.sap_batch_partitions(bh)[i],
                            O.SAP_D)
        dt = (time.perf_counter() - t0) * 1e3
        rows = sum(Ns[i] for i in idx)
        cpu = {"value": dt * sum(Ns) / rows, "unit": "ms", "cores": 1, "kind": "oracle",
               "sample": f"3 smallest systems ({rows} rows) timed, scaled by rows to the batch's {sum(Ns)}"}
    if rank == 0:
        line = {
            "metric": METRIC, "value": ms / world, "unit": "ms", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": "batch of 64 dense banded systems, N ~ U{10000..100000}, K ~ U{8..64}, d=1.0, "
                                   "SaP-D, FP32 preconditioner + FP64 BiCGStab(2), fwd + adjoint to relres 1e-10 "
                                   "(solved concurrently; the adjoint right-hand sides are given)",
                       "systems": 64, "rows": int(sum(Ns)), "partitions": S.sap_batch_partitions(bh),
                       "l2": "flushed (512 MB write) before every timed step"},
            "clocks": clocks,
            "e2e": {"value": statistics.mean(e2e), "unit": "ms",
                    "h2d_bytes_per_step": int(sum(b.numel() for b in hb) * 8 + 2 * sum(r.numel() for r in hr) * 8),
                    "d2h_bytes_per_step": int(2 * sum(x.numel() for x in hx) * 8)},
            "gpu_launches": int(launches),
            "roofline": None,
            "cpu_baseline": cpu,
            "detail": {"max_err_x_vs_x_true": err, "sequential_solves_ms": sequential,
                       "iters_fwd_max": max(i.iters for i in i1), "iters_adj_max": max(i.iters for i in i2),
                       "relres_fwd_max": max(i.relres for i in i1), "relres_adj_max": max(i.relres for i in i2),
                       "graphed": all(i.graphed for i in i1)},
        }
        print(json.dumps(line), flush=True)


# Sensitivity studies of Sec. 4.1.1 (time to solution against the partition
# count P: N = 200000, K = 200, d = 1) and Sec. 4.1.2 (against the degree of
# diagonal dominance d: N = 200000, K = 200, P = 50), SaP-D against SaP-C.
# Per point: D_pre / C_pre = the preconditioner's set-up (the whole
# factorisation phase, t_factor_ms of the refactor before the solve), D_it /
# C_it = BiCGStab(2) iterations in quarters, D_Kry / C_Kry = the Krylov phase
# (t_kry_ms), D_Tot = D_pre + D_Kry (likewise C), SpdUp = D_Tot / C_Tot, each
# the median of `reps` refactor + forward solves to relres 1e-10 (FP32
# preconditioner, FP64 Krylov).  A point whose solve does not converge
# within max_iters keeps its status in status_D / status_C.
SWEEP_P = (2, 5, 10, 20, 30, 40, 50, 60, 70, 80, 90, 100, 152, 304)
SWEEP_D = (0.06, 0.08, 0.1, 0.2, 0.3, 0.4, 0.5, 0.6, 0.7, 0.8, 0.9, 1.0, 1.1, 1.2)


def sweep_point(S, torch, band, b, N, K, P, reps=3, max_iters=200):
    """One (P, d) point of the sensitivity studies: both variants (see above)."""
    row = {}
    for tag, var in (("D", S.SAP_D), ("C", S.SAP_C)):
        h = S.sap_factor(band, N, K, P=P, variant=var, precision=S.SAP_FP32, max_iters=max_iters)
        pre, kry, its, sts = [], [], [], []
        x = torch.empty_like(b)
        for _ in range(reps):
            S.sap_refactor(h)
            _, info, st = S.sap_solve(h, b, x, raise_on_error=False)
            pre.append(info.t_factor_ms)
            kry.append(info.t_kry_ms)
            its.append(info.iters)
            sts.append(st)
        row[f"{tag}_pre"] = statistics.median(pre)
        row[f"{tag}_it"] = statistics.median(its)
        row[f"{tag}_Kry"] = statistics.median(kry)
        row[f"{tag}_Tot"] = row[f"{tag}_pre"] + row[f"{tag}_Kry"]
        row[f"status_{tag}"] = max(sts)
        del h
    row["SpdUp"] = row["D_Tot"] / row["C_Tot"]
    return row


def run_sweep(args, N=200000, K=200, Ps=SWEEP_P, ds=SWEEP_D, P_d=50, reps=3, out=sys.stdout):
    """--sweep P | d: one JSON line per point, then a table."""
    import torch
    import sap_inputs as G
    import paper_1509_07919_gb300 as S

    rows = []
    points = [(P, 1.0) for P in Ps] if args.sweep == "P" else [(P_d, d) for d in ds]
    cache = {}
    for P, d in points:
        if d not in cache:
            band_np = G.dense_banded(N, K, d, 7)
            band = torch.from_numpy(band_np).cuda()
            b = S.sap_spmv(band, N, K, torch.from_numpy(G.x_true(N, 7)).cuda())
            cache = {d: (band, b)}
        band, b = cache[d]
        if P > N // (2 * K):
            continue
        row = {"sweep": args.sweep, "N": N, "K": K, "P": P, "d": d}
        row.update(sweep_point(S, torch, band, b, N, K, P, reps=reps))
        rows.append(row)
        print(json.dumps(row), file=out, flush=True)
    key = "P" if args.sweep == "P" else "d"
    print(f"| {key} | D_pre | C_pre | D_it | C_it | D_Kry | C_Kry | D_Tot | C_Tot | SpdUp |", file=out)
    print("|---|---|---|---|---|---|---|---|---|---|", file=out)
    for r in rows:
        print(f"| {r[key]} | {r['D_pre']:.2f} | {r['C_pre']:.2f} | {r['D_it']:g} | {r['C_it']:g} | {r['D_Kry']:.2f} "
              f"| {r['C_Kry']:.2f} | {r['D_Tot']:.2f} | {r['C_Tot']:.2f} | {r['SpdUp']:.2f} |", file=out)
    return rows


def run_sparse(args, n=200000, K0=50, fill=0.1, d=1.0, seed=41, out=sys.stdout):
    """--sparse: the sparse front end (Sec. 2.2) on a synthetic sparse matrix
    (a band of half-bandwidth K0 with a fraction `fill` of its off-diagonals,
    rows shuffled and indices scrambled; sap_inputs.sparse_scrambled), then
    SaP on the reordered band: the time of each stage (ms, CUDA events around
    each call; the host stages synchronise inside their calls), K before and
    after, and the true relative residual of the original system."""
    import numpy as np
    import torch
    import sap_inputs as G
    import paper_1509_07919_gb300 as S

    sysm = G.sparse_scrambled(n, K0, fill, d, seed)
    A = S.Csr(n, torch.from_numpy(sysm.rowptr).cuda(), torch.from_numpy(sysm.col).cuda(),
              torch.from_numpy(sysm.val).cuda())
    b = torch.from_numpy(G.x_true(n, seed)).cuda()
    t = {}

    def timed(name, fn):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        w0 = time.perf_counter()
        e0.record()
        r = fn()
        e1.record()
        torch.cuda.synchronize()
        t[name] = max(e0.elapsed_time(e1), (time.perf_counter() - w0) * 1e3)
        return r

    K_in = S.sap_sparse_bandwidth(A)
    for rep in range(2):                      # the first pass warms up; the second is reported
        rownew, r, s, lp = timed("db", lambda: S.sap_db_reorder(A, scale=True))
        perm, K = timed("cm", lambda: S.sap_cm_reorder(A, rownew))
        rn = S.sap_perm_compose(perm, rownew)
        band = timed("band", lambda: S.sap_sparse_to_band(A, rn, perm, K, r, s))
        bb = S.sap_sparse_permute_rhs(b, rn, r)
        h = timed("factor", lambda: S.sap_factor(band, n, K, P=50, variant=S.SAP_D, precision=S.SAP_FP32))
        y, info, st = timed("solve", lambda: S.sap_solve(h, bb))
        x = S.sap_sparse_unpermute_solution(y, perm, s)
        del h, band
        # element drop-off: SaP of the band kept after dropping 0.1% of the
        # entries' weight, the outer iteration on the reordered sparse matrix
        Kd = timed("drop", lambda: S.sap_sparse_drop_bandwidth(A, rn, perm, K, 1e-3, r, s))
        bandd = timed("band_drop", lambda: S.sap_sparse_to_band(A, rn, perm, Kd, r, s, drop=True))
        hd = timed("factor_drop", lambda: S.sap_factor(bandd, n, Kd, P=50, variant=S.SAP_D, precision=S.SAP_FP32))
        S.sap_set_operator_csr(hd, A, rn, perm, r, s)
        yd, infod, std = timed("solve_drop", lambda: S.sap_solve(hd, bb))
        xd = S.sap_sparse_unpermute_solution(yd, perm, s)
        del hd, bandd
    # true residuals of the original sparse system on the host
    rows = np.repeat(np.arange(n), np.diff(sysm.rowptr))
    bh = b.cpu().numpy()

    def relres(xt):
        xs = xt.cpu().numpy()
        Ax = np.zeros(n)
        np.add.at(Ax, rows, sysm.val * xs[sysm.col])
        return float(np.linalg.norm(bh - Ax) / np.linalg.norm(bh))

    line = {"sparse": {"n": n, "nnz": int(sysm.rowptr[-1]), "K_in": K_in, "K0": K0, "K": K, "fill": fill, "d": d},
            "ms": t, "status": st, "iters": info.iters, "relres": relres(x),
            "drop": {"frac": 1e-3, "K": Kd, "status": std, "iters": infod.iters, "relres": relres(xd)}}
    print(json.dumps(line), file=out, flush=True)
    return line


def run_blocks(args, N=200000, K=100, P=50, d=1.0, seed=90, reps=5, out=sys.stdout):
    """--blocks: SaP with a bandwidth of its own per block (the third-stage
    reordering of Sec. 2.2) against SaP on the whole band, on a synthetic band
    whose blocks are scrambled narrow bands (sap_inputs.block_scrambled,
    half-bandwidth K, hidden per-block bandwidths in [0.4, 1] (K + 1) / 2):
    the per-block CM, then for SaP-D and SaP-C with FP32 factors the refactor
    (median over `reps`, L2 flushed before each; the phase timers of
    sap_info_t) and the solve.  The entire-spike kernel's work is reported
    against the FP32 FMA rate (t_spk_ms brackets that kernel alone)."""
    import numpy as np
    import torch
    import sap_inputs as G
    import paper_1509_07919_gb300 as S

    off = np.asarray([0] + [N // P + (1 if i < N % P else 0) for i in range(P)]).cumsum()
    sysm = G.block_scrambled(N, K, off, d, seed)
    band = torch.from_numpy(sysm.band).cuda()
    xt = torch.from_numpy(G.x_true(N, seed)).cuda()
    b = S.sap_spmv(band, N, K, xt)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    w0 = time.perf_counter()
    perm, Ki = S.sap_block_cm_reorder(band, N, K, P)
    t_cm = (time.perf_counter() - w0) * 1e3
    line = {"blocks": {"N": N, "K": K, "P": P, "d": d, "K_i_min": min(Ki), "K_i_max": max(Ki),
                       "K_i_mean": float(np.mean(Ki))},
            "ms": {"block_cm": t_cm}, "precision": "fp32 factors, fp64 Krylov"}
    for tag, var in (("D", S.SAP_D), ("C", S.SAP_C)):
        row = {}
        for kind in ("blocks", "whole_band"):
            h = (S.sap_factor_blocks(band, N, K, perm, P=P, variant=var, precision=S.SAP_FP32) if kind == "blocks"
                 else S.sap_factor(band, N, K, P=P, variant=var, precision=S.SAP_FP32))
            x = torch.empty_like(b)
            rec = {k: [] for k in ("t_factor_ms", "t_lu_ms", "t_spk_ms", "t_rdcd_ms", "t_kry_ms", "iters")}
            st = 0
            for _ in range(reps):
                flush.fill_(1.0)
                S.sap_refactor(h)
                _, info, st = S.sap_solve(h, b, x, raise_on_error=False)
                for k in rec:
                    rec[k].append(getattr(info, k))
            row[kind] = {k: statistics.median(v) for k, v in rec.items()}
            row[kind]["status"] = st
            row[kind]["err_x"] = float((x - xt).abs().max() / xt.abs().max())
            row[kind]["total_ms"] = row[kind]["t_factor_ms"] + row[kind]["t_kry_ms"]
            del h
        if var == S.SAP_C:
            # entire spikes: forward from the first nonzero row (about the whole
            # block on average), backward over all rows: 2 n_b K_b K FMAs per
            # sweep and spike column set
            fl = sum(2.0 * 2 * 2 * (off[i + s + 1] - off[i + s]) * Ki[i + s] * K for i in range(P - 1) for s in (0, 1))
            ms = row["blocks"]["t_spk_ms"]
            row["spike_kernel"] = {"flops_upper": fl, "tflops": fl / (ms * 1e-3) / 1e12 if ms > 0 else None,
                                   "note": "upper bound of the work (the forward sweep starts at the first "
                                           "row with a nonzero right-hand side)"}
        line[tag] = row
    print(json.dumps(line), file=out, flush=True)
    return line


def main():
    args = parse()
    if args.sparse:
        run_sparse(args)
    elif args.blocks:
        run_blocks(args, K=args.blocks_k)
    elif args.sweep:
        run_sweep(args)
    elif args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch64":
        run_gpu_batch(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
