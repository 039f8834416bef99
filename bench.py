"""Benchmark: FP64 RCLUPP, RCLUPPr, CholeskyQR2 and LC2 side by side on one
tall-skinny matrix (m = 2^20, n = 128, Gaussian sketch s = 256).

One step = the four factorizations of the same resident X through the C ABI
(every row of the tall path runs: Gaussian sketch, tall LU with partial
pivoting, sketch of M, small LU / Householder / Cholesky, fused TRSM + Gram
passes, final TRSM).  Metric: TSQR GFLOP/s in the 2 m n^2 model, summed over
the four factorizations.  Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank factors its own matrix (replicas, weak
scaling, no collective on the data path); timing is the max over ranks.
--impl reference times the CPU oracle (the plain FP64 C implementation) on a
bounded row sample of the same workload.

Besides the headline step, the line carries one sub-record per remaining
single-GPU workload (untimed for the headline, each with its own CUDA-event
timings and a roofline per form): the precision form (m = 2^22, n = 256,
s = 512, kappa 1e2 / 1e8 / 1e14: binary64 against the tensor-core sketch
tiers and the binary64-emulating tiers, at equal orthogonality), the small
single matrix (m = 4096, n = 64), the batch of 512 uneven problems and the
large sparse-sign RCLUPPr (m = 2^24, n = 64).  --no-configs leaves them out.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synth  # noqa: E402

M, N, S_SKETCH, KAPPA = 1 << 20, 128, 256, 1e4
SEED_X, SEED_S = synth.kappa_seed(1, 0), synth.kappa_seed(1, 0) + 7
PATHS = ["rclupp", "rcluppr", "cholqr2", "lc2"]
# algorithmic FP64 flops per factorization (leading terms, 2-flop FMAs):
#   RCLUPP  : sketch 2smn + 2 x (TRSM mn^2 + Gram mn^2) + final TRSM mn^2
#   RCLUPPr : + tall LU mn^2 (the sketch of M replaces the sketch of X)
#   CholeskyQR2: Gram + (TRSM + Gram) + TRSM = 4 mn^2;  LC2: LU + 4 mn^2
ALGO_FLOPS = {
    "rclupp": lambda m, n, s: 2 * s * m * n + 5 * m * n * n,
    "rcluppr": lambda m, n, s: 2 * s * m * n + 6 * m * n * n,
    "cholqr2": lambda m, n, s: 4 * m * n * n,
    "lc2": lambda m, n, s: 5 * m * n * n,
}
SAMPLE_M = 1 << 15  # rows of the CPU-oracle sample
METRIC = "TSQR GFLOP/s (2mn^2 model) & roofline fraction, mixed vs FP64 at equal ||Q^T Q - I||"


def _measured_peaks():
    """Measured copy bandwidth and cuBLAS bf16 rates of this GPU type
    (MEASURED_PEAKS.json), else the fallback figures of an earlier GB300."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return (float(d["hbm_gbs"]), float(d["bf16_tflops"]), float(d["bf16_tflops_sustained"]),
                "measured")
    except (OSError, KeyError, ValueError):
        return 6800.0, 1900.0, 1700.0, "fallback"


HBM_PEAK_GBS, BF16_BURST_TFLOPS, BF16_SUSTAINED_TFLOPS, PEAKS_SOURCE = _measured_peaks()
# FP64-pipe rate: measured by the library's DFMA microbenchmark at the start of
# each run (fp64_peak()); this derived figure (SMs x 2 DFMA/clk x 2 flop x max
# SM clock, both read from the device) stands in only until then.
FP64_PEAK = {"gflops": 152 * 2070e6 * 4 / 1e9, "source": "derived before measurement"}


def measure_fp64_peak(rq):
    """FP64-pipe peak for the rooflines: the DFMA microbenchmark's rate, with
    the derived SMs x 2 DFMA/clk x 2 flop x clock beside it."""
    r = rq.fp64_peak()
    derived = r["sms"] * 2 * 2 * r["clock_mhz"] * 1e6 / 1e9
    FP64_PEAK.update({"gflops": r["gflops"], "source": "DFMA microbenchmark (measured this run)",
                      "derived_gflops": derived, "sms": r["sms"], "clock_mhz": r["clock_mhz"],
                      "microbenchmark_ms": r["ms"]})
    return FP64_PEAK


# DRAM bytes per launch of the fused TRSM + Gram kernel, from one ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum) of `bench.py --case trsm_gram
# --m 262144 --n 128 --reps 1`, scaled by the rows processed to the bench's m
# (the pass streams its rows once, so traffic grows with m).  The capture holds
# only for the kernel source it was taken on: TRAFFIC_SRC_SHA is the SHA-256 of
# csrc/tall.cu + csrc/common.cuh at capture time, and a different source gives
# traffic null.
TRAFFIC_CAPTURE = {"kernel": "trsm_gram", "m": 262144, "n": 128, "read": 269122816.0, "write": 234647296.0}
TRAFFIC_SRC_SHA = "c4e1f9dc422c538778a5481e69582956b0ddbe31e7fa437ce919b0471a710126"


def kernel_source_sha():
    import hashlib
    h = hashlib.sha256()
    for name in ("tall.cu", "common.cuh"):
        with open(os.path.join(ROOT, "paper_2412_06551_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def workload_config():
    return {
        "workload": "FP64 RCLUPP + RCLUPPr + CholeskyQR2 + LC2 side by side, one tall-skinny X",
        "m": M, "n": N, "s": S_SKETCH, "sketch": "gaussian N(0,1/s), generated on the fly",
        "kappa": KAPPA, "matrix": "U diag(sigma) V^T, sigma geometric 1 .. 1/kappa",
        "seed_x": SEED_X, "seed_s": SEED_S,
        "l2": "input 1.07 GB > 129 MB L2, no flush between steps",
        "parallelism": "replicas",
    }


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-configs", action="store_true",
                   help="leave out the sub-records of the other workloads")
    p.add_argument("--accuracy-sweep", action="store_true",
                   help="also report orthogonality/residual at kappa 1e10 and 1e15")
    p.add_argument("--case", choices=["trsm_gram", "trsm", "gram", "gram_emu", "trsm_emu", "sketch_gauss",
                                      "sketch_sparse", "sketch_srht", "precond", "lu", "rclupp",
                                      "dfma_peak", "trsm_wellcond"],
                   help="run one kernel class on an m x n matrix instead (profiler captures)")
    p.add_argument("--workload", choices=["side_by_side", "precision", "batched", "small",
                                          "large_sparse"],
                   default="side_by_side",
                   help="precision: FP64 vs tensor-core sketch RCLUPP at m=2^22, n=256, s=512; "
                        "batched: 512 uneven RCLUPP problems in one batched call")
    p.add_argument("--prec", type=int, default=0, help="precision tier for --case runs")
    p.add_argument("--kind", type=int, default=0, help="sketch kind for --case rclupp (0 Gaussian, "
                   "1 sparse-sign, 2 SRHT)")
    p.add_argument("--r0", type=int, default=0, help="R0 method for --case rclupp / precond "
                   "(0 Householder, 1 Givens)")
    p.add_argument("--m", type=int, default=1 << 18)
    p.add_argument("--n", type=int, default=N)
    p.add_argument("--reps", type=int, default=3)
    return p.parse_args()


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(t_ms, device=None):
    """Slowest rank's time (the job's time); identity without a process group."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(t_ms)
    tt = torch.tensor([float(t_ms)], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


def job_throughput(per_rank_flops, steps, t_ms, world):
    """Whole-job GFLOP/s: every rank factors its own matrix (weak scaling), so
    the job does world x per-rank work in the slowest rank's time."""
    return world * per_rank_flops * steps / (t_ms / 1e3) / 1e9


# ------------------------------------------------------------ CPU oracle ---

def oracle_sample_step(x, S):
    import oracle
    t0 = time.perf_counter()
    oracle.rclupp(x, S=S)
    oracle.rcluppr(x, S=S)
    oracle.cholqr2(x)
    oracle.lc2(x)
    return time.perf_counter() - t0


def oracle_sample_inputs():
    xs = synth.svd_matrix(SAMPLE_M, N, KAPPA, SEED_X)
    Ss = synth.gaussian_sketch(S_SKETCH, SAMPLE_M, SEED_S)
    return xs, Ss


def cpu_baseline(repeats=1):
    import oracle
    xs, Ss = oracle_sample_inputs()
    t = min(oracle_sample_step(xs, Ss) for _ in range(repeats))
    model = len(PATHS) * 2.0 * SAMPLE_M * N * N
    return {
        "value": model / t / 1e9, "unit": "GFLOP/s", "cores": oracle.num_threads(), "kind": "oracle",
        "sample": "the four factorizations on a %d x %d row sample of the same construction "
                  "(kappa %.0e, Gaussian s=%d), %.2f s per sample" % (SAMPLE_M, N, KAPPA, S_SKETCH, t),
    }


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle
    xs, Ss = oracle_sample_inputs()
    for _ in range(args.warmup):
        oracle_sample_step(xs, Ss)
    times = [oracle_sample_step(xs, Ss) for _ in range(args.steps)]
    t = sum(times) / len(times)
    model = len(PATHS) * 2.0 * SAMPLE_M * N * N
    val = model / t / 1e9
    sample = "the four factorizations on a %d x %d row sample of the workload" % (SAMPLE_M, N)
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": "GFLOP/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(),
        "cpu_baseline": {"value": val, "unit": "GFLOP/s", "cores": oracle.num_threads(),
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": val, "unit": "GFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- clocks ---

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(
                ["nvidia-smi", "-i", str(gpu_index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
                for nm, v in zip(names, r[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ GPU ---

def to_dev(a, torch, device):
    a = np.asfortranarray(a)
    return torch.from_numpy(np.ascontiguousarray(a.T)).to(device).t()


def run_path(rq, name, X, Q, R):
    if name == "rclupp":
        rq.rclupp_factor(X, s=S_SKETCH, seed=SEED_S, Q=Q, R=R)
    elif name == "rcluppr":
        rq.rclupp_r_factor(X, s=S_SKETCH, seed=SEED_S, Q=Q, R=R)
    elif name == "cholqr2":
        rq.cholqr2_factor(X, Q=Q, R=R)
    else:
        rq.lc2_factor(X, Q=Q, R=R)


def run_paths(rq, X, outs, torch):
    Qs, Rs = outs
    for i, name in enumerate(PATHS):
        run_path(rq, name, X, Qs[i], Rs[i])


def accuracy(torch, X, Q, R):
    n = Q.shape[1]
    eye = torch.eye(n, dtype=torch.float64, device=Q.device)
    orth = float(torch.linalg.norm(Q.t() @ Q - eye))
    res = float(torch.linalg.norm(Q @ R - X) / torch.linalg.norm(X))
    return orth, res


def time_call(torch, stream, fn, reps):
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    out = None
    for _ in range(reps):
        out = fn()
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1) / reps, out


# ------------------------------------------------------------ rooflines ---
#
# Roofline of one factorization in a given form (spec: the slower of the
# FP64 pipe, the tensor pipe and the bytes over HBM):
#   T_roof = max(F64 / P64, Ftc / Ptc, B / BW),  frac = T_roof / measured time.
# Counts are the algorithmic ones of the path that ran (leading terms):
#   F64  binary64 flops: Gaussian sketch 2smn, sparse sketch zeta*m*n adds,
#        tall LU mn^2, each triangular solve mn^2, each Gram m n (n+1); in the
#        emulated forms only the solves' diagonal blocks ((b+1) m n per solve,
#        b = 16 for n <= 160 else 32) and, in EMULATED, the final-pass Gram.
#   Ftc  tensor-pipe flops the split issues: tensor-core sketch 2smn per bf16
#        term (or digit: six at the digit tier) of X; emulated Gram 36 digit pairs x 2 x m x (128 x 64 tiles of
#        the upper triangle); emulated solve 36 x 2 x m x b^2 x nb(nb-1)/2.
#   B    HBM bytes: sketch read 8mn, fused solve + Gram passes 16mn each (56mn
#        for binary64 RCLUPP), a separate Gram pass 8mn (72mn emulated); the
#        LU adds its copy and one read + write of X (32mn).
# A failed reduced-tier attempt (escalation) adds its sketch and first pass.

def _emu_gram_tiles(n):
    nj, nk = -(-n // 128), -(-n // 64)
    return sum(nk - 2 * jb for jb in range(nj))


def form_counts(m, n, s, form, *, algo="rclupp", kind="gaussian", zeta=8, prec_used=None,
                first_tier=None):
    """(F64, Ftc, B) of one RCLUPP / RCLUPPr factorization in `form`
    ("fp64", "bf16", "fp32", "emulated", "emulated_all").  The sketch starts at
    `first_tier` (0 binary64, 1 bf16, 2 three-term; default: the form's) and
    ends at `prec_used` (default: no escalation)."""
    mn, mnn = float(m) * n, float(m) * n * n
    emu = form in ("emulated", "emulated_all")
    b = 16 if n <= 160 else 32
    nb = -(-n // b)
    emu_trsm_tc = 72.0 * m * b * b * nb * (nb - 1) / 2
    emu_gram_tc = 72.0 * m * _emu_gram_tiles(n) * 128 * 64
    f64 = ftc = byt = 0.0
    # sketch tiers run, in order (escalation bf16 -> three-term -> binary64;
    # the digit tier, 5, is never escalated)
    tiers = [0]
    if kind == "gaussian":
        if first_tier is None:
            first_tier = {"fp64": 0, "bf16": 1, "fp32": 2, "digits": 5, "emulated": 5,
                          "emulated_all": 5}[form]
        tiers = [first_tier]
        if first_tier in (1, 2):
            last = first_tier if prec_used is None else int(prec_used)
            order = [1, 2, 0]
            i = order.index(first_tier)
            while tiers[-1] != last and i < 2:
                i += 1
                tiers.append(order[i])
    for k, t in enumerate(tiers):
        if kind == "sparse":
            f64 += zeta * mn
        elif t == 0:
            f64 += 2.0 * s * m * n
        else:
            ftc += 2.0 * s * m * n * {1: 1, 2: 3, 5: 6}[t]
        byt += (16 if t == 5 else 8) * mn  # the digit tier's column-exponent pass reads X once more
        if k < len(tiers) - 1:  # failed attempt: its first pass too
            if emu:
                f64 += (b + 1) * mn
                ftc += emu_trsm_tc + emu_gram_tc
                byt += 24 * mn
            else:
                f64 += 2 * mnn
                byt += 16 * mn
    if algo == "rcluppr":
        f64 += mnn
        byt += 32 * mn
    if emu:
        f64 += 3 * (b + 1) * mn
        ftc += 3 * emu_trsm_tc + emu_gram_tc
        if form == "emulated":
            f64 += mnn
        else:
            ftc += emu_gram_tc
        byt += 64 * mn
    else:
        f64 += 5 * mnn
        byt += 48 * mn
    return f64, ftc, byt


def roofline_of(counts, ms, p64=None, ptc_tflops=None):
    """Roofline block of a path that took `ms` with algorithmic counts
    (F64, Ftc, B); peaks: FP64 measured this run, bf16 sustained, HBM copy."""
    f64, ftc, byt = counts
    p64 = p64 or FP64_PEAK["gflops"]
    ptc = (ptc_tflops or BF16_SUSTAINED_TFLOPS) * 1e3
    t = {"fp64": f64 / p64 / 1e6, "tensor": ftc / ptc / 1e6, "hbm": byt / HBM_PEAK_GBS / 1e6}
    bound = max(t, key=t.get)
    return {"bound": bound, "t_roof_ms": t[bound], "frac": t[bound] / ms, "fp64_flops": f64,
            "tensor_flops": ftc, "bytes": byt, "t_fp64_ms": t["fp64"], "t_tensor_ms": t["tensor"],
            "t_hbm_ms": t["hbm"]}


def svd_matrix_gpu(torch, m, n, kappa, seed, device):
    """X = U diag(sigma) V^T as in synth.svd_matrix, built on the GPU (torch's
    QR of seeded normal matrices), column-major; the host needs no copy."""
    gen = torch.Generator(device=device).manual_seed(int(seed))
    U, _ = torch.linalg.qr(torch.randn(m, n, generator=gen, dtype=torch.float64, device=device))
    V, _ = torch.linalg.qr(torch.randn(n, n, generator=gen, dtype=torch.float64, device=device))
    sig = float(kappa) ** (-torch.arange(n, dtype=torch.float64, device=device) / max(n - 1, 1))
    Xr = (U * sig) @ V.t()
    del U
    X = torch.empty((n, m), dtype=torch.float64, device=device).t()  # column-major
    X.copy_(Xr)
    del Xr
    return X


FORMS = (("fp64", 0), ("bf16", 1), ("fp32", 2), ("digits", 5), ("emulated", 3), ("emulated_all", 4))


def mixed_on_same_x(rq, torch, X, stream, fp64_paths, reps):
    """RCLUPP and RCLUPPr with the tensor-core sketch (starting at the bf16
    tier, escalating as needed) on the same X, against the FP64 paths."""
    m, n = X.shape
    out = {}
    for tier, prec in (("", rq.PREC_SKETCH_BF16), ("_emulated", rq.PREC_EMULATED),
                       ("_emulated_all", rq.PREC_EMULATED_ALL)):
        for name, fn in (("rclupp", rq.rclupp_factor), ("rcluppr", rq.rclupp_r_factor)):
            call = lambda: fn(X, s=S_SKETCH, seed=SEED_S, prec=prec)
            call()
            ms, (Q, R, info) = time_call(torch, stream, call, max(2, reps))
            o, r = accuracy(torch, X, Q, R)
            form = {"": "bf16", "_emulated": "emulated", "_emulated_all": "emulated_all"}[tier]
            cnt = form_counts(m, n, S_SKETCH, form, algo=name, prec_used=int(info.prec_used))
            out[name + tier] = {"ms": ms, "gflops_2mn2": 2.0 * m * n * n / (ms / 1e3) / 1e9,
                                "orth": o, "res": r, "prec_used": int(info.prec_used),
                                "emulated_gram": int(info.emulated),
                                "speedup_vs_fp64": fp64_paths[name]["ms"] / ms,
                                "orth_fp64": fp64_paths[name]["orth"],
                                "roofline": roofline_of(cnt, ms)}
            del Q, R
    return out


def c3_precision(rq, torch, device, reps=2):
    """RCLUPP on m = 2^22, n = 256, s = 512 at kappa 1e2, 1e8, 1e14: binary64
    against the tensor-core sketch tiers (bf16 / three-term, escalating when
    the first Cholesky shows Q1 too ill-conditioned) and the binary64-emulating
    tiers, with orthogonality and residual beside each, and the roofline of
    each form."""
    m, n, s = 1 << 22, 256, 512
    stream = torch.cuda.current_stream(device)
    rows = {}
    for k_i, kap in enumerate((1e2, 1e8, 1e14)):
        seed = synth.kappa_seed(2, k_i)
        X = svd_matrix_gpu(torch, m, n, kap, seed, device)
        row = {}
        for label, prec in FORMS:
            call = lambda: rq.rclupp_factor(X, s=s, seed=seed + 7, prec=prec, check=False)
            call()
            ms, (Q, R, info) = time_call(torch, stream, call, reps)
            entry = {"ms": ms, "gflops_2mn2": 2.0 * m * n * n / (ms / 1e3) / 1e9,
                     "status": int(info.status), "prec_used": int(info.prec_used),
                     "emulated": int(info.emulated)}
            if info.status == 0:
                o, r = accuracy(torch, X, Q, R)
                entry.update({"orth": o, "res": r})
            entry["roofline"] = roofline_of(form_counts(m, n, s, label, prec_used=int(info.prec_used)), ms)
            row[label] = entry
            del Q, R
        f = row["fp64"]
        for label, _ in FORMS[1:]:
            e = row[label]
            e["speedup_vs_fp64"] = f["ms"] / e["ms"]
            e["equal_orth"] = bool("orth" in e and "orth" in f and e["orth"] <= max(f["orth"], 1e-13))
        rows["%.0e" % kap] = row
        del X
        torch.cuda.empty_cache()
    best = {}
    for kap, row in rows.items():
        cand = [(row[l]["gflops_2mn2"], l) for l, _ in FORMS[1:] if row[l].get("equal_orth")]
        g, l = max(cand) if cand else (row["fp64"]["gflops_2mn2"], "fp64")
        best[kap] = {"fp64_gflops_2mn2": row["fp64"]["gflops_2mn2"], "best_form": l,
                     "best_gflops_2mn2": g, "speedup": g / row["fp64"]["gflops_2mn2"],
                     "orth_fp64": row["fp64"].get("orth"), "orth_best": row[l].get("orth")}
    return {"workload": "RCLUPP, m=2^22, n=256, Gaussian s=512, X = U diag(sigma) V^T (GPU-built), "
                        "binary64 vs tensor-core sketch tiers vs binary64-emulating tiers",
            "m": m, "n": n, "s": s, "reps": reps, "results": rows,
            "mixed_vs_fp64_at_equal_orth": best}


def c1_small(rq, torch, device, reps=20):
    """RCLUPP on the small single-matrix case m = 4096, n = 64, kappa = 1e8,
    Gaussian s = 128: binary64 and the emulated tiers against the oracle on
    the same X and S (the oracle runs this size in full)."""
    import oracle
    m, n, s, kap = 4096, 64, 128, 1e8
    seed = synth.kappa_seed(0, 0)
    stream = torch.cuda.current_stream(device)
    x = synth.svd_matrix(m, n, kap, seed)
    X = to_dev(x, torch, device)
    S = oracle.gaussian_sketch_matrix(s, m, seed + 7)
    t0 = time.perf_counter()
    q_o, r_o, _ = oracle.rclupp(x, S=S)
    t_oracle = time.perf_counter() - t0
    cores = oracle.num_threads()
    oracle.set_num_threads(1)  # the same factorization on one core
    t0 = time.perf_counter()
    oracle.rclupp(x, S=S)
    t_oracle1 = time.perf_counter() - t0
    oracle.set_num_threads(cores)
    rows = {"oracle": {"ms": t_oracle * 1e3, "cores": cores, "ms_one_core": t_oracle1 * 1e3,
                       "orth": oracle.orthogonality(q_o), "res": oracle.residual(x, q_o, r_o)}}
    for label, prec in (("fp64", rq.PREC_FP64), ("emulated", rq.PREC_EMULATED),
                        ("emulated_all", rq.PREC_EMULATED_ALL)):
        call = lambda: rq.rclupp_factor(X, s=s, seed=seed + 7, prec=prec)
        for _ in range(3):
            call()
        ms, (Q, R, info) = time_call(torch, stream, call, reps)
        o, r = accuracy(torch, X, Q, R)
        rows[label] = {"ms": ms, "gflops_2mn2": 2.0 * m * n * n / (ms / 1e3) / 1e9, "orth": o, "res": r,
                       "prec_used": int(info.prec_used), "emulated": int(info.emulated),
                       "roofline": roofline_of(form_counts(m, n, s, label,
                                                           prec_used=int(info.prec_used)), ms)}
        if label == "fp64":  # realised kappa: the 2-norm condition number of the computed R
            rows[label]["kappa_realised"] = float(np.linalg.cond(R.cpu().numpy()))
    return {"workload": "RCLUPP, one matrix m=4096, n=64, kappa=1e8, Gaussian s=128 "
                        "(latency-bound: X is 2 MB, L2-resident)",
            "m": m, "n": n, "s": s, "kappa": kap, "seed_x": seed, "results": rows}


def c5_large_sparse(rq, torch, device, reps=2):
    """RCLUPPr with the sparse-sign sketch on m = 2^24, n = 64 (8.6 GB),
    kappa = 1e15, s = 256, zeta = 8: binary64 and the emulated tiers."""
    m, n, s, zeta, kap = 1 << 24, 64, 256, 8, 1e15
    seed = synth.kappa_seed(4, 0)
    stream = torch.cuda.current_stream(device)
    X = svd_matrix_gpu(torch, m, n, kap, seed, device)
    torch.cuda.empty_cache()
    rows = {}
    for label, prec in (("fp64", rq.PREC_FP64), ("emulated", rq.PREC_EMULATED),
                        ("emulated_all", rq.PREC_EMULATED_ALL)):
        call = lambda: rq.rclupp_r_factor(X, s=s, kind=rq.SKETCH_SPARSE_SIGN, zeta=zeta, seed=seed + 7,
                                          prec=prec, check=False)
        call()
        ms, (Q, R, info) = time_call(torch, stream, call, reps)
        entry = {"ms": ms, "gflops_2mn2": 2.0 * m * n * n / (ms / 1e3) / 1e9, "status": int(info.status),
                 "emulated": int(info.emulated),
                 "roofline": roofline_of(form_counts(m, n, s, label, algo="rcluppr", kind="sparse",
                                                     zeta=zeta), ms)}
        if info.status == 0:
            o, r = accuracy(torch, X, Q, R)
            entry.update({"orth": o, "res": r})
        rows[label] = entry
        del Q, R
        torch.cuda.empty_cache()
    rows["speedup_emulated"] = rows["fp64"]["ms"] / rows["emulated"]["ms"]
    rows["speedup_emulated_all"] = rows["fp64"]["ms"] / rows["emulated_all"]["ms"]
    del X
    torch.cuda.empty_cache()
    return {"workload": "RCLUPPr, sparse-sign sketch s=256 zeta=8, m=2^24, n=64, kappa=1e15 "
                        "(X generated on the GPU)", "m": m, "n": n, "results": rows}


def batched_problems(count=512):
    """The batched workload: m = floor(2^U(12,17)), n uniform in
    {16, 32, 48, 64, 96, 128}, kappa = 10^U(2,12), Gaussian s = 2n."""
    return synth.batched_problems(count, synth.kappa_seed(3, 0))


# sketch tier of each form inside a batch (no escalation is possible in a
# graph): binary64, the three-term tensor-core sketch, or the digit tier
BATCH_SKETCH_TIER = {"fp64": 0, "fp32": 2, "digits": 5, "emulated": 5, "emulated_all": 5}


def c4_batched(rq, torch, device, steps=3, warmup=3):
    """512 uneven RCLUPP factorizations: one batched call (cached CUDA graph,
    autotuned branch count) against the same problems as single calls, in
    binary64 and in the precision forms, with the roofline of each."""
    stream = torch.cuda.current_stream(device)
    ms, ns, kap = batched_problems()
    base = synth.kappa_seed(3, 0)
    Xs = [svd_matrix_gpu(torch, int(m), int(n), float(k), base + 1 + i, device)
          for i, (m, n, k) in enumerate(zip(ms, ns, kap))]
    model = float(np.sum(2.0 * ms * ns * ns))
    branches, tune_ms = rq.rclupp_autotune_batched(Xs, algo=rq.ALGO_RCLUPP, seed=base)
    _, grid_div, fine_tiles = rq.rclupp_get_batch_policy()
    Qs = [rq.empty_colmajor(int(m), int(n), device) for m, n in zip(ms, ns)]
    Rs = [rq.empty_colmajor(int(n), int(n), device) for n in ns]

    def counts(form):
        tot = [0.0, 0.0, 0.0]
        for m, n in zip(ms, ns):
            c = form_counts(int(m), int(n), 2 * int(n), form, first_tier=BATCH_SKETCH_TIER[form])
            tot = [a + b for a, b in zip(tot, c)]
        return tuple(tot)

    def worst():
        wo, wr = 0.0, 0.0
        for i in range(len(Xs)):
            o, r = accuracy(torch, Xs[i], Qs[i], Rs[i])
            wo, wr = max(wo, o), max(wr, r)
        return wo, wr

    out = {}
    for label, prec in (("fp64", rq.PREC_FP64), ("fp32", rq.PREC_SKETCH_FP32),
                        ("digits", rq.PREC_SKETCH_DIGITS), ("emulated", rq.PREC_EMULATED),
                        ("emulated_all", rq.PREC_EMULATED_ALL)):
        call = lambda: rq.rclupp_factor_batched(Xs, algo=rq.ALGO_RCLUPP, seed=base, Qs=Qs, Rs=Rs,
                                                prec=prec, check=False)
        for _ in range(warmup):
            call()
        l0 = rq.kernel_launches()
        b_ms, (_, _, st) = time_call(torch, stream, call, steps)
        launches = (rq.kernel_launches() - l0) // steps
        wo, wr = worst()
        out[label] = {"ms_per_batch": b_ms, "gflops_2mn2": model / (b_ms / 1e3) / 1e9,
                      "gpu_launches_per_batch": int(launches),
                      "statuses_nonzero": int(np.count_nonzero(st)), "worst_orth": wo, "worst_res": wr,
                      "roofline": roofline_of(counts(label), b_ms)}
    for label in ("fp32", "digits", "emulated", "emulated_all"):
        out[label]["speedup_vs_fp64_batch"] = out["fp64"]["ms_per_batch"] / out[label]["ms_per_batch"]

    # the same problems as sequential single calls
    def seq():
        for i, X in enumerate(Xs):
            rq.rclupp_factor(X, seed=base + i, Q=Qs[i], R=Rs[i], check=False)
    seq()
    seq_ms, _ = time_call(torch, stream, seq, 1)
    out["fp64"]["sequential_ms"] = seq_ms
    out["fp64"]["speedup_vs_sequential"] = seq_ms / out["fp64"]["ms_per_batch"]
    del Xs, Qs, Rs
    torch.cuda.empty_cache()
    return {"workload": "batched RCLUPP: 512 problems, m=floor(2^U(12,17)), n in {16..128}, "
                        "kappa=10^U(2,12), Gaussian s=2n (GPU-built X)",
            "problems": int(len(ms)), "rows_total": int(ms.sum()), "model_flops": model,
            "branches_autotuned": branches, "grid_div_autotuned": grid_div,
            "fine_tiles_autotuned": fine_tiles, "results": out}


def run_ours(args):
    import torch

    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    device = torch.device("cuda", torch.cuda.current_device())
    import paper_2412_06551_gb300 as rq
    rq.load()
    measure_fp64_peak(rq)

    x = synth.svd_matrix(M, N, KAPPA, SEED_X + rank)
    X = to_dev(x, torch, device)
    Qs = [rq.empty_colmajor(M, N, device) for _ in PATHS]
    Rs = [rq.empty_colmajor(N, N, device) for _ in PATHS]
    stream = torch.cuda.current_stream(device)

    for _ in range(max(3, args.warmup)):
        run_paths(rq, X, (Qs, Rs), torch)
    torch.cuda.synchronize()

    # per-path times (untimed for the metric; one pass each)
    path_ms = {}
    for i, name in enumerate(PATHS):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        run_path(rq, name, X, Qs[i], Rs[i])
        e1.record(stream)
        e1.synchronize()
        path_ms[name] = e0.elapsed_time(e1)

    # ---- timed region (device-resident inputs) ----
    sampler = ClockSampler(local) if rank == 0 else None
    rq.profile_reset()
    rq.profile_enable(True)
    launches0 = rq.kernel_launches()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        run_paths(rq, X, (Qs, Rs), torch)
    e1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    launches = rq.kernel_launches() - launches0
    rq.profile_enable(False)
    prof = rq.profile_read()
    clocks = sampler.stop() if sampler else None
    t_ms = max_over_ranks(e0.elapsed_time(e1), device)
    ms_per_step = t_ms / args.steps
    model_flops = len(PATHS) * 2.0 * M * N * N
    value = job_throughput(model_flops, args.steps, t_ms, world)

    # ---- end to end: pinned host X in, Q and R of every path out ----
    # Copies run on a second stream: the next step's X is uploaded into the
    # other of two device buffers and each path's Q, R are read back while the
    # next path computes; events order every buffer's reuse.
    xh = torch.from_numpy(np.ascontiguousarray(np.asfortranarray(x).T)).pin_memory()
    Xd = [torch.empty((N, M), dtype=torch.float64, device=device) for _ in range(2)]
    qh = [torch.empty((N, M), dtype=torch.float64).pin_memory() for _ in PATHS]
    rh = [torch.empty((N, N), dtype=torch.float64).pin_memory() for _ in PATHS]
    e2e_steps = max(2, min(args.steps, 5))
    copy_s = torch.cuda.Stream(device)
    ev = lambda: torch.cuda.Event()
    x_ready, x_free = [ev(), ev()], [ev(), ev()]
    out_free = [ev() for _ in PATHS]
    torch.cuda.synchronize()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    copy_s.wait_event(f0)
    with torch.cuda.stream(copy_s):
        Xd[0].copy_(xh, non_blocking=True)
        x_ready[0].record(copy_s)
    for k in range(e2e_steps):
        b = k % 2
        stream.wait_event(x_ready[b])
        if k + 1 < e2e_steps:  # upload the next step's X meanwhile
            with torch.cuda.stream(copy_s):
                if k >= 1:
                    copy_s.wait_event(x_free[1 - b])
                Xd[1 - b].copy_(xh, non_blocking=True)
                x_ready[1 - b].record(copy_s)
        for i, name in enumerate(PATHS):
            if k >= 1:
                stream.wait_event(out_free[i])  # the previous step's Q, R are read back
            run_path(rq, name, Xd[b].t(), Qs[i], Rs[i])
            done = ev()
            done.record(stream)
            with torch.cuda.stream(copy_s):
                copy_s.wait_event(done)
                qh[i].copy_(Qs[i].t(), non_blocking=True)
                rh[i].copy_(Rs[i].t(), non_blocking=True)
                out_free[i].record(copy_s)
        x_free[b].record(stream)
    last = ev()
    last.record(copy_s)
    stream.wait_event(last)
    f1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(f0.elapsed_time(f1) / e2e_steps, device)
    h2d = M * N * 8
    d2h = len(PATHS) * (M * N * 8 + N * N * 8)

    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return

    # accuracy of the timed run (same X) and optional kappa sweep
    acc = {}
    for i, name in enumerate(PATHS):
        o, r = accuracy(torch, X, Qs[i], Rs[i])
        acc[name] = {"orth": o, "res": r}
    sweep = {}
    if args.accuracy_sweep:
        for k_i, kap in ((1, 1e10), (2, 1e15)):
            xk = to_dev(synth.svd_matrix(M, N, kap, synth.kappa_seed(1, k_i)), torch, device)
            row = {}
            for name, fn in (("rclupp", lambda Z: rq.rclupp_factor(Z, s=S_SKETCH, seed=SEED_S, check=False)),
                             ("rcluppr", lambda Z: rq.rclupp_r_factor(Z, s=S_SKETCH, seed=SEED_S, check=False)),
                             ("cholqr2", lambda Z: rq.cholqr2_factor(Z, check=False)),
                             ("lc2", lambda Z: rq.lc2_factor(Z, check=False))):
                Q, R, info = fn(xk)
                if info.status != 0:
                    row[name] = {"status": int(info.status), "step": int(info.failed_step)}
                else:
                    o, r = accuracy(torch, xk, Q, R)
                    row[name] = {"orth": o, "res": r}
            sweep["%.0e" % kap] = row
            del xk

    # dominant kernel: largest share of the timed kernel time
    tot = {k: v for k, v in prof.items() if v[0] > 0}
    dom = max(tot, key=lambda k: tot[k][1])
    dom_launches, dom_ms = tot[dom]
    avg_ms = dom_ms / dom_launches
    per_launch_flops = {
        "trsm_gram": M * (2.0 * N * N + N),
        "trsm": M * 1.0 * N * N,
        "gram": M * 1.0 * N * (N + 1),
        "sketch_gauss": 2.0 * S_SKETCH * M * N,
    }
    ach = per_launch_flops.get(dom, float("nan")) / (avg_ms / 1e3) / 1e9
    traffic, traffic_source = None, None
    if dom == TRAFFIC_CAPTURE["kernel"]:
        scale = M / TRAFFIC_CAPTURE["m"]
        if TRAFFIC_SRC_SHA is not None and kernel_source_sha() == TRAFFIC_SRC_SHA:
            traffic = (TRAFFIC_CAPTURE["read"] + TRAFFIC_CAPTURE["write"]) * scale
            traffic_source = ("ncu dram__bytes_read.sum + dram__bytes_write.sum of one launch at "
                              "m=%d, n=%d, scaled x%g; algorithmic 16 m n = %.3g bytes"
                              % (TRAFFIC_CAPTURE["m"], TRAFFIC_CAPTURE["n"], scale, 16.0 * M * N))
        else:
            traffic_source = "kernel source changed since the ncu capture: no counters for it"
    p64 = FP64_PEAK["gflops"]
    roofline = {"kernel": dom, "bound": "alu", "achieved": ach, "peak": p64,
                "unit": "GFLOP/s", "frac": ach / p64, "traffic": traffic,
                "traffic_source": traffic_source,
                "peak_source": "FP64 pipe, %s; derived %d SMs x 2 DFMA/clk x 2 flop x %d MHz = %.1f"
                               % (FP64_PEAK["source"], FP64_PEAK.get("sms", 152),
                                  FP64_PEAK.get("clock_mhz", 2070),
                                  FP64_PEAK.get("derived_gflops", 1258.56)),
                "frac_of_derived": ach / FP64_PEAK.get("derived_gflops", 1258.56),
                "avg_launch_ms": avg_ms, "launches": dom_launches}
    kernel_share = {k: round(v[1] / sum(w[1] for w in tot.values()), 4) for k, v in tot.items()}

    paths = {}
    for name in PATHS:
        f = ALGO_FLOPS[name](M, N, S_SKETCH)
        t = path_ms[name] / 1e3
        paths[name] = {"ms": path_ms[name], "gflops_2mn2": 2.0 * M * N * N / t / 1e9,
                       "fp64_gflops": f / t / 1e9, "roofline_frac": f / t / 1e9 / p64,
                       **acc[name]}
    # realised kappa of X: the 2-norm condition number of the computed R (n x n)
    kappa_realised = float(np.linalg.cond(Rs[0].cpu().numpy()))
    line = {
        "metric": METRIC, "value": value, "unit": "GFLOP/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {**workload_config(), "kappa_realised": kappa_realised},
        "roofline": roofline, "kernel_share": kernel_share,
        "paths": paths, "gpu_launches": int(launches),
        "e2e": {"value": world * model_flops / (e2e_ms / 1e3) / 1e9, "unit": "GFLOP/s",
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms},
        "clocks": clocks,
    }
    if sweep:
        line["accuracy_sweep"] = sweep
    line["mixed"] = mixed_on_same_x(rq, torch, X, stream, paths, args.steps)
    line["peaks"] = {"fp64": FP64_PEAK, "hbm_gbs": HBM_PEAK_GBS, "bf16_tflops_sustained":
                     BF16_SUSTAINED_TFLOPS, "bf16_tflops_burst": BF16_BURST_TFLOPS,
                     "source": PEAKS_SOURCE + " (MEASURED_PEAKS.json) for HBM and bf16"}
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
    if world == 1 and not args.no_configs:
        del X, Qs, Rs, Xd
        torch.cuda.empty_cache()
        t0 = time.perf_counter()
        cfg = {"c3_precision": c3_precision(rq, torch, device),
               "c1_small": c1_small(rq, torch, device),
               "c5_large_sparse": c5_large_sparse(rq, torch, device),
               "c4_batched": c4_batched(rq, torch, device)}
        cfg["wall_s"] = time.perf_counter() - t0
        line["configs"] = cfg
        line["mixed_vs_fp64"] = {"workload": cfg["c3_precision"]["workload"],
                                 "kappa": cfg["c3_precision"]["mixed_vs_fp64_at_equal_orth"]}
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def run_case(args):
    """One kernel class on a smaller matrix (for profiler captures)."""
    import torch
    import paper_2412_06551_gb300 as rq
    m, n = args.m, args.n
    x = synth.svd_matrix(m, n, KAPPA, SEED_X) if m <= (1 << 20) else \
        np.asfortranarray(synth.rng(SEED_X).standard_normal((m, n)))
    device = torch.device("cuda", 0)
    X = to_dev(x, torch, device)
    R = to_dev(np.triu(synth.rng(3).standard_normal((n, n))) / math.sqrt(n) + 2 * np.eye(n), torch,
               device)
    Yp = rq.rclupp_sketch(X, s=2 * n, seed=1) if args.case == "precond" else None
    if args.case == "dfma_peak":
        print(json.dumps({"case": "dfma_peak", **measure_fp64_peak(rq)}))
        return
    measure_fp64_peak(rq)

    def one():
        if args.case == "trsm_gram":
            rq.rclupp_trsm_gram(X, R)
        elif args.case == "trsm":
            rq.rclupp_trsm_gram(X, R, gram=False)
        elif args.case == "gram":
            rq.rclupp_gram(X)
        elif args.case == "gram_emu":
            rq.rclupp_gram_emulated(X)
        elif args.case == "trsm_emu":
            rq.rclupp_trsm_emulated(X, R)
        elif args.case == "trsm_wellcond":
            rq.rclupp_trsm_emulated_wellcond(X, R)
        elif args.case == "sketch_gauss":
            rq.rclupp_sketch(X, s=2 * n, seed=1, prec=args.prec)
        elif args.case == "sketch_sparse":
            rq.rclupp_sketch(X, s=2 * n, kind=rq.SKETCH_SPARSE_SIGN, zeta=8, seed=1)
        elif args.case == "sketch_srht":
            rq.rclupp_sketch(X, s=2 * n, kind=rq.SKETCH_SRHT, seed=1)
        elif args.case == "lu":
            rq.rclupp_tall_lupp(X)
        elif args.case == "precond":
            rq.rclupp_sketch_precond(Yp, r0=args.r0)
        elif args.case == "rclupp":
            rq.rclupp_factor(X, s=2 * n, seed=1, prec=args.prec, kind=args.kind, r0=args.r0)

    one()  # first call: workspace, tensor maps, module load
    torch.cuda.synchronize()
    rq.profile_reset()
    rq.profile_enable(True)
    for _ in range(args.reps):
        one()
    torch.cuda.synchronize()
    rq.profile_enable(False)
    prof = {k: v for k, v in rq.profile_read().items() if v[0] > 0}
    # FP64 flops of one pass: m n^2 per triangular solve or symmetric Gram
    # (n(n+1)/2 dot products of length m), 2 s m n per sketch, m n^2 - n^3/3
    # per tall LU
    flops = {"trsm_gram": 2.0 * m * n * n, "trsm": 1.0 * m * n * n, "gram": 1.0 * m * n * n,
             "gram_emu": 1.0 * m * n * n, "trsm_emu": 1.0 * m * n * n, "trsm_wellcond": 1.0 * m * n * n,
             "sketch_gauss": 4.0 * m * n * n, "lu": m * n * n - n ** 3 / 3.0}.get(args.case)
    total = sum(v[1] for v in prof.values()) / args.reps
    line = {"case": args.case, "m": m, "n": n, "reps": args.reps, "ms_per_call": total,
            "kernels": {k: {"launches": v[0] // args.reps, "ms": v[1] / args.reps} for k, v in prof.items()}}
    if flops:
        line["gflops"] = flops / (total * 1e-3) / 1e9
        line["frac_fp64_peak"] = line["gflops"] / FP64_PEAK["gflops"]
        line["fp64_peak"] = FP64_PEAK
    if args.case.startswith("sketch"):
        # the sketches read X once: 8 m n algorithmic bytes
        line["gbs"] = 8.0 * m * n / (total * 1e-3) / 1e9
        line["frac_hbm_peak"] = line["gbs"] / HBM_PEAK_GBS
    print(json.dumps(line))


def run_workload(args):
    """One sub-record on its own (one JSON line)."""
    import torch
    import paper_2412_06551_gb300 as rq
    device = torch.device("cuda", 0)
    measure_fp64_peak(rq)
    fn = {"precision": c3_precision, "small": c1_small, "large_sparse": c5_large_sparse,
          "batched": c4_batched}[args.workload]
    print(json.dumps({**fn(rq, torch, device), "fp64_peak": FP64_PEAK}), flush=True)


def main():
    args = parse()
    if args.warmup < 3:
        args.warmup = 3
    if args.case:
        run_case(args)
    elif args.workload != "side_by_side":
        run_workload(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
