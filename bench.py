#!/usr/bin/env python
"""Benchmark of one self-consistent parquet iteration on GB300.

A step is one parquet iteration (Dyson, bubbles, kernel functions, parquet
equations with the kernel fill, regulated Schwinger-Dyson self-energy,
Bethe-Salpeter products, mixing) of a seeded synthetic Hubbard workload.
`value` is whole-job iterations per second with the state resident in HBM;
`e2e` is the same metric through the public API from a fresh context,
including its set-up, with the self-energy copied to host every step.

  python bench.py [--gpus N --steps K --warmup W --workload NAME --precision P]
  python bench.py --impl reference ...   # the FP64 CPU oracle on a bounded sample

With N > 1 (torchrun, one process per GPU) every rank runs its own replica
solve: the solves are independent, so no collective touches the data path
(weak scaling).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1510_03330_gb300.workloads import (CONFIGS, FP64, SPLIT_BF16X3, SPLIT_BF16X6, SPLIT_FP16X3,  # noqa: E402
                                              SPLIT_TF32X3, batch_draw, device_bytes_planes)

METRIC = "parquet iter/s and BSE TFLOP/s: split-precision vs FP64 path at a stated Σ error"
UNIT = "iter/s"
DEFAULT_WORKLOAD = "square8_u2_b4"
DEFAULT_PRECISION = SPLIT_FP16X3
DTYPE = {FP64: "f64", SPLIT_TF32X3: "tf32x3 (split TF32 operands, fp32 accumulate)",
         SPLIT_BF16X3: "bf16x3 (split BF16 operands, fp32 accumulate in chunks)",
         SPLIT_FP16X3: "fp16x3 (split FP16 operands, power-of-two scaled per channel, fp32 accumulate in chunks)",
         SPLIT_BF16X6: "bf16x6"}
PLANES = (SPLIT_BF16X3, SPLIT_FP16X3)
# DRAM bytes of one launch of the products / their algorithmic bytes (32 n^2 per GEMM), from
# one ncu capture (dram__bytes_read.sum + dram__bytes_write.sum) of the same kernel on a small
# batch, scaled to the launch by its GEMM count (the traffic of one GEMM depends on n, not on the
# batch): FP16x3 at n = 1024 on 64 GEMMs; TF32x3 at n = 256 on the 4x4 lattice, scaled by
# n^2 x batch.  Kernels changed since a capture have none.
BSE_TRAFFIC = {SPLIT_FP16X3: (1.036, "ncu capture of this kernel at n = 1024 on 64 GEMMs, scaled by the GEMM count"),
               SPLIT_TF32X3: (0.986, "ncu capture on the 4x4 lattice scaled by n^2 x batch")}
FULL_TRAFFIC = {}
# kernels launched by one iteration: Dyson (2), bubbles (1), K1/K2 (1), Sigma~1 (7),
# Sigma~2 (8: tables, their prefix sums, two output passes), parquet assembly (1),
# Sigma update (1), BSE (1); FP16 planes add the kernel of the operand scales (1)
LAUNCHES_PER_ITER = 22
OWN_N = 512  # batch members with n >= OWN_N keep their own product launch (the rest are grouped)
FP64_NOMINAL_TFLOPS = 1.25  # GB300 FP64, nominal


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return d, "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def library_gemm_tflops(torch, kind):
    """Dense GEMM rate of the vendor library on this GPU (torch.matmul, i.e. cuBLAS), timed with
    CUDA events: the measured peak for the FP64 products ("fp64": DGEMM, n = 4096) and for the
    TF32 products ("tf32": FP32 GEMM on the TF32 tensor cores, n = 8192); the bf16 peak is
    MEASURED_PEAKS.json's."""
    n, dt, tf32, reps = (4096, torch.float64, False, 3) if kind == "fp64" else (8192, torch.float32, True, 20)
    old = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = tf32
    try:
        x = torch.randn(n, n, dtype=dt, device="cuda")
        y = torch.randn(n, n, dtype=dt, device="cuda")
        z = torch.empty(n, n, dtype=dt, device="cuda")
        for _ in range(2):
            torch.matmul(x, y, out=z)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(reps):
            torch.matmul(x, y, out=z)
        e1.record()
        torch.cuda.synchronize()
        tflops = 2.0 * n**3 * reps / (e0.elapsed_time(e1) * 1e-3) / 1e12
        del x, y, z
        return tflops
    finally:
        torch.backends.cuda.matmul.allow_tf32 = old
        torch.cuda.empty_cache()


def describe(name, p, precision):
    return {
        "workload": f"{name}: {p.lattice} lattice {p.L}x{p.L} k, Nnu={p.n_nu}, NOmega={p.n_Omega}, U={p.U}, "
                    f"beta={p.beta}, mu={p.mu}; BSE {4 * p.n_Q} complex GEMMs of {p.n}^3",
        "precision": precision,
        "n": p.n,
        "N_Q": p.n_Q,
        "l2": "inputs larger than L2 (vertex arrays of several GB are streamed every step)",
    }


# ----------------------------------------------------------------------------- clocks


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------- CPU oracle


def oracle_sample(p, target_s=20.0):
    """Time the FP64 oracle on a bounded sample of one iteration from the zero
    state and extrapolate to the full iteration.  Every step runs in full
    except the per-slice ones: assembly + BSE on a sample of transfer slices,
    Sigma~2 on a sample of outputs, the dF box sum on a sample of row legs."""
    from oracle import parquet_oracle as O

    g = O.make_grid(p)
    rng = np.random.default_rng(1510)
    phi = np.broadcast_to(np.zeros((), np.complex128), (4, p.n_Q, p.n, p.n))  # the zero state, held as a view
    sigma = np.zeros((p.n_k, p.n_ext), np.complex128)
    lam = O.lambda0(p.U)
    t = {}
    t0 = time.perf_counter()
    G = O.Propagator(g, sigma)
    X = O.bubbles(g, G)
    K = O.extract_kernels(g, phi)
    s1 = O.sigma1_second_order(g, sigma)
    t["full_steps"] = time.perf_counter() - t0
    del s1
    # per-slice steps: add samples round-robin until about target_s seconds of work
    cost = {"slice": [0, 0.0], "out": [0, 0.0], "row": [0, 0.0]}
    start = time.perf_counter()
    while True:
        t0 = time.perf_counter()
        Qs = rng.choice(p.n_Q, 1, replace=False)
        gam, F = O.assemble(g, phi, K, lam, Qs=Qs)
        for r in range(4):
            Xr = (X[0] if r < 2 else X[1])[Qs]
            O.BSE_SIGN[r] * np.matmul(gam[r] * Xr[:, None, :], F[r])
        cost["slice"][0] += 1
        cost["slice"][1] += time.perf_counter() - t0
        t0 = time.perf_counter()
        O.sigma2_kernel_terms(g, G, K, outputs=[(int(rng.integers(g.nk)), int(rng.integers(g.e_lo, g.e_hi + 1)))])
        cost["out"][0] += 1
        cost["out"][1] += time.perf_counter() - t0
        t0 = time.perf_counter()
        ks = rng.choice(p.n, 1, replace=False)
        gam_r, F_r = O.assemble(g, phi, K, lam, ks=ks)
        O.sigma_delta_F(g, G, F_r, K, lam, ks=ks)
        cost["row"][0] += 1
        cost["row"][1] += time.perf_counter() - t0
        if time.perf_counter() - start + t["full_steps"] > target_s:
            break
    per = {k: v[1] / v[0] for k, v in cost.items()}
    total = t["full_steps"] + per["slice"] * p.n_Q + per["out"] * g.nk * p.n_ext + per["row"] * p.n
    sampled = t["full_steps"] + sum(v[1] for v in cost.values())
    sample = (f"one iteration from the zero state: Dyson, bubbles, K1/K2, Sigma~1 in full; assembly+BSE on "
              f"{cost['slice'][0]}/{p.n_Q} transfer slices, Sigma~2 on {cost['out'][0]}/{g.nk * p.n_ext} "
              f"outputs, dF sum on {cost['row'][0]}/{p.n} row legs; {sampled:.1f} s measured, extrapolated "
              f"linearly to {total:.1f} s per iteration")
    return 1.0 / total, sample, sampled


def blas_threads():
    try:
        from threadpoolctl import threadpool_info

        return max(i.get("num_threads", 1) for i in threadpool_info())
    except Exception:
        return int(os.environ.get("OPENBLAS_NUM_THREADS", os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1)))


def oracle_baseline(workload, target_s=12.0):
    """The oracle on its bounded sample twice: with the BLAS threads the host offers (numpy's
    element-wise work runs on one thread either way, only the products of the sample use
    several) and on one core (a child process with one BLAS thread)."""
    p = CONFIGS[workload]
    v, sample, secs = oracle_sample(p, target_s)
    multi = {"value": v, "unit": UNIT, "cores": blas_threads(), "kind": "oracle",
             "sample": sample, "threads_note": "BLAS threads for the matrix products of the sample; "
                                               "the element-wise numpy work is single-threaded"}
    env = dict(os.environ, OPENBLAS_NUM_THREADS="1", OMP_NUM_THREADS="1", MKL_NUM_THREADS="1")
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-sample-only", workload,
                        "--oracle-seconds", str(target_s)], env=env, capture_output=True, text=True)
    try:
        one = json.loads(r.stdout.strip().splitlines()[-1])
        multi["one_core"] = {"value": one["value"], "unit": UNIT, "cores": 1, "sample": one["sample"]}
    except Exception:
        multi["one_core"] = {"value": None, "error": (r.stderr or r.stdout)[-300:]}
    return multi, secs


# ----------------------------------------------------------------------------- main


def max_over_ranks(x, dist, device):
    """The largest value of x over the ranks (the job takes as long as its slowest rank)."""
    if dist is None:
        return x
    import torch

    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank, world, elapsed_s):
    """Whole-job throughput of N replica ranks: all ranks' units over the slowest rank's time."""
    return world * units_per_rank / elapsed_s


BATCH = "batch64_seed1510"


def pack_waves(draw, budget, precision=SPLIT_FP16X3):
    """First-fit decreasing packing of the solves into waves of at most budget device bytes."""
    waves = []
    for i in sorted(range(len(draw)), key=lambda i: -device_bytes_planes(draw[i], precision)):
        b = device_bytes_planes(draw[i], precision)
        for w in waves:
            if w[1] + b <= budget:
                w[0].append(i)
                w[1] += b
                break
        else:
            waves.append([[i], b])
    return [sorted(w[0]) for w in waves]


def run_batch(a, world, barrier, clk_factory):
    """The 64 uneven solves: per memory wave, the solves iterated one at a time and then as one
    batch (one graph per iteration; one grouped tensor-core launch for the products of the members
    with n < OWN_N, the larger members keep their own); times summed over the waves."""
    import torch

    from paper_1510_03330_gb300.binding import Batch, Solver

    draw = batch_draw(1510, 64)
    torch.cuda.empty_cache()
    free, _ = torch.cuda.mem_get_info()
    prec = a.precision if a.precision in PLANES else SPLIT_FP16X3
    waves = pack_waves(draw, free - (8 << 30), prec)
    stream = torch.cuda.current_stream()
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    seq_ms = bat_ms = bse_ms = 0.0
    tuned = []
    clk = clk_factory()
    clk.start()
    for w in waves:
        sols = [Solver(draw[i], precision=prec, q_chunk=draw[i].n_k, time_steps=True) for i in w]
        for s_ in sols:
            s_.iterate(1)
        torch.cuda.synchronize()
        barrier()
        e0, e1 = ev(), ev()
        e0.record(stream)
        seq_steps = {}
        for _ in range(a.steps):
            for s_ in sols:
                s_.iterate(1)
                for k_, v_ in s_.step_times().items():  # each iteration ends synchronised
                    seq_steps[k_] = seq_steps.get(k_, 0.0) + v_
        e1.record(stream)
        torch.cuda.synchronize()
        wave_seq = e0.elapsed_time(e1)
        seq_ms += wave_seq
        b = Batch(sols, time_steps=True)
        b.iterate(a.warmup + 5)  # a warm-up and four tuning iterations, then the graph is captured
        torch.cuda.synchronize()
        barrier()
        f0, f1 = ev(), ev()
        f0.record(stream)
        bse = it_ms = 0.0
        for _ in range(a.steps):
            b.iterate(1)
            bse += b.times()["bse"]
            it_ms += b.times()["iteration"]
        f1.record(stream)
        torch.cuda.synchronize()
        wave_bat = f0.elapsed_time(f1)
        bat_ms += wave_bat
        bse_ms += bse
        tuned.append(dict(b.config(), solves=len(w), max_n=max(draw[i].n for i in w),
                          one_at_a_time_ms=wave_seq / a.steps, batched_ms=wave_bat / a.steps,
                          batched_over_one_at_a_time=wave_seq / wave_bat,
                          one_at_a_time_bse_ms=seq_steps.get("bse", 0.0) / a.steps,
                          one_at_a_time_assemble_ms=seq_steps.get("assemble", 0.0) / a.steps,
                          batched_bse_ms=bse / a.steps, batched_members_ms=(it_ms - bse) / a.steps))
        b.close()
        for s_ in sols:
            s_.close()
        del sols, b
        torch.cuda.empty_cache()
    clocks = clk.stop()
    # the grouped launch holds the products of the members with n < OWN_N
    flops = sum(8.0 * p.n**3 * 4 * p.n_Q for p in draw if p.n < OWN_N)
    fp16 = prec == SPLIT_FP16X3
    launches = sum((LAUNCHES_PER_ITER - 1 + fp16) * len(w) + sum(draw[i].n >= OWN_N for i in w)
                   + any(draw[i].n < OWN_N for i in w) + 1 for w in waves)
    return {"waves": len(waves), "seq_ms": seq_ms, "batch_ms": bat_ms, "bse_ms": bse_ms, "tuned": tuned,
            "flops_per_iter": flops, "clocks": clocks, "launches_per_iter": launches}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=list(CONFIGS) + [BATCH])
    ap.add_argument("--precision", default=DEFAULT_PRECISION,
                    choices=[FP64, SPLIT_TF32X3, SPLIT_BF16X3, SPLIT_FP16X3, SPLIT_BF16X6])
    ap.add_argument("--q-chunk", type=int, default=0,
                    help="q-momenta per pass of the iteration (0: all that fit in device memory)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--oracle-sample-only", default=None, help=argparse.SUPPRESS)
    ap.add_argument("--oracle-seconds", type=float, default=12.0, help=argparse.SUPPRESS)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-fp64-compare", action="store_true",
                    help="skip the FP64 run that states the split path's error and the FP64 iteration rate")
    a = ap.parse_args()
    if a.warmup < 3:
        a.warmup = 3
    if a.oracle_sample_only:
        v, sample, _ = oracle_sample(CONFIGS[a.oracle_sample_only], a.oracle_seconds)
        print(json.dumps({"value": v, "sample": sample}), flush=True)
        return 0

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if a.workload == BATCH:
        p = None
        cfg = {"workload": "64 square-lattice Hubbard solves drawn with seed 1510 (numpy PCG64): L in 2..6, "
                           "Nnu in {8,16,24,32}, NOmega = Nnu, U in [0.5, 3], beta in [2, 10], half filling",
               "precision": a.precision if a.precision in PLANES else SPLIT_FP16X3,
               "l2": "inputs larger than L2 (vertex arrays of up to 171 GB per solve)"}
    else:
        p = CONFIGS[a.workload]
        cfg = describe(a.workload, p, a.precision)
    if a.q_chunk:
        cfg["q_chunk"] = a.q_chunk
    cfg["parallelism"] = f"replicas x{world}" if world > 1 else "single GPU"

    if a.impl == "reference":
        if rank != 0:
            return 0
        if p is None:
            # the batch: the oracle on the smallest solve of the draw, scaled by the BSE flops of all 64
            draw = batch_draw(1510, 64)
            small = min(draw, key=lambda q: q.n**3 * q.n_Q)
            v1, sample1, secs = oracle_sample(small)
            scale = sum(q.n**3 * q.n_Q for q in draw) / (small.n**3 * small.n_Q)
            v = v1 / scale
            base = {"value": v, "unit": UNIT, "cores": blas_threads(), "kind": "oracle",
                    "sample": f"{sample1}; smallest solve of the draw (L={small.L}, Nnu={small.n_nu}), "
                              f"x{scale:.0f} by BSE flops"}
        else:
            base, secs = oracle_baseline(a.workload, target_s=20.0)
            v = base["value"]
        # one bounded sample of one iteration, measured once and extrapolated (see cpu_baseline.sample)
        line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": a.gpus,
                "steps": 1, "steps_requested": a.steps, "warmup": 0, "extrapolated": True,
                "ms_per_step": 1e3 / v, "measured_seconds": secs, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": cfg,
                "cpu_baseline": base,
                "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return 0

    import torch

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1510_03330_gb300 import build as B

    if rank == 0:
        B.build()
    if dist:
        dist.barrier()
    from paper_1510_03330_gb300.binding import Solver

    def barrier():
        if dist:
            dist.barrier()

    if a.workload == BATCH:
        r = run_batch(a, world, barrier, lambda: ClockSampler(local))
        ms = max_over_ranks(r["batch_ms"], dist, "cuda")
        pk, src = peaks()
        bse_tflops = r["flops_per_iter"] * a.steps / (r["bse_ms"] * 1e-3) / 1e12 if r["bse_ms"] > 0 else 0.0
        roof = {"bound": "tensor", "achieved": bse_tflops, "peak": pk["bf16_tflops"], "unit": "TFLOP/s",
                "frac": bse_tflops / pk["bf16_tflops"], "traffic": None,
                "kernel": f"bse (the grouped launch: products of the members with n < {OWN_N})",
                "executed_tensor_frac": 3.0 * bse_tflops / pk["bf16_tflops"],
                "peak_source": f"{src} bf16 burst"}
        line = {"metric": METRIC, "value": job_rate(a.steps, world, ms / 1e3), "unit": "batch iter/s (64 solves)",
                "n_gpus": world, "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms / a.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": DTYPE[cfg["precision"]],
                "data": "synthetic", "config": dict(cfg, waves=r["waves"]), "roofline": roof,
                "one_at_a_time": {"value": a.steps / (r["seq_ms"] / 1e3), "unit": "batch iter/s (64 solves)",
                                  "batched_over_one_at_a_time": r["seq_ms"] / r["batch_ms"]},
                "tuned": r["tuned"], "bse_tflops": bse_tflops, "clocks": r["clocks"],
                "gpu_launches": r["launches_per_iter"] * a.steps,
                "note": "per memory wave: solves iterated one at a time, then as one batch; times summed"}
        if rank == 0:
            print(json.dumps(line), flush=True)
        if dist:
            dist.destroy_process_group()
        return 0

    compare = None
    fp64_bytes = 16 * 4 * p.n_Q * p.n * p.n  # one complex128 copy of Phi
    free_bytes = torch.cuda.mem_get_info()[0]
    if a.precision != FP64 and not a.no_fp64_compare and 3 * fp64_bytes > free_bytes:
        # the FP64 state does not fit (a single pass needs Phi and the two operands, several
        # passes two copies of Phi): measure the FP64 product rate on the 4x4 lattice and
        # bound the FP64 iteration by its Bethe-Salpeter products alone
        small = CONFIGS["square4_u2_b5"]
        ref = Solver(small, precision=FP64, time_steps=True)
        ref.iterate(2)
        fp64_tf = 8.0 * small.n**3 * 4 * small.n_Q / (ref.step_times()["bse"] * 1e-3) / 1e12
        ref.close()
        del ref
        torch.cuda.empty_cache()
        bse_s = 8.0 * p.n**3 * 4 * p.n_Q / (fp64_tf * 1e12)
        compare = {"extrapolated": True, "fp64_bse_tflops": fp64_tf, "fp64_iter_per_s": 1.0 / bse_s,
                   "note": (f"the FP64 state ({fp64_bytes / 1e9:.0f} GB per copy of Phi) does not fit on one GPU: "
                            "FP64 product rate measured live on square4_u2_b5, FP64 iteration bounded above by "
                            "its Bethe-Salpeter products alone; the split path's errors are stated by "
                            "tests/test_gpu_parity.py::test_full_size_sampled_parity against the oracle")}
    elif a.precision != FP64 and not a.no_fp64_compare:
        # FP64 path alongside: two iterations from the zero state; the split run below starts the
        # same way, so its Sigma, F and chi_m after two iterations are compared with these
        ref = Solver(p, precision=FP64, time_steps=True)
        ref.iterate(1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ref.iterate(1)
        torch.cuda.synchronize()
        fp64_s = time.perf_counter() - t0
        fp64_bse_ms = ref.step_times()["bse"]
        ref_sig = ref.sigma()
        ref_F = [ref.F(r, p.n_Q // 2) for r in range(4)]
        ref_chi = [ref.chi(r) for r in range(4)]
        ref.close()
        del ref
        torch.cuda.empty_cache()
        compare = {"fp64_iter_per_s": 1.0 / fp64_s,
                   "fp64_bse_tflops": 8.0 * p.n**3 * 4 * p.n_Q / (fp64_bse_ms * 1e-3) / 1e12}

    def relerr(x, y):
        return float(np.abs(x - y).max() / np.abs(y).max())

    def errors_vs_fp64(sol):
        # each channel relative to its own max (F at Q = N_Q/2, chi over all Q)
        eF = [relerr(sol.F(r, p.n_Q // 2), ref_F[r]) for r in range(4)]
        eC = [relerr(sol.chi(r), ref_chi[r]) for r in range(4)]
        return {"iterations": 2, "sigma_rel_err": relerr(sol.sigma(), ref_sig),
                "F_rel_err": dict(zip("dmst", eF)), "F_max_rel_err": max(eF),
                "chi_rel_err": dict(zip("dmst", eC)), "chi_max_rel_err": max(eC),
                "F_m_rel_err": eF[1], "chi_m_rel_err": eC[1]}

    lib_peaks = {"dgemm_tflops": library_gemm_tflops(torch, "fp64"),
                 "tf32_gemm_tflops": library_gemm_tflops(torch, "tf32"),
                 "source": "cuBLAS through torch.matmul, timed live on this GPU"}
    if compare is not None:
        compare["fp64_frac_of_measured_dgemm"] = compare["fp64_bse_tflops"] / lib_peaks["dgemm_tflops"]
    solver = Solver(p, precision=a.precision, time_steps=True, q_chunk=a.q_chunk)
    if compare is not None and not compare.get("extrapolated"):
        solver.iterate(2)
        compare.update(errors_vs_fp64(solver))
        compare["note"] = ("max-norm errors relative to max|FP64| of each quantity and channel after two "
                           "iterations from the zero state; F at Q = N_Q/2, chi over all Q")
    for _ in range(a.warmup):
        solver.iterate(1)
    stream = torch.cuda.current_stream()
    clk = ClockSampler(local)
    clk.start()
    time.sleep(0.3)
    barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    step_sum = {}
    e0.record(stream)
    for _ in range(a.steps):
        solver.iterate(1)
        for k, v in solver.step_times().items():
            step_sum[k] = step_sum.get(k, 0.0) + v
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clocks = clk.stop()
    ms = max_over_ranks(e0.elapsed_time(e1), dist, "cuda")
    value = job_rate(a.steps, world, ms / 1e3)
    dev_bytes = solver.device_bytes
    solver.close()
    del solver
    torch.cuda.empty_cache()

    # roofline of the dominant kernel, timed live by the library's events on its stream
    pk, src = peaks()
    esz = 16 if a.precision == FP64 else 8
    n, nQ = p.n, p.n_Q
    steps = {k: v / a.steps for k, v in step_sum.items() if k != "total"}
    top = max(steps, key=steps.get)
    bse_flops = 8.0 * n**3 * 4 * nQ
    full_tr = FULL_TRAFFIC.get((a.workload, a.precision), {}) if a.q_chunk == 0 else {}
    # remap: read 4 Phi, write the BSE operands of 4 channels; BF16 planes are 8 bytes per
    # complex for Gamma X and 12 for F (three pieces), otherwise one complex of esz each
    # (FP16 planes: 8 + 8 bytes, the twelve complex64 words per (Q, k, k') over the channels;
    # BF16 planes: 8 + 12 with the third F piece)
    op_bytes = {SPLIT_BF16X3: 20, SPLIT_FP16X3: 16}.get(a.precision, 2 * esz)
    remap_bytes = 4.0 * nQ * n * n * (esz + op_bytes)
    bse_tflops = bse_flops / (steps["bse"] * 1e-3) / 1e12
    remap_gbs = remap_bytes / (steps["assemble"] * 1e-3) / 1e9
    if a.precision == FP64:
        bse_roof = {"bound": "alu", "achieved": bse_tflops, "peak": lib_peaks["dgemm_tflops"], "unit": "TFLOP/s",
                    "frac": bse_tflops / lib_peaks["dgemm_tflops"], "traffic": None,
                    "peak_source": "cuBLAS DGEMM measured live (FP64 pipe)",
                    "frac_of_nominal": bse_tflops / FP64_NOMINAL_TFLOPS}
    else:
        if a.precision == SPLIT_TF32X3:
            ratio, peak, psrc = None, lib_peaks["tf32_gemm_tflops"], "cuBLAS TF32 GEMM measured live"
        else:
            ratio = 1.0  # FP16 and BF16 inputs run at the same dense tensor rate
            peak, psrc = pk["bf16_tflops"] * ratio, f"{src} bf16 burst (fp16 dense rate is the same)"
        # DRAM bytes per launch as a multiple of the algorithmic 32 n^2 bytes per GEMM (read A,
        # B, Phi; write Phi)
        tr, tsrc = full_tr.get("bse"), "ncu capture of this launch at full size"
        if tr is None and a.precision in BSE_TRAFFIC and (a.precision != SPLIT_FP16X3 or n == 1024):
            tr, tsrc = BSE_TRAFFIC[a.precision]
        bse_roof = {"bound": "tensor", "achieved": bse_tflops, "peak": peak, "unit": "TFLOP/s",
                    "frac": bse_tflops / peak, "traffic": tr * 32.0 * n * n * 4 * nQ if tr else None,
                    "traffic_source": tsrc if tr else None,
                    "executed_tensor_frac": 3.0 * bse_tflops / peak,
                    "executed_note": "the split schemes issue three real products per complex product term",
                    "peak_source": psrc}
    tr = full_tr.get("assemble")
    remap_roof = {"bound": "hbm", "achieved": remap_gbs, "peak": pk["hbm_gbs"], "unit": "GB/s",
                  "frac": remap_gbs / pk["hbm_gbs"], "traffic": tr * remap_bytes if tr else None,
                  "traffic_source": "ncu capture of this launch at full size" if tr else None,
                  "peak_source": f"{src} copy bandwidth"}
    roof = bse_roof if top == "bse" else (remap_roof if top == "assemble" else bse_roof)
    roof = dict(roof, kernel=top)

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": ms / a.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": DTYPE[a.precision],
            "data": "synthetic", "config": cfg, "roofline": roof,
            "kernels": {"ms_per_iter": steps, "bse": bse_roof, "assemble": remap_roof},
            "bse_tflops": bse_tflops, "measured_library_peaks": lib_peaks,
            "gpu_launches": (LAUNCHES_PER_ITER + (a.precision == SPLIT_FP16X3)) * a.steps, "clocks": clocks,
            "device_bytes": dev_bytes}
    if compare is not None:
        compare["split_over_fp64"] = value / compare["fp64_iter_per_s"]
        line["fp64_compare"] = compare
        if a.precision != FP64 and not compare.get("extrapolated"):
            # the other split schemes on the same workload, for the same comparison
            for alt_prec in [q for q in (SPLIT_FP16X3, SPLIT_BF16X3, SPLIT_TF32X3) if q != a.precision]:
                other = Solver(p, precision=alt_prec, time_steps=True)
                other.iterate(2)
                alt = errors_vs_fp64(other)
                for _ in range(a.warmup):
                    other.iterate(1)
                torch.cuda.synchronize()
                f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                bse_ms = asm_ms = 0.0
                f0.record(stream)
                for _ in range(a.steps):
                    other.iterate(1)
                    st_ = other.step_times()
                    bse_ms += st_["bse"]
                    asm_ms += st_["assemble"]
                f1.record(stream)
                torch.cuda.synchronize()
                alt_ms = f0.elapsed_time(f1)
                other.close()
                del other
                torch.cuda.empty_cache()
                alt.update({"iter_per_s": a.steps / (alt_ms / 1e3),
                            "bse_tflops": bse_flops / (bse_ms / a.steps * 1e-3) / 1e12,
                            "ms_per_iter": {"bse": bse_ms / a.steps, "assemble": asm_ms / a.steps},
                            "over_fp64": (a.steps / (alt_ms / 1e3)) / compare["fp64_iter_per_s"]})
                alt_peak = lib_peaks["tf32_gemm_tflops"] if alt_prec == SPLIT_TF32X3 else pk["bf16_tflops"]
                alt["bse_frac"] = alt["bse_tflops"] / alt_peak
                alt["executed_tensor_frac"] = 3.0 * alt["bse_tflops"] / alt_peak
                alt["peak_source"] = ("cuBLAS TF32 GEMM measured live" if alt_prec == SPLIT_TF32X3
                                      else f"{src} bf16 burst (fp16 dense rate is the same)")
                line[alt_prec] = alt

    if not a.no_e2e:
        # end to end through the public API: a fresh context (set-up, table uploads), K iterations
        # each followed by a device->host copy of Sigma, then chi read back
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        s = Solver(p, precision=a.precision, q_chunk=a.q_chunk)
        for _ in range(a.steps):
            s.iterate(1)
            sig = s.sigma()
        chi = s.chi(1)
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        s.close()
        el = max_over_ranks(el, dist, "cuda")
        ntau = p.tau_panels * p.tau_order
        h2d = 16 * (ntau * p.n_ext + 2 * p.n_k**2) + 8 * ntau  # small transform tables (E is built on the device)
        line["e2e"] = {"value": job_rate(a.steps, world, el), "unit": UNIT, "h2d_bytes_per_step": h2d / a.steps,
                       "d2h_bytes_per_step": sig.nbytes + chi.nbytes / a.steps,
                       "note": "includes context set-up (allocation, zero state, imaginary-time transform tables)"}

    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        line["cpu_baseline"], _ = oracle_baseline(a.workload)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
