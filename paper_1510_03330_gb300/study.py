"""Convergence study of the single-site parquet approximation at large U.

Sec. III of the paper compares the parquet approximation (PA, Lambda = (U, -U, 2U, 0)) with
DMFT for the half-filled Bethe lattice and reports that the PA iteration still converges at
U = 6 and 8 for beta = 2, with its quality degrading there (the large-U paragraph and its
figure).  This module runs that scan on the GPU solver: for each U and each linear-mixing
weight alpha it iterates the Bethe single-site solve from Phi = 0, Sigma = 0 until
max|dSigma| < tol, until divergence is detected (max|dSigma| growing for `window` iterations
in a row to 10x its first values, pq_options.diverge_window) or until max_iter, and
records the outcome, the iteration count, the last max|dSigma|, Im Sigma at the lowest
Matsubara frequency, and the
high-frequency tail coefficient c1 = -nu Im Sigma(i nu) at the edge of the stored range,
which the regulated self-energy keeps near U^2 n (1 - n) = U^2 / 4 (Sec. II.B).

    python -m paper_1510_03330_gb300.study [--U 1 2 4 6 8] [--alpha 0.5 0.3 0.1 0.05] [--json out.json]

The iteration itself runs in the CUDA library; this module only drives it and tabulates.
A runner other than the GPU one can be passed (same call signature) to drive another
implementation of the same iteration through the same protocol.
"""
from __future__ import annotations

import argparse
import json
import time
from dataclasses import asdict, dataclass

import numpy as np

from .workloads import BETHE, FP64, Params


@dataclass
class StudyPoint:
    U: float
    alpha: float
    status: str          # "converged", "diverged", "not converged", "non-finite"
    iterations: int
    last_dsigma: float
    im_sigma0: float     # Im Sigma(i pi T)
    tail_c1: float       # -nu Im Sigma(i nu) at the two edges of the stored range, averaged
    tail_ref: float      # U^2 n (1 - n) at half filling
    seconds: float


def bethe_params(U: float, alpha: float, beta: float = 2.0, n_nu: int = 16, n_Omega: int = 15,
                 D: float = 1.0) -> Params:
    """Half-filled single-site solve on the Bethe lattice (semicircle of half-bandwidth D)."""
    return Params(BETHE, beta=beta, U=U, mu=0.0, L=1, n_nu=n_nu, n_Omega=n_Omega, hop=D, mix=alpha)


def tail_coefficient(p: Params, sigma: np.ndarray) -> float:
    """-nu Im Sigma(i nu) at the lowest and highest stored frequency, averaged (and over momenta)."""
    e_lo = -(p.n_Omega // 2) - p.n_nu // 2
    e_hi = e_lo + p.n_ext - 1
    nu_lo, nu_hi = (2 * e_lo + 1) * np.pi / p.beta, (2 * e_hi + 1) * np.pi / p.beta
    return float(np.mean(-(nu_lo * sigma[:, 0].imag + nu_hi * sigma[:, -1].imag) / 2.0))


def im_sigma_lowest(p: Params, sigma: np.ndarray) -> float:
    """Im Sigma at nu_0 = pi T (momentum averaged)."""
    e_lo = -(p.n_Omega // 2) - p.n_nu // 2
    return float(np.mean(sigma[:, -e_lo].imag))


def gpu_runner(p: Params, max_iter: int, tol: float, window: int, precision: str = FP64):
    """Iterate with the CUDA solver; returns (status, iterations, last max|dSigma|, Sigma)."""
    from .binding import PQ_EDIVERGED, PQ_ENAN, ParquetError, Solver

    with Solver(p, precision=precision, diverge_window=window) as s:
        try:
            its, d, conv = s.iterate(max_iter, tol)
        except ParquetError as e:
            if e.status == PQ_ENAN:
                return "non-finite", -1, float("nan"), np.full((p.n_k, p.n_ext), np.nan, complex)
            raise
        status = "converged" if conv else ("diverged" if s.last_status == PQ_EDIVERGED else "not converged")
        return status, its, d, s.sigma()


def run_point(p: Params, runner, max_iter: int, tol: float, window: int) -> StudyPoint:
    t0 = time.perf_counter()
    status, its, d, sigma = runner(p, max_iter, tol, window)
    secs = time.perf_counter() - t0
    finite = bool(np.isfinite(sigma).all())
    return StudyPoint(U=p.U, alpha=p.mix, status=status, iterations=its, last_dsigma=float(d),
                      im_sigma0=im_sigma_lowest(p, sigma) if finite else float("nan"),
                      tail_c1=tail_coefficient(p, sigma) if finite else float("nan"),
                      tail_ref=p.U**2 / 4.0, seconds=secs)


def pa_convergence_study(Us=(1.0, 2.0, 4.0, 6.0, 8.0), alphas=(0.5, 0.3, 0.1, 0.05), beta: float = 2.0,
                         n_nu: int = 16, n_Omega: int = 15, max_iter: int = 3000, tol: float = 1e-8,
                         window: int = 8, runner=None) -> list[StudyPoint]:
    """The scan over U and alpha (see the module docstring)."""
    runner = runner or gpu_runner
    return [run_point(bethe_params(U, a, beta, n_nu, n_Omega), runner, max_iter, tol, window)
            for U in Us for a in alphas]


def format_table(points: list[StudyPoint]) -> str:
    rows = ["    U  alpha  status          iters  max|dSigma|  Im Sigma(i pi T)  c1 / (U^2/4)"]
    for q in points:
        rows.append(f"{q.U:5.1f}  {q.alpha:5.2f}  {q.status:14s}  {q.iterations:5d}  {q.last_dsigma:11.3e}  "
                    f"{q.im_sigma0:16.6f}  {q.tail_c1 / q.tail_ref:12.5f}")
    return "\n".join(rows)


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--U", type=float, nargs="+", default=[1.0, 2.0, 4.0, 6.0, 8.0])
    ap.add_argument("--alpha", type=float, nargs="+", default=[0.5, 0.3, 0.1, 0.05])
    ap.add_argument("--beta", type=float, default=2.0)
    ap.add_argument("--n-nu", type=int, default=16)
    ap.add_argument("--n-Omega", type=int, default=15)
    ap.add_argument("--max-iter", type=int, default=3000)
    ap.add_argument("--tol", type=float, default=1e-8)
    ap.add_argument("--window", type=int, default=8)
    ap.add_argument("--json", default=None)
    a = ap.parse_args(argv)
    pts = pa_convergence_study(a.U, a.alpha, a.beta, a.n_nu, a.n_Omega, a.max_iter, a.tol, a.window)
    print(format_table(pts))
    if a.json:
        with open(a.json, "w") as f:
            json.dump([asdict(q) for q in pts], f, indent=1)
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
