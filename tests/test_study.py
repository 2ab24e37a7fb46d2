"""The large-U convergence study of the parquet approximation (Sec. III): its bookkeeping
driven by the FP64 oracle on the CPU, and the GPU solver against the same protocol (-m gpu).

The oracle runner below applies pq_iterate's stopping rules (tolerance; divergence: max|dSigma|
grown `window` times in a row and 10x above the first `window` changes) to the oracle's iteration, so the two
runners must agree point by point."""
import numpy as np
import pytest

from oracle import parquet_oracle as O
from paper_1510_03330_gb300 import study

SMALL_BOX = dict(n_nu=8, n_Omega=7)


def oracle_runner(p, max_iter, tol, window):
    st = O.zero_state(p)
    prev, grown, dref = np.inf, 0, 0.0
    for it in range(1, max_iter + 1):
        res = O.iterate(p, st)
        st, d = res.state, res.max_dsigma
        if d < tol:
            return "converged", it, d, st.sigma
        grown = grown + 1 if d > prev else 0
        prev = d
        if it <= window:
            dref = max(dref, d)
        if window > 0 and grown >= window and d > 10.0 * dref:
            return "diverged", it, d, st.sigma
    return "not converged", max_iter, d, st.sigma


def test_small_U_converges_with_the_perturbative_tail():
    """U = 1, beta = 2: the PA converges, Im Sigma < 0, and the regulated self-energy keeps
    the tail -nu Im Sigma -> U^2 n(1 - n) = U^2/4 at the edge of the stored range (Sec. II.B)."""
    pts = study.pa_convergence_study(Us=(1.0,), alphas=(0.5,), max_iter=100, tol=1e-10, window=4,
                                     runner=oracle_runner, **SMALL_BOX)
    q = pts[0]
    assert q.status == "converged" and q.iterations < 60 and q.last_dsigma < 1e-10
    assert q.im_sigma0 < 0
    assert abs(q.tail_c1 / q.tail_ref - 1.0) < 0.02


def test_undamped_large_U_is_flagged_as_diverging():
    """U = 6 without damping (alpha = 1) diverges; the study records it as such within a few
    iterations, while strong damping (alpha = 0.1) keeps it bounded over the same span."""
    pts = study.pa_convergence_study(Us=(6.0,), alphas=(1.0, 0.1), max_iter=12, tol=1e-10, window=2,
                                     runner=oracle_runner, **SMALL_BOX)
    assert pts[0].status == "diverged" and pts[0].iterations <= 8
    assert pts[1].status == "not converged" and np.isfinite(pts[1].last_dsigma) and pts[1].last_dsigma < 10.0


def test_table_lists_every_point():
    pts = study.pa_convergence_study(Us=(0.5, 1.0), alphas=(0.5,), max_iter=3, tol=1e-12, window=0,
                                     runner=oracle_runner, **SMALL_BOX)
    t = study.format_table(pts)
    assert len(t.splitlines()) == 3 and "not converged" in t


@pytest.mark.gpu
def test_gpu_study_matches_the_oracle_protocol():
    """The GPU runner against the oracle runner, point by point: outcome, iteration count,
    last max|dSigma| and the recorded Sigma observables (FP64 path, 1e-9)."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    kw = dict(Us=(1.0, 6.0), alphas=(1.0, 0.5), max_iter=30, tol=1e-9, window=2, **SMALL_BOX)
    ref = study.pa_convergence_study(runner=oracle_runner, **kw)
    got = study.pa_convergence_study(**kw)
    for r, g in zip(ref, got):
        assert (g.U, g.alpha, g.status, g.iterations) == (r.U, r.alpha, r.status, r.iterations), (g, r)
        for f in ("last_dsigma", "im_sigma0", "tail_c1"):
            a, b = getattr(g, f), getattr(r, f)
            assert abs(a - b) <= 1e-9 * max(1.0, abs(b)), (f, g, r)
