"""GPU parity of the tabulated fully irreducible vertex (pq_set_Lambda, Sec. III.A):
a local Lambda table on a frequency box smaller than the vertex box, supplemented by
(U, -U, 2U, 0) outside, in every channel; the GPU iteration must follow the oracle's
with the same table (FP64 path to 1e-10, BF16x3 to its split bound)."""
import numpy as np
import pytest

from oracle import parquet_oracle as O
from paper_1510_03330_gb300.workloads import FP64, SPLIT_BF16X3, SPLIT_FP16X3, Params

pytestmark = pytest.mark.gpu

P = Params("square", beta=2.5, U=1.2, mu=0.0, L=2, n_nu=8, n_Omega=7)
NL = 3


@pytest.fixture(scope="module", autouse=True)
def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    return torch


def rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def tables(p, nl, seed=11):
    rng = np.random.default_rng(seed)
    shape = (2 * nl + 1, 2 * nl, 2 * nl)
    return {r: (0.3 * p.U * (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)), nl) for r in range(4)}


@pytest.mark.parametrize("precision,tol,tol_phi", [(FP64, 1e-10, 1e-10), (SPLIT_FP16X3, 1e-6, 2e-6), (SPLIT_BF16X3, 5e-6, 1.5e-5)])
def test_tabulated_lambda_matches_oracle(precision, tol, tol_phi):
    from paper_1510_03330_gb300.binding import Solver

    tabs = tables(P, NL)
    lam = O.lambda_tabulated(P, tabs)
    st = O.zero_state(P)
    with Solver(P, precision=precision) as s:
        for r in range(4):
            s.set_Lambda(r, tabs[r][0], NL)
        for it in range(3):
            res = O.iterate(P, st, lam=lam)
            st = res.state
            s.iterate(1)
            assert rel(s.sigma(), st.sigma) < tol, (precision, it)
        phi = np.stack([np.stack([s.Phi(r, Q) for Q in range(P.n_Q)]) for r in range(4)])
        assert rel(phi, st.phi) < tol_phi
        F = np.stack([np.stack([s.F(r, Q) for Q in range(P.n_Q)]) for r in range(4)])
        assert rel(F, res.F) < tol


def test_set_lambda_rejects_bad_arguments():
    import ctypes as C

    from paper_1510_03330_gb300.binding import PQ_EINVAL, Solver

    t = np.zeros((5, 4, 4), dtype=np.complex128)
    ptr = t.ctypes.data_as(C.POINTER(C.c_double))
    with Solver(P) as s:
        assert s.lib.pq_set_Lambda(s.h, 4, ptr, 2) == PQ_EINVAL   # channel
        assert s.lib.pq_set_Lambda(s.h, 0, None, 2) == PQ_EINVAL  # no table
        assert s.lib.pq_set_Lambda(s.h, 0, ptr, 0) == PQ_EINVAL   # n_lambda
        assert s.lib.pq_set_Lambda(s.h, 0, ptr, 2) == 0
