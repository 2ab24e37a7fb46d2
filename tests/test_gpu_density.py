"""Filling and chemical potential on the GPU (pq_density, pq_options.target_density) against
the oracle: the FP64 density of G with closed-form tails, and iterations that hold a filling
away from half filling by a mu search at the start of every iteration."""
import numpy as np
import pytest

from oracle import parquet_oracle as O
from paper_1510_03330_gb300.workloads import FP64, SPLIT_FP16X3, Params

pytestmark = pytest.mark.gpu


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


def fermi(e, beta):
    return 0.5 * (1.0 - np.tanh(0.5 * beta * e))


@pytest.mark.parametrize("L,mu", [(3, 0.35), (4, -0.8), (1, 0.3)])
def test_density_of_the_free_lattice(L, mu):
    """Sigma = 0: the density is the Fermi sum (2/N) sum_k f(eps_k - mu), and the oracle's."""
    from paper_1510_03330_gb300.binding import Solver

    p = Params("square", beta=3.0, U=1.0, mu=mu, L=L, n_nu=4, n_Omega=3, hop=0.9)
    g = O.make_grid(p)
    ref = 2.0 * np.mean(fermi(g.eps - mu, p.beta))
    with Solver(p) as s:
        n = s.density()
    assert abs(n - ref) < 1e-9
    assert abs(n - O.density(p, np.zeros((p.n_k, p.n_ext), complex))) < 1e-12


@pytest.mark.parametrize("precision,tol", [(FP64, 1e-10), (SPLIT_FP16X3, 1e-6)])
def test_fixed_density_iterations_match_oracle(precision, tol):
    """Three iterations holding 0.85 electrons per site on the 3x3 lattice: mu of every
    iteration, Sigma and the density of the final state against the oracle."""
    from paper_1510_03330_gb300.binding import Solver

    p = Params("square", beta=2.5, U=1.2, mu=0.0, L=3, n_nu=4, n_Omega=3, density=0.85)
    st = O.zero_state(p)
    with Solver(p, precision=precision) as s:
        for it in range(3):
            res = O.iterate(p, st)
            st = res.state
            s.iterate(1)
            assert abs(s.mu() - res.mu) < max(tol, 1e-11) * max(1.0, abs(res.mu)), (it, s.mu(), res.mu)
            assert rel(s.sigma(), st.sigma) < tol, it
        # the state's own density at the last mu, as the oracle computes it
        n_ref = O.density(p.with_(mu=s.mu(), density=0.0), st.sigma)
        assert abs(s.density() - n_ref) < 10 * tol
    assert res.mu < 0 and np.abs(st.sigma.real).max() > 1e-4  # away from half filling


def test_fixed_density_is_refused_where_it_is_undefined():
    from paper_1510_03330_gb300.binding import Batch, ParquetError, Solver

    with pytest.raises(ParquetError):
        Solver(Params("bethe", beta=2.0, U=1.0, mu=0.0, L=1, n_nu=8, n_Omega=7, density=0.9))
    p = Params("square", beta=2.0, U=1.0, mu=0.0, L=2, n_nu=4, n_Omega=3, density=0.9)
    with Solver(p, precision=SPLIT_FP16X3) as s, pytest.raises(ParquetError):
        Batch([s])  # a batch iterates in one graph; the mu search waits on the host
