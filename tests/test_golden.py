"""Stored closed-form values (tests/golden/, written by tests/golden/make_golden.py with numpy
and scipy only) against the oracle (CPU) and against the FP64 GPU path (-m gpu): the worked
first iteration of Sec. II.A on the 2x2 and 3x3 square lattices, the second-order
self-energy of the half-filled Bethe lattice and of the free 3x3 square lattice away from
half filling (Sec. II.B: the regulated Sigma of the first iteration from Phi = 0 is the
second-order diagram)."""
import os

import numpy as np
import pytest

from oracle import parquet_oracle as O
from paper_1510_03330_gb300.workloads import FP64, Params

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
SQUARE = Params("square", beta=3.0, U=1.5, mu=0.0, L=2, n_nu=8, n_Omega=8)
BETHE = Params("bethe", beta=5.0, U=1.0, mu=0.0, L=1, n_nu=16, n_Omega=15)
SQUARE3 = Params("square", beta=2.0, U=1.1, mu=0.15, L=3, n_nu=6, n_Omega=5, hop=0.8)


def load(name):
    return np.loadtxt(os.path.join(GOLD, name), comments="#")


def square_golden(p=SQUARE, name="first_iteration_square2_b3_u1p5.txt"):
    t = load(name)
    assert t.shape == (p.n_Q, 5) and np.array_equal(t[:, 0], np.arange(p.n_Q))
    return t[:, 1] + 1j * t[:, 2], t[:, 3] + 1j * t[:, 4]


def square3_first():
    return square_golden(SQUARE3, "first_iteration_square3_b2_u1p1_mu0p15.txt")


def square3_sigma2():
    t = load("second_order_square3_b2_u1p1_mu0p15.txt")
    g = O.make_grid(SQUARE3)
    out = np.zeros((SQUARE3.n_k, SQUARE3.n_ext), complex)
    out[t[:, 0].astype(int), t[:, 1].astype(int) - g.e_lo] = t[:, 2] + 1j * t[:, 3]
    assert t.shape[0] == out.size
    return out


def bethe_golden():
    t = load("bethe_second_order_b5_u1.txt")
    return t[:, 0].astype(int), t[:, 1] + 1j * t[:, 2]


def test_oracle_first_iteration_matches_golden():
    d, s_ = square_golden()
    res = O.iterate(SQUARE, O.zero_state(SQUARE))
    phi = res.phi_new
    scale = np.abs(d).max()
    for Q in range(SQUARE.n_Q):
        assert np.abs(phi[0, Q] - d[Q]).max() < 1e-12 * scale
        assert np.abs(phi[1, Q] - d[Q]).max() < 1e-12 * scale
        assert np.abs(phi[2, Q] - s_[Q]).max() < 1e-12 * scale
        assert np.abs(phi[3, Q]).max() == 0.0


def test_oracle_first_iteration_3x3_matches_golden():
    """The 3x3 lattice away from half filling: the first iterate and its self-energy (the
    second-order diagram with Fermi functions) against the stored values."""
    d, s_ = square3_first()
    res = O.iterate(SQUARE3, O.zero_state(SQUARE3))
    scale = np.abs(d).max()
    for Q in range(SQUARE3.n_Q):
        assert np.abs(res.phi_new[0, Q] - d[Q]).max() < 1e-12 * scale
        assert np.abs(res.phi_new[1, Q] - d[Q]).max() < 1e-12 * scale
        assert np.abs(res.phi_new[2, Q] - s_[Q]).max() < 1e-12 * scale
        assert np.abs(res.phi_new[3, Q]).max() == 0.0
    sig = square3_sigma2()
    assert np.abs(res.sigma_new - sig).max() < 1e-11 * np.abs(sig).max()


def test_oracle_bethe_first_sigma_matches_golden():
    ns, sig = bethe_golden()
    g = O.make_grid(BETHE)
    res = O.iterate(BETHE, O.zero_state(BETHE))
    got = res.sigma_new[0, ns - g.e_lo]
    assert np.abs(got - sig).max() < 2e-7


@pytest.mark.gpu
def test_gpu_first_iteration_matches_golden():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    from paper_1510_03330_gb300.binding import Solver

    d, s_ = square_golden()
    a = SQUARE.mix  # the state after one iteration from zero is a x the new iterate
    with Solver(SQUARE, precision=FP64) as s:
        s.iterate(1)
        scale = np.abs(d).max()
        for Q in range(SQUARE.n_Q):
            assert np.abs(s.Phi(0, Q) - a * d[Q]).max() < 1e-10 * scale
            assert np.abs(s.Phi(2, Q) - a * s_[Q]).max() < 1e-10 * scale
            assert np.abs(s.Phi(3, Q)).max() < 1e-14 * scale
    ns, sig = bethe_golden()
    g = O.make_grid(BETHE)
    with Solver(BETHE, precision=FP64) as s:
        s.iterate(1)
        got = s.sigma()[0, ns - g.e_lo] / BETHE.mix
    assert np.abs(got - sig).max() < 2e-7


@pytest.mark.gpu
def test_gpu_3x3_first_iteration_and_second_order_match_golden():
    """FP64 GPU path on the 3x3 lattice away from half filling against the stored values:
    the first iterate (Phi_d, Phi_s, Phi_t) and the self-energy, which at the first iteration
    is the second-order diagram; and pq_sigma_second_order of Sigma = 0 alone."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    from paper_1510_03330_gb300.binding import Solver

    d, s_ = square3_first()
    sig = square3_sigma2()
    a = SQUARE3.mix
    with Solver(SQUARE3, precision=FP64) as s:
        assert np.abs(s.sigma_second_order(np.zeros_like(sig)) - sig).max() < 1e-10 * np.abs(sig).max()
        s.iterate(1)
        scale = np.abs(d).max()
        for Q in range(SQUARE3.n_Q):
            assert np.abs(s.Phi(0, Q) - a * d[Q]).max() < 1e-10 * scale
            assert np.abs(s.Phi(1, Q) - a * d[Q]).max() < 1e-10 * scale
            assert np.abs(s.Phi(2, Q) - a * s_[Q]).max() < 1e-10 * scale
            assert np.abs(s.Phi(3, Q)).max() < 1e-14 * scale
        assert np.abs(s.sigma() - a * sig).max() < 1e-10 * np.abs(a * sig).max()
