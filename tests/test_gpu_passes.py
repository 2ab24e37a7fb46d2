"""GPU parity of the multi-pass iteration (pq_options.q_chunk): the transfers are
assembled and multiplied q_chunk q-momenta at a time, Gamma and F are rebuilt per
pass and Phi is double buffered.  The arithmetic of every element is that of the
single-pass iteration, so the result must match the oracle to the same bounds and
the single-pass Phi exactly; only the order in which the dF part of Sigma adds
its per-pass partial sums differs (rounding level)."""
import numpy as np
import pytest

from oracle import parquet_oracle as O
from paper_1510_03330_gb300.workloads import FP64, SPLIT_BF16X3, SPLIT_FP16X3, SPLIT_TF32X3, Params, random_state

# tolerances of the plane formats against the oracle: (Sigma, F, chi), raw product Phi
PLANE = {SPLIT_FP16X3: (1e-6, 2e-6), SPLIT_BF16X3: (5e-6, 1.5e-5)}

pytestmark = pytest.mark.gpu

P33 = Params("square", beta=2.0, U=1.0, mu=0.3, L=3, n_nu=8, n_Omega=7, hop=0.8)  # n = 72, 9 q-momenta
P22 = Params("square", beta=3.0, U=1.5, mu=0.0, L=2, n_nu=8, n_Omega=8)


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


def all_phi(s, p):
    return np.stack([np.stack([s.Phi(r, Q) for Q in range(p.n_Q)]) for r in range(4)])


@pytest.mark.parametrize("q_chunk", [1, 4])
def test_fp64_passes_match_oracle(q_chunk):
    from paper_1510_03330_gb300.binding import ParquetError, Solver

    p = P33
    st = O.zero_state(p)
    with Solver(p, precision=FP64, q_chunk=q_chunk) as s:
        for it in range(3):
            res = O.iterate(p, st)
            st = res.state
            s.iterate(1)
            assert rel(s.sigma(), st.sigma) < 1e-10, (q_chunk, it)
        assert rel(all_phi(s, p), st.phi) < 1e-10
        chi = O.susceptibility(res.F, res.X_ph, res.X_pp)
        for r in range(4):
            assert rel(s.chi(r), chi[r]) < 1e-10, ("chi", r)
        # F is kept for the transfers of the last pass only
        last_qb = ((p.n_k - 1) // q_chunk) * q_chunk
        Q_last = last_qb * p.n_Omega
        for r in range(4):
            assert rel(s.F(r, Q_last), res.F[r, Q_last]) < 1e-10
            assert rel(s.F(r, p.n_Q - 1), res.F[r, p.n_Q - 1]) < 1e-10
        with pytest.raises(ParquetError):
            s.F(0, 0)


@pytest.mark.parametrize("precision", [FP64, SPLIT_TF32X3, SPLIT_BF16X3, SPLIT_FP16X3])
def test_passes_reproduce_single_pass(precision):
    """From one synthetic state, one iteration in 3 passes (3 + 3 + 3 momenta) and in 1 pass
    give the same Phi bit for bit, and the same Sigma and chi up to summation order: the dF
    box sum is accumulated per CTA in the arithmetic of the path (FP64, or FP32 for the split
    forms) and the passes split it into partial sums."""
    from paper_1510_03330_gb300.binding import Solver

    p = P33
    phi, sig = random_state(p, seed=1510)
    out = {}
    for qc in (0, 3):
        with Solver(p, precision=precision, q_chunk=qc) as s:
            s.set_state(phi, sig)
            s.iterate(1)
            out[qc] = (all_phi(s, p), s.sigma(), np.stack([s.chi(r) for r in range(4)]))
    tol = 1e-13 if precision == FP64 else 1e-6
    assert np.array_equal(out[0][0], out[3][0])
    assert rel(out[3][1], out[0][1]) < tol
    assert rel(out[3][2], out[0][2]) < 10 * tol


@pytest.mark.parametrize("precision", list(PLANE))
def test_plane_passes_match_oracle(precision):
    from paper_1510_03330_gb300.binding import Solver

    tol, tol_phi = PLANE[precision]
    p = P22
    st = O.zero_state(p)
    errs = {}
    with Solver(p, precision=precision, q_chunk=3) as s:  # passes of 3 and 1 momenta
        for it in range(3):
            res = O.iterate(p, st)
            st = res.state
            s.iterate(1)
            errs[f"sigma{it}"] = rel(s.sigma(), st.sigma)
        errs["phi"] = rel(all_phi(s, p), st.phi)
        chi = O.susceptibility(res.F, res.X_ph, res.X_pp)
        errs["chi_m"] = rel(s.chi(1), chi[1])
        errs["F_last"] = rel(s.F(1, p.n_Q - 1), res.F[1, p.n_Q - 1])
    print(errs)
    assert max(v for k, v in errs.items() if k != "phi") < tol, errs
    assert errs["phi"] < tol_phi, errs


@pytest.mark.parametrize("precision", list(PLANE))
def test_plane_rows_not_multiple_of_eight(precision):
    """n = 10 (Bethe, Nnu = 10): the operand planes use rows padded to 16 elements, which the
    tensor maps treat as out of range (zero fill)."""
    from paper_1510_03330_gb300.binding import Solver

    tol, tol_phi = PLANE[precision]
    p = Params("bethe", beta=4.0, U=1.0, mu=0.0, L=1, n_nu=10, n_Omega=9)
    st = O.zero_state(p)
    with Solver(p, precision=precision) as s:
        for it in range(3):
            res = O.iterate(p, st)
            st = res.state
            s.iterate(1)
        assert rel(s.sigma(), st.sigma) < tol
        assert rel(all_phi(s, p), st.phi) < tol_phi
        Fg = np.stack([np.stack([s.F(r, Q) for Q in range(p.n_Q)]) for r in range(4)])
        assert rel(Fg, res.F) < tol


@pytest.mark.parametrize("precision", list(PLANE))
def test_plane_row_sums_follow_the_state(precision):
    """The plane-format products sum the new Phi's row edges for the next iteration's kernel
    functions (and, for FP16, the bound of the new Phi that sets the next scales); after
    pq_set_state those are stale and must not be used.  Two iterations, then a new synthetic
    state and one more iteration, against the oracle."""
    from paper_1510_03330_gb300.binding import Solver

    tol, tol_phi = PLANE[precision]
    p = P22
    phi, sig = random_state(p, seed=7)
    with Solver(p, precision=precision) as s:
        s.iterate(2)
        s.set_state(phi, sig)
        s.iterate(1)
        res = O.iterate(p, O.State(phi, sig))
        assert rel(s.sigma(), res.state.sigma) < tol
        assert rel(all_phi(s, p), res.state.phi) < tol_phi
        s.iterate(1)  # the row sums of the products just run now serve the kernel functions
        res2 = O.iterate(p, res.state)
        assert rel(s.sigma(), res2.state.sigma) < tol
