"""GPU parity of the ablations the paper argues from: the kernel approximation of Sec. II.A
(pq_options.kernel_level, pq_options.edge_rule: the first-level fill, K1 only, and
second-level kernels read at the lower frequency edge alone) and the self-energy of Sec.
II.B (pq_options.sde: Eq. PA_Sigma truncated to the box instead of the regulated sum).  From one synthetic state with stripes (so that the rules
differ), one iteration on the GPU against the FP64 oracle with the same Params, in the
FP64 path (1e-10) and on the BF16x3 path (whose products also sum the row edges for the
next iteration: the lower-edge rule must not use them); a second iteration checks the
state the first one leaves."""
import numpy as np
import pytest

from oracle import parquet_oracle as O
from paper_1510_03330_gb300.workloads import FP64, SPLIT_BF16X3, SPLIT_FP16X3, Params, random_state

pytestmark = pytest.mark.gpu

BASE = Params("square", beta=3.0, U=1.5, mu=0.1, L=2, n_nu=8, n_Omega=8)


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


@pytest.mark.parametrize("precision,tol,tol_phi", [(FP64, 1e-10, 1e-10), (SPLIT_FP16X3, 1e-6, 2e-6), (SPLIT_BF16X3, 5e-6, 1.5e-5)])
@pytest.mark.parametrize("variant", [dict(kernel_level=1), dict(edge_rule="lower"),
                                     dict(kernel_level=1, edge_rule="lower"), dict(sde="truncated")])
def test_kernel_ablation_matches_oracle(precision, tol, tol_phi, variant):
    from paper_1510_03330_gb300.binding import Solver

    p = BASE.with_(**variant)
    phi, sig = random_state(p, seed=21)
    st = O.State(phi, sig)
    with Solver(p, precision=precision) as s:
        s.set_state(phi, sig)
        for it in range(2):
            res = O.iterate(p, st)
            st = res.state
            s.iterate(1)
            assert rel(s.sigma(), st.sigma) < tol, (variant, it)
        assert rel(all_phi(s, p), st.phi) < tol_phi, variant
        chi = O.susceptibility(res.F, res.X_ph, res.X_pp)
        assert rel(s.chi(0), chi[0]) < tol and rel(s.chi(2), chi[2]) < tol
    # the rule matters for this state: the default gives another Sigma
    ref = O.iterate(BASE, O.State(phi, sig))
    assert rel(O.iterate(p, O.State(phi, sig)).sigma_new, ref.sigma_new) > 1e-6
