"""GPU parity of the tiled plane-format assembly (pq_options.assembly = 0, the default wherever
Nnu % 4 == 0) against the general assembly kernel (assembly = 1) and against the FP64
oracle.  The two kernels evaluate the same FP32 expressions per element, so from one state
they must give the same F and, through the same products, the same Phi; only the dF part of
Sigma adds its partial sums in another order.  The shapes cover blocks of G = 4, 2 and 1
k'-momenta per CTA (L = 4, 2, 3 and the Bethe lattice), the delay line of the single-pass
kernel, and the two-gather passes of a multi-pass iteration."""
import numpy as np
import pytest

from oracle import parquet_oracle as O
from paper_1510_03330_gb300.workloads import SPLIT_BF16X3, SPLIT_FP16X3, Params, random_state

PLANE = {SPLIT_FP16X3: (1e-6, 2e-6), SPLIT_BF16X3: (5e-6, 1.5e-5)}

pytestmark = pytest.mark.gpu

SHAPES = {
    "L4_nu8": Params("square", beta=3.0, U=1.5, mu=0.1, L=4, n_nu=8, n_Omega=8),     # G = 4, delay line
    "L2_nu8": Params("square", beta=3.0, U=1.5, mu=0.0, L=2, n_nu=8, n_Omega=8),     # G = 2
    "L3_nu8": Params("square", beta=2.0, U=1.0, mu=0.3, L=3, n_nu=8, n_Omega=7, hop=0.8),  # G = 1, odd NOmega
    "bethe_nu12": Params("bethe", beta=4.0, U=1.0, mu=0.0, L=1, n_nu=12, n_Omega=9),  # nk = 1
    "L4_nu16": Params("square", beta=4.0, U=2.0, mu=0.0, L=4, n_nu=16, n_Omega=16),  # the bench block shape
    "L4_nu4": Params("square", beta=3.0, U=1.5, mu=0.1, L=4, n_nu=4, n_Omega=4),     # G = 4 at oracle-friendly size
    "L4_nu24": Params("square", beta=3.0, U=1.2, mu=0.2, L=4, n_nu=24, n_Omega=6),   # 30-word R boxes, 6 row threads
    "L2_nu32": Params("square", beta=2.5, U=1.0, mu=0.0, L=2, n_nu=32, n_Omega=9),   # G = 2, 34-word boxes, odd NOmega
}


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


@pytest.mark.parametrize("precision", list(PLANE))
@pytest.mark.parametrize("name,q_chunk", [("L4_nu8", 0), ("L4_nu8", 3), ("L2_nu8", 0), ("L3_nu8", 0),
                                          ("L3_nu8", 4), ("bethe_nu12", 0), ("L4_nu16", 0), ("L4_nu24", 0),
                                          ("L4_nu24", 2), ("L2_nu32", 0)])
def test_tiled_matches_general(name, q_chunk, precision):
    from paper_1510_03330_gb300.binding import Solver

    p = SHAPES[name]
    phi, sig = random_state(p, seed=11)
    out = {}
    for asm in (0, 1):
        with Solver(p, precision=precision, q_chunk=q_chunk, assembly=asm) as s:
            s.set_state(phi, sig)
            s.iterate(1)
            last = 0 if q_chunk == 0 else ((p.n_k - 1) // q_chunk) * q_chunk * p.n_Omega
            Fs = np.stack([np.stack([s.F(r, Q) for Q in range(last, p.n_Q)]) for r in range(4)])
            out[asm] = (all_phi(s, p), s.sigma(), np.stack([s.chi(r) for r in range(4)]), Fs)
    d = {"F": rel(out[0][3], out[1][3]), "Phi": rel(out[0][0], out[1][0]), "Sigma": rel(out[0][1], out[1][1]),
         "chi": rel(out[0][2], out[1][2])}
    print(name, q_chunk, d)
    assert d["F"] < 1e-6 and d["Phi"] < 1e-6, d
    assert rel(out[0][1], out[1][1]) < 1e-6, "Sigma"
    assert rel(out[0][2], out[1][2]) < 1e-6, "chi"


@pytest.mark.parametrize("precision", list(PLANE))
@pytest.mark.parametrize("q_chunk", [0, 5])
def test_tiled_matches_oracle(q_chunk, precision):
    from paper_1510_03330_gb300.binding import Solver

    tol, tol_phi = PLANE[precision]
    p = SHAPES["L4_nu4"]
    st = O.zero_state(p)
    errs = {}
    with Solver(p, precision=precision, q_chunk=q_chunk) as s:
        for it in range(3):
            res = O.iterate(p, st)
            st = res.state
            s.iterate(1)
            errs[f"sigma{it}"] = rel(s.sigma(), st.sigma)
        errs["phi"] = rel(all_phi(s, p), st.phi)
        chi = O.susceptibility(res.F, res.X_ph, res.X_pp)
        errs["chi_d"] = rel(s.chi(0), chi[0])
        errs["chi_s"] = rel(s.chi(2), chi[2])
        errs["F_t_last"] = rel(s.F(3, p.n_Q - 1), res.F[3, p.n_Q - 1])
    print(errs)
    assert max(v for k, v in errs.items() if k != "phi") < tol, errs
    assert errs["phi"] < tol_phi, errs
