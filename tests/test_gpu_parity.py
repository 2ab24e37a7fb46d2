"""GPU parity of the CUDA parquet iteration with the FP64 oracle, through the C ABI.

The FP64 path must agree with the oracle to 1e-10 (max-norm relative error
per quantity) on the same seeded inputs: from the zero state for several
iterations, and from seeded synthetic states for one iteration.  Sizes span
several GEMM tiles and ragged tails (n = 72 is not a multiple of 64)."""
import numpy as np
import pytest

from oracle import parquet_oracle as O
from paper_1510_03330_gb300.workloads import CONFIGS, SPLIT_FP16X3, Params, random_state

pytestmark = pytest.mark.gpu
TOL_FP64 = 1e-10

CASES = {
    "square_2x2_nu8_om8": Params("square", beta=3.0, U=1.5, mu=0.0, L=2, n_nu=8, n_Omega=8),
    "square_2x2_nu6_om5": Params("square", beta=2.5, U=1.2, mu=0.0, L=2, n_nu=6, n_Omega=5),
    "square_3x3_nu8_om7_mu": Params("square", beta=2.0, U=1.0, mu=0.3, L=3, n_nu=8, n_Omega=7, hop=0.8),
    "bethe_u1_b10": CONFIGS["bethe_u1_b10"],
    "square_3x3_nu16_om8": Params("square", beta=3.0, U=1.6, mu=0.0, L=3, n_nu=16, n_Omega=8),
    "square_1x1_nu6_om5": Params("square", beta=2.0, U=1.0, mu=0.2, L=1, n_nu=6, n_Omega=5, hop=0.5),
}
TOL_SPLIT = 1e-6


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


def all_slices(s, getter, p):
    return np.stack([np.stack([getter(r, Q) for Q in range(p.n_Q)]) for r in range(4)])


@pytest.mark.parametrize("name", list(CASES))
def test_fp64_iterations_from_zero_match_oracle(name):
    from paper_1510_03330_gb300.binding import Solver

    p = CASES[name]
    st = O.zero_state(p)
    with Solver(p) as s:
        for it in range(3):
            res = O.iterate(p, st)
            st = res.state
            s.iterate(1)
            assert rel(s.sigma(), st.sigma) < TOL_FP64, (name, it, "sigma")
        assert rel(all_slices(s, s.Phi, p), st.phi) < TOL_FP64
        assert rel(all_slices(s, s.F, p), res.F) < TOL_FP64
        chi = O.susceptibility(res.F, res.X_ph, res.X_pp)
        for r in range(4):
            assert rel(s.chi(r), chi[r]) < TOL_FP64, ("chi", r)


@pytest.mark.parametrize("name", list(CASES))
def test_fp64_one_iteration_from_synthetic_state(name):
    from paper_1510_03330_gb300.binding import Solver

    p = CASES[name]
    phi, sig = random_state(p, seed=1510)
    res = O.iterate(p, O.State(phi, sig))
    with Solver(p) as s:
        s.set_state(phi, sig)
        _, dmax, _ = s.iterate(1)
        assert rel(s.sigma(), res.state.sigma) < TOL_FP64
        assert abs(dmax - res.max_dsigma) < TOL_FP64 * res.max_dsigma
        assert rel(all_slices(s, s.Phi, p), res.state.phi) < TOL_FP64
        assert rel(all_slices(s, s.F, p), res.F) < TOL_FP64


def test_solver_reports_convergence_and_state_roundtrip():
    from paper_1510_03330_gb300.binding import Solver

    p = CASES["square_2x2_nu6_om5"]
    with Solver(p) as s:
        its, d, conv = s.iterate(200, 1e-9)
        assert conv and its < 200 and d < 1e-9
        sig = s.sigma()
        phi = all_slices(s, s.Phi, p)
        with Solver(p) as t:
            t.set_state(phi, sig)
            assert rel(t.sigma(), sig) == 0.0
            assert rel(all_slices(t, t.Phi, p), phi) == 0.0


@pytest.mark.parametrize("name", ["square_3x3_nu8_om7_mu", "bethe_u1_b10"])
def test_second_order_self_energy_matches_oracle(name):
    """pq_sigma_second_order (the paper's Sigma~1) against the oracle's imaginary-time route."""
    from paper_1510_03330_gb300.binding import Solver

    p = CASES[name]
    g = O.make_grid(p)
    _, sig = random_state(p, seed=7)
    ref = O.sigma1_second_order(g, sig)
    with Solver(p) as s:
        assert rel(s.sigma_second_order(sig), ref) < TOL_FP64
        s.set_state(sigma=sig)
        assert rel(s.sigma_second_order(), ref) < TOL_FP64


@pytest.mark.parametrize("name", ["square_2x2_nu8_om8", "square_3x3_nu8_om7_mu", "bethe_u1_b10",
                                  "square_3x3_nu16_om8", "square_1x1_nu6_om5"])
def test_split_tf32x3_iterations_match_oracle(name):
    """Split path (complex64 vertices, TF32x3 tensor-core BSE) against the FP64
    oracle after three iterations from zero and one from a seeded state: Sigma,
    F and chi within 1e-6; the raw BSE output Phi, whose k''-sums cancel, within
    5e-6 (TF32x3 keeps ~2^-22 per product)."""
    from paper_1510_03330_gb300.binding import Solver
    from paper_1510_03330_gb300.workloads import SPLIT_TF32X3

    p = CASES[name]
    st = O.zero_state(p)
    errs = {}
    with Solver(p, precision=SPLIT_TF32X3) as s:
        for it in range(3):
            res = O.iterate(p, st)
            st = res.state
            s.iterate(1)
            errs[f"sigma{it}"] = rel(s.sigma(), st.sigma)
        errs["phi"] = rel(all_slices(s, s.Phi, p), st.phi)
        errs["F"] = rel(all_slices(s, s.F, p), res.F)
        chi = O.susceptibility(res.F, res.X_ph, res.X_pp)
        errs["chi_m"] = rel(s.chi(1), chi[1])
    phi, sig = random_state(p, seed=1510)
    res = O.iterate(p, O.State(phi, sig))
    with Solver(p, precision=SPLIT_TF32X3) as s:
        s.set_state(phi, sig)
        s.iterate(1)
        errs["sigma_rand"] = rel(s.sigma(), res.state.sigma)
        errs["phi_rand"] = rel(all_slices(s, s.Phi, p), res.state.phi)
        errs["F_rand"] = rel(all_slices(s, s.F, p), res.F)
    print(name, errs)
    assert max(v for k, v in errs.items() if not k.startswith("phi")) < TOL_SPLIT, errs
    assert max(v for k, v in errs.items() if k.startswith("phi")) < 5 * TOL_SPLIT, errs


# Tolerances of the plane formats on the small shapes (max-norm relative error of Sigma, F and
# chi; of the raw product Phi, whose k''-sums cancel, in the second entry): FP16x3 keeps 2^-22
# per product and its accumulation in chunks, the split path's bound of 1e-6; BF16x3 keeps
# 2^-16 per product, which is not averaged down at these sizes (measured up to 2.3e-6 on F).
PLANE_TOL = {"split_fp16x3": (TOL_SPLIT, 2 * TOL_SPLIT), "split_bf16x3": (5 * TOL_SPLIT, 1.5e-5)}


@pytest.mark.parametrize("precision", list(PLANE_TOL))
@pytest.mark.parametrize("name", list(CASES))
def test_split_planes_iterations_match_oracle(name, precision):
    """Plane-format split paths (the assembly writes FP16 or BF16 operand planes, the TMA-fed
    tensor-core products read them) against the FP64 oracle: three iterations from zero and
    one from a seeded state with stripes; Sigma, F and chi of all four channels."""
    from paper_1510_03330_gb300.binding import Solver

    p = CASES[name]
    tol, tol_phi = PLANE_TOL[precision]
    st = O.zero_state(p)
    errs = {}
    with Solver(p, precision=precision) as s:
        for it in range(3):
            res = O.iterate(p, st)
            st = res.state
            s.iterate(1)
            errs[f"sigma{it}"] = rel(s.sigma(), st.sigma)
        errs["phi"] = rel(all_slices(s, s.Phi, p), st.phi)
        errs["F"] = rel(all_slices(s, s.F, p), res.F)
        chi = O.susceptibility(res.F, res.X_ph, res.X_pp)
        for r in range(4):
            errs[f"chi{r}"] = rel(s.chi(r), chi[r])
    phi, sig = random_state(p, seed=1510)
    res = O.iterate(p, O.State(phi, sig))
    with Solver(p, precision=precision) as s:
        s.set_state(phi, sig)
        s.iterate(1)
        errs["sigma_rand"] = rel(s.sigma(), res.state.sigma)
        errs["phi_rand"] = rel(all_slices(s, s.Phi, p), res.state.phi)
        errs["F_rand"] = rel(all_slices(s, s.F, p), res.F)
    print(name, precision, errs)
    assert max(v for k, v in errs.items() if not k.startswith("phi")) < tol, errs
    assert max(v for k, v in errs.items() if k.startswith("phi")) < tol_phi, errs


def _oracle_sampled_iteration(p, phi, sigma, Qs, outs):
    """One oracle iteration restricted to sampled transfer slices Qs (Phi_new, F)
    and sampled self-energy outputs outs = [(ik, n), ...] (Sigma_new)."""
    g = O.make_grid(p)
    lam = O.lambda0(p.U)
    G = O.Propagator(g, sigma)
    X_ph, X_pp = O.bubbles(g, G)
    K = O.extract_kernels(g, phi)
    gam, F = O.assemble(g, phi, K, lam, Qs=Qs)
    phi_new = np.empty_like(gam)
    for r in range(4):
        X = (X_ph if r < 2 else X_pp)[Qs]
        phi_new[r] = O.BSE_SIGN[r] * np.matmul(gam[r] * X[:, None, :], F[r])
    s1 = O.sigma1_second_order(g, sigma)
    s2 = O.sigma2_kernel_terms(g, G, K, outputs=outs)
    sig_new = {}
    for ik, n in outs:
        v = s1[ik, n - g.e_lo] + s2[ik, n - g.e_lo]
        if g.n_lo <= n <= g.n_hi:
            kr = ik * p.n_nu + (n - g.n_lo)
            _, Fr = O.assemble(g, phi, K, lam, ks=[kr])
            v += O.sigma_delta_F(g, G, Fr, K, lam, ks=[kr])[ik, n - g.e_lo]
        sig_new[(ik, n)] = v
    return phi_new, F, sig_new, s1, X_ph, X_pp


@pytest.mark.gpu
def test_full_size_vertex_keeps_spin_rotation_crossing():
    """The 8x8 workload at full size (n = 1024, FP16x3, the launch configuration bench.py
    times), after three iterations: F satisfies the crossing relations (App. A) and the ph <->
    ph-bar crossing of SU(2) symmetry,
      F_d(k, k+d; q) = -F_d(k, k+q; d)/2 - 3 F_m(k, k+q; d)/2,  F_m(k, k+d; q) = -F_d/2 + F_m/2,
    for every k of two sampled transfers q whose shifted arguments stay in the box, with one
    shift d, so that all partners lie in the one slice d.  A property of the exact solution at
    any size; here it holds to the split path's accuracy."""
    from paper_1510_03330_gb300.binding import Solver

    p = CONFIGS["square8_u2_b4"]
    g = O.make_grid(p)
    kk, kn, qk, qm = O.box_indices(g)
    L, nom = p.L, p.n_Omega
    where = {(int(kk[i]), int(kn[i])): i for i in range(p.n)}
    dq, dm = L * 1 + 2, 1                       # shift d = (momentum (1, 2), bosonic frequency 1)
    Qd = dq * nom + dm - g.m_lo
    Qs = [3 * nom + 0 - g.m_lo, 37 * nom + 2 - g.m_lo]
    # the printed crossing F_d(k, k'; q) = F_s(k, k'; k+k'+q)/2 + 3 F_t(k, k'; k+k'+q)/2 on the
    # pairs with k + k' = c: all partners in the one slice c + q
    cq, cn = L * 3 + 5, -1                    # c = (momentum (3, 5), frequencies n + n' = -1)
    Qc = (((3 + divmod(int(qk[Qs[0]]), L)[0]) % L) * L + (5 + divmod(int(qk[Qs[0]]), L)[1]) % L) * nom \
        + cn + int(qm[Qs[0]]) + 1 - g.m_lo
    with Solver(p, precision=SPLIT_FP16X3) as s:
        s.iterate(3)
        Fd = [s.F(r, Qd) for r in (0, 1)]
        FQ = {Q: [s.F(r, Q) for r in (0, 1)] for Q in Qs}
        Fst = [s.F(r, Qc) for r in (2, 3)]
    scale = max(np.abs(f).max() for f in Fd + [x for v in FQ.values() for x in v])
    checked, worst = 0, 0.0
    for Q in Qs:
        qx, qy = divmod(int(qk[Q]), L)
        for k in range(p.n):
            kx, ky = divmod(int(kk[k]), L)
            kq = where.get((((kx + qx) % L) * L + (ky + qy) % L, int(kn[k] + qm[Q])))
            kd = where.get((((kx + dq // L) % L) * L + (ky + dq % L) % L, int(kn[k] + dm)))
            if kq is None or kd is None:
                continue
            rd = FQ[Q][0][k, kd] - (-0.5 * Fd[0][k, kq] - 1.5 * Fd[1][k, kq])
            rm = FQ[Q][1][k, kd] - (-0.5 * Fd[0][k, kq] + 0.5 * Fd[1][k, kq])
            worst = max(worst, abs(rd), abs(rm))
            checked += 1
    print("spin-rotation crossing, full size:", checked, worst / scale)
    assert checked > p.n
    assert worst <= 5 * TOL_SPLIT * scale
    Q0, checked, worst = Qs[0], 0, 0.0
    scale2 = max(scale, max(np.abs(f).max() for f in Fst))
    for k in range(p.n):
        kx, ky = divmod(int(kk[k]), L)
        kp = where.get((((cq // L - kx) % L) * L + (cq % L - ky) % L, cn - int(kn[k])))
        if kp is None:
            continue
        r1 = FQ[Q0][0][k, kp] - (0.5 * Fst[0][k, kp] + 1.5 * Fst[1][k, kp])
        r2 = FQ[Q0][1][k, kp] - (-0.5 * Fst[0][k, kp] + 0.5 * Fst[1][k, kp])
        worst = max(worst, abs(r1), abs(r2))
        checked += 1
    print("pp-ph crossing, full size:", checked, worst / scale2)
    assert checked >= p.n // 2
    assert worst <= 5 * TOL_SPLIT * scale2


@pytest.mark.parametrize("name,precision,tol,tol_F,tol_phi", [
    ("square4_u2_b5", "fp64", TOL_FP64, TOL_FP64, TOL_FP64),
    # n = 1024 with TF32 pieces: one FP32 accumulator per tile over the whole k range (the
    # kernel of the complex64 operands), measured bounds above the 1e-6 target for F and Phi
    ("square8_u2_b4", "split_tf32x3", TOL_SPLIT, 5 * TOL_SPLIT, 15 * TOL_SPLIT),
    # FP16 planes, chunked accumulation: the 1e-6 bound on Sigma, F and chi, every channel.
    # The raw product Phi of the second iteration is a small difference of large k''-terms
    # built from the complex64 (FP32) assembly: its error, ~3.7e-6 of the vertex scale, is
    # that rounding amplified by the cancellation, not the products' (BF16x3 4.2e-6, TF32x3
    # 9.6e-6 on the same slices)
    ("square8_u2_b4", "split_fp16x3", TOL_SPLIT, TOL_SPLIT, 6 * TOL_SPLIT),
    # BF16 planes (2^-16 per product), chunked accumulation
    ("square8_u2_b4", "split_bf16x3", TOL_SPLIT, 3 * TOL_SPLIT, 15 * TOL_SPLIT),
    # the large solve (n = 1536, 116 GB of Phi): several passes over the q-momenta, so F is
    # kept for the last pass only and is checked on the sampled slices that fall in it
    ("square8_u3_b8_nu24", "split_fp16x3", TOL_SPLIT, TOL_SPLIT, 6 * TOL_SPLIT)])
def test_full_size_sampled_parity(name, precision, tol, tol_F, tol_phi):
    """The benchmark workloads at full size, in the launch configuration bench.py
    times: iterations 1 and 2 from the zero state, compared on sampled transfer
    slices (Phi, F) and sampled self-energy outputs.  The oracle holds the zero
    state and the first iterate (constant in k, k' per Q by the worked example of
    Sec. II.A) as broadcast views, so it needs no full-size host arrays."""
    from paper_1510_03330_gb300.binding import ParquetError, Solver

    p = CONFIGS[name]
    g = O.make_grid(p)
    rng = np.random.default_rng(3)
    Qs = np.array(sorted({0, p.n_Q - 1, int(rng.integers(p.n_Q)), int(rng.integers(p.n_Q))}))
    outs = [(0, g.e_lo), (int(rng.integers(g.nk)), 0), (g.nk - 1, g.n_hi)]
    shape = (4, p.n_Q, p.n, p.n)
    def kept_F(s):
        # every sampled slice of a single-pass solve; the last pass's slices of a multi-pass one
        out = {}
        for Q in Qs:
            try:
                out[Q] = [s.F(r, Q) for r in range(4)]
            except ParquetError:
                pass
        assert p.n_Q - 1 in out
        return out

    with Solver(p, precision=precision) as s:
        s.iterate(1)
        gpu1 = {"sigma": s.sigma(), "phi": {Q: [s.Phi(r, Q) for r in range(4)] for Q in Qs}, "F": kept_F(s)}
        s.iterate(1)
        gpu2 = {"sigma": s.sigma(), "phi": {Q: [s.Phi(r, Q) for r in range(4)] for Q in Qs}, "F": kept_F(s),
                "chi": [s.chi(r) for r in range(4)]}
    a = p.mix
    # iteration 1 from the zero state
    zero = np.broadcast_to(np.zeros((), complex), shape)
    sig0 = np.zeros((p.n_k, p.n_ext), complex)
    phi1, F1, sig1, s1, X_ph, X_pp = _oracle_sampled_iteration(p, zero, sig0, Qs, outs)

    def check(gpu, refs, bound, what, per_channel):
        # max-norm error over the sampled slices, relative to the channel's own max |ref| (F),
        # or to the vertex's max |ref| over the four channels (Phi: Psi_t, a difference of
        # channels, is far smaller than the others at the first iterations)
        vscale = max(np.abs(refs[i][r]).max() for i in range(len(Qs)) for r in range(4))
        for r in range(4):
            kept = [(i, Q) for i, Q in enumerate(Qs) if Q in gpu]
            scale = max(np.abs(refs[i][r]).max() for i, _ in kept) if per_channel else vscale
            if scale == 0.0:  # Psi_t of the first iterate vanishes identically
                scale = vscale
            err = max(np.abs(gpu[Q][r] - refs[i][r]).max() for i, Q in kept)
            print(what, r, err / scale)
            assert err <= bound * scale + 1e-300, (what, r, err, scale)

    check(gpu1["phi"], [[a * phi1[r, i] for r in range(4)] for i in range(len(Qs))], tol_phi, "phi1", False)
    check(gpu1["F"], [[F1[r, i] for r in range(4)] for i in range(len(Qs))], tol_F, "F1", True)
    for (ik, n), v in sig1.items():
        assert abs(gpu1["sigma"][ik, n - g.e_lo] - a * v) <= tol * np.abs(a * s1).max()
    # the first iterate: Sigma~2 and dF vanish (K = 0, F = Lambda), Phi is constant per (r, Q)
    l0 = O.lambda0(p.U)
    const = np.stack([O.BSE_SIGN[r] * l0[r] ** 2 * (X_ph if r < 2 else X_pp).sum(axis=1) for r in range(4)])
    for i, Q in enumerate(Qs):
        assert np.abs(phi1[:, i] - const[:, Q, None, None]).max() <= 1e-12 * np.abs(const).max()
    phi_state = np.broadcast_to((a * const)[:, :, None, None], shape)
    sig_state = a * s1
    phi2, F2, sig2, s1b, _, _ = _oracle_sampled_iteration(p, phi_state, sig_state, Qs, outs)
    scale = np.abs(s1b).max()
    for (ik, n), v in sig2.items():
        ref = a * v + (1 - a) * sig_state[ik, n - g.e_lo]
        assert abs(gpu2["sigma"][ik, n - g.e_lo] - ref) <= tol * scale
    check(gpu2["phi"], [[a * phi2[r, i] + (1 - a) * phi_state[r, Q] for r in range(4)] for i, Q in enumerate(Qs)],
          tol_phi, "phi2", False)
    check(gpu2["F"], [[F2[r, i] for r in range(4)] for i in range(len(Qs))], tol_F, "F2", True)
    # chi of the second iteration at the sampled transfers, all four channels (App. A, "Notations")
    X2 = O.bubbles(g, O.Propagator(g, sig_state))
    for r in range(4):
        X = (X2[0] if r < 2 else X2[1])[Qs]
        ref = -X.sum(axis=1) - np.einsum("qk,qkl,ql->q", X, F2[r], X)
        err = np.abs(gpu2["chi"][r][Qs] - ref).max() / np.abs(ref).max()
        print("chi2", r, err)
        assert err <= tol, ("chi", r, err)


def test_nonfinite_self_energy_is_reported_and_poisons_the_context():
    """A NaN planted in Sigma on the host comes back as PQ_ENAN from pq_iterate;
    the context then refuses further work with PQ_ESTATE (no device fault involved)."""
    from paper_1510_03330_gb300.binding import PQ_ENAN, PQ_ESTATE, ParquetError, Solver

    p = CASES["square_2x2_nu6_om5"]
    _, sig = random_state(p, seed=5)
    sig[1, 3] = np.nan
    with Solver(p) as s:
        s.set_state(sigma=sig)
        with pytest.raises(ParquetError) as e:
            s.iterate(1)
        assert e.value.status == PQ_ENAN
        with pytest.raises(ParquetError) as e2:
            s.iterate(1)
        assert e2.value.status == PQ_ESTATE
