"""Pins of the FP64 oracle against facts fixed by the paper and the mathematics.

Each test checks the oracle against something other than itself: a closed form
(second-order self-energy, free bubbles), the paper's worked first iteration,
identities the exact equations obey (crossing, Pauli, particle-hole symmetry,
the BSE fixed point), the high-frequency tail, or brute force on tiny inputs.
"""
import numpy as np
import pytest
from scipy import integrate

from oracle import parquet_oracle as O
from paper_1510_03330_gb300.workloads import CONFIGS, Params

SMALL = Params("square", beta=3.0, U=1.5, mu=0.0, L=2, n_nu=8, n_Omega=8)
SMALL_ODD = Params("square", beta=2.5, U=1.2, mu=0.0, L=2, n_nu=6, n_Omega=5)
BETHE_SMALL = Params("bethe", beta=5.0, U=1.0, mu=0.0, L=1, n_nu=16, n_Omega=15)


def fermi(e, beta):
    return 0.5 * (1.0 - np.tanh(0.5 * beta * e))


# --------------------------------------------------------------------------- one-particle pins


@pytest.mark.parametrize("hop,mu,beta", [(0.1, 0.0, 5.0), (0.0, 0.0, 4.0), (0.3, 0.5, 3.0)])
def test_second_order_single_level_closed_form(hop, mu, beta):
    """Sigma~1 of a single level a (L = 1 square lattice, Sigma = 0) equals the
    textbook second-order result U^2 f(a)(1-f(a))/(i nu - a) (Sec. II.B: Sigma~1
    is the second-order diagram)."""
    p = Params("square", beta=beta, U=0.7, mu=mu, L=1, n_nu=8, n_Omega=7, hop=hop)
    g = O.make_grid(p)
    s1 = O.sigma1_second_order(g, np.zeros((1, p.n_ext), complex))
    a = -4.0 * hop - mu
    f = fermi(a, beta)
    n = np.arange(-(p.n_Omega // 2) - p.n_nu // 2, p.n_ext - (p.n_Omega // 2) - p.n_nu // 2)
    nu = (2 * n + 1) * np.pi / beta
    ref = p.U**2 * f * (1 - f) / (1j * nu - a)
    assert np.abs(s1[0] - ref).max() < 1e-11 * np.abs(ref).max()


def test_second_order_lattice_closed_form():
    """Sigma~1 on a 2x2 lattice with free propagators equals the momentum-space
    second-order formula with Fermi functions,
    (U^2/N^2) sum_{a,b} [(1-f_a)(1-f_b) f_c + f_a f_b (1-f_c)] / (i nu - e_a - e_b + e_c),
    c = a + b - k.  Pins the 1/N per momentum sum and the real-space route."""
    p = Params("square", beta=2.0, U=1.1, mu=0.2, L=2, n_nu=4, n_Omega=5, hop=0.6)
    g = O.make_grid(p)
    s1 = O.sigma1_second_order(g, np.zeros((4, p.n_ext), complex))
    L = 2
    mom = [(i, j) for i in range(L) for j in range(L)]
    e = np.array([-2 * p.hop * (np.cos(2 * np.pi * i / L) + np.cos(2 * np.pi * j / L)) - p.mu for i, j in mom])
    f = fermi(e, p.beta)
    n = np.arange(p.n_ext) - (p.n_Omega // 2) - p.n_nu // 2
    nu = (2 * n + 1) * np.pi / p.beta
    for ik, (kx, ky) in enumerate(mom):
        ref = np.zeros_like(nu, dtype=complex)
        for ia, (ax, ay) in enumerate(mom):
            for ib, (bx, by) in enumerate(mom):
                ic = mom.index(((ax + bx - kx) % L, (ay + by - ky) % L))
                num = (1 - f[ia]) * (1 - f[ib]) * f[ic] + f[ia] * f[ib] * (1 - f[ic])
                ref += num / (1j * nu - e[ia] - e[ib] + e[ic])
        ref *= p.U**2 / len(mom) ** 2
        assert np.abs(s1[ik] - ref).max() < 1e-11 * np.abs(ref).max()


def test_bethe_weiss_function_is_semicircle_hilbert_transform():
    """The Bethe G0 equals int rho(e)/(i nu - e) de with rho the semicircle of half-bandwidth D."""
    p = CONFIGS["bethe_u1_b10"]
    g = O.make_grid(p)
    Dh = p.hop
    rho = lambda e: 2.0 / (np.pi * Dh**2) * np.sqrt(max(Dh * Dh - e * e, 0.0))  # noqa: E731
    for n in (-5, -1, 0, 3, 20):
        nu = (2 * n + 1) * np.pi / p.beta
        re = integrate.quad(lambda e: rho(e) * (-e) / (nu * nu + e * e), -Dh, Dh, epsabs=1e-14)[0]
        im = integrate.quad(lambda e: rho(e) * (-nu) / (nu * nu + e * e), -Dh, Dh, epsabs=1e-14)[0]
        got = 1.0 / O.g0_inverse(g, 0, n)
        assert abs(got - (re + 1j * im)) < 1e-10


def test_bethe_first_iteration_sigma_is_ipt_second_order():
    """At the first iteration Sigma = U^2 int e^{i nu tau} G0(tau)^3 d tau at half
    filling (Sec. II.B), with G0(tau) from the semicircular DOS, integrated
    independently with scipy quadrature."""
    p = BETHE_SMALL
    g = O.make_grid(p)
    Dh = p.hop
    rho = lambda e: 2.0 / (np.pi * Dh**2) * np.sqrt(max(Dh * Dh - e * e, 0.0))  # noqa: E731

    def g0tau(t):
        return -integrate.quad(lambda e: rho(e) * np.exp(-e * t) * fermi(-e, p.beta), -Dh, Dh, epsabs=1e-13)[0]

    ts = np.linspace(0, p.beta, 801)
    gt = np.array([g0tau(t) for t in ts])
    res = O.iterate(p, O.zero_state(p))
    for n in (0, 2, 7):
        nu = (2 * n + 1) * np.pi / p.beta
        from scipy.interpolate import CubicSpline

        sp = CubicSpline(ts, p.U**2 * gt**3)
        re = integrate.quad(lambda t: np.cos(nu * t) * sp(t), 0, p.beta, limit=400, epsabs=1e-13)[0]
        im = integrate.quad(lambda t: np.sin(nu * t) * sp(t), 0, p.beta, limit=400, epsabs=1e-13)[0]
        got = res.sigma_new[0, n - g.e_lo]
        assert abs(got - (re + 1j * im)) < 2e-7


# --------------------------------------------------------------------------- worked example


def _g0_square(p, kx, ky, n):
    nu = (2 * n + 1) * np.pi / p.beta
    return 1.0 / (1j * nu + p.mu + 2 * p.hop * (np.cos(kx) + np.cos(ky)))


@pytest.mark.parametrize("p", [SMALL, SMALL_ODD])
def test_first_iteration_closed_form(p):
    """Sec. II.A worked example: with Lambda = F = Gamma = (U, -U, 2U, 0), the BSE
    gives Phi_d = Phi_m = U^2 (T/N) sum G G(k''+q), Psi_s = -2 U^2 (T/N) sum G G(q-k''),
    Psi_t = 0, constant in k and k'.  The bubbles are summed over the box here
    with the test's own G0."""
    res = O.iterate(p, O.zero_state(p))
    L, T, N = p.L, 1.0 / p.beta, p.L * p.L
    n_lo, m_lo = -p.n_nu // 2, -(p.n_Omega // 2)
    for iq in range(N):
        qx, qy = divmod(iq, L)
        for im in range(p.n_Omega):
            m = m_lo + im
            ph = pp = 0.0
            for ik in range(N):
                kx, ky = divmod(ik, L)
                for n in range(n_lo, n_lo + p.n_nu):
                    k = (2 * np.pi * kx / L, 2 * np.pi * ky / L)
                    kq = (2 * np.pi * (kx + qx) / L, 2 * np.pi * (ky + qy) / L)
                    qk = (2 * np.pi * (qx - kx) / L, 2 * np.pi * (qy - ky) / L)
                    gk = _g0_square(p, *k, n)
                    ph += gk * _g0_square(p, *kq, n + m)
                    pp += gk * _g0_square(p, *qk, m - n - 1)
            Q = iq * p.n_Omega + im
            want = [p.U**2 * T / N * ph, p.U**2 * T / N * ph, -2 * p.U**2 * T / N * pp, 0.0]
            for r in range(4):
                blk = res.phi_new[r, Q]
                assert np.abs(blk - want[r]).max() < 1e-13 * max(1.0, abs(want[0]))


def test_second_iteration_kernels_are_the_first_iterate():
    """From a state constant in k, k' (the first iterate), K1 = Phi and K2 = 0:
    the kernel fill reproduces the constant vertex (Sec. II.A)."""
    p = SMALL
    res = O.iterate(p, O.zero_state(p))
    g = O.make_grid(p)
    K1, K2r, K2c = O.extract_kernels(g, res.state.phi)
    assert np.abs(K1 - res.state.phi[:, :, 0, 0]).max() < 1e-15
    assert np.abs(K2r).max() < 1e-15 and np.abs(K2c).max() < 1e-15


def test_kernel_reconstruction_of_separable_vertex():
    """Brute force: for Phi = a(Q) + b(Q,k) + c(Q,k') the level-2 kernel
    K1 + K2row(k) + K2col(k') reproduces Phi on the whole box; a swapped row and
    column or a missing K1 subtraction breaks it."""
    p = SMALL_ODD
    g = O.make_grid(p)
    rng = np.random.default_rng(3)
    a = rng.standard_normal((4, p.n_Q)) + 1j * rng.standard_normal((4, p.n_Q))
    b = rng.standard_normal((4, p.n_Q, p.n)) + 1j * rng.standard_normal((4, p.n_Q, p.n))
    c = rng.standard_normal((4, p.n_Q, p.n)) + 1j * rng.standard_normal((4, p.n_Q, p.n))
    phi = a[:, :, None, None] + b[:, :, :, None] + c[:, :, None, :]
    K = O.extract_kernels(g, phi)
    kk, kn, qk, qm = O.box_indices(g)
    for x in range(4):
        v = O.kernel_value(
            g, K, x, (kk[None, :, None], kn[None, :, None]), (kk[None, None, :], kn[None, None, :]),
            (qk[:, None, None], qm[:, None, None]))
        assert np.abs(v - phi[x]).max() < 1e-13


def test_kernel_ablations_lower_edge_and_first_level():
    """The ablations of Sec. II.A.  (i) A separable Phi = a(Q) + b(Q,k) + c(Q,k') is
    rebuilt exactly by the lower-edge rule too.  (ii) A Phi living only on the upper
    frequency edge of the column leg (n' = n_hi, rows n > n_lo) has zero kernels under the
    lower-edge rule (it never looks at that edge) and K2row = 1/2 of it under the two-edge
    rule (the mean of the edges).  (iii) The first level keeps K1 and sets K2 = 0."""
    base = SMALL_ODD
    rng = np.random.default_rng(5)
    a = rng.standard_normal((4, base.n_Q)) + 1j * rng.standard_normal((4, base.n_Q))
    b = rng.standard_normal((4, base.n_Q, base.n)) + 1j * rng.standard_normal((4, base.n_Q, base.n))
    c = rng.standard_normal((4, base.n_Q, base.n)) + 1j * rng.standard_normal((4, base.n_Q, base.n))
    phi = a[:, :, None, None] + b[:, :, :, None] + c[:, :, None, :]
    p = base.with_(edge_rule="lower")
    g = O.make_grid(p)
    K = O.extract_kernels(g, phi)
    kk, kn, qk, qm = O.box_indices(g)
    for x in range(4):
        v = O.kernel_value(
            g, K, x, (kk[None, :, None], kn[None, :, None]), (kk[None, None, :], kn[None, None, :]),
            (qk[:, None, None], qm[:, None, None]))
        assert np.abs(v - phi[x]).max() < 1e-13
    # (ii) upper column edge only
    nn = p.n_nu
    f = np.arange(p.n) % nn
    edge = np.zeros((4, p.n_Q, p.n, p.n), dtype=np.complex128)
    edge[:, :, f > 0, :] = 1.0
    edge[:, :, :, f != nn - 1] = 0.0
    K1, K2r, K2c = O.extract_kernels(g, edge)
    assert np.abs(K1).max() == 0 and np.abs(K2r).max() == 0 and np.abs(K2c).max() == 0
    K1b, K2rb, K2cb = O.extract_kernels(O.make_grid(base), edge)
    # two-edge rule: corners (n_hi, n_hi) of 4 -> K1 = 1/4; rows n > n_lo see one of two edges
    assert np.allclose(K1b, 0.25)
    assert np.allclose(K2rb[:, :, f > 0], 0.5 - 0.25) and np.allclose(K2rb[:, :, f == 0], -0.25)
    # (iii) first level
    K1f, K2rf, K2cf = O.extract_kernels(O.make_grid(base.with_(kernel_level=1)), phi)
    K1s, _, _ = O.extract_kernels(O.make_grid(base), phi)
    assert np.array_equal(K1f, K1s) and not K2rf.any() and not K2cf.any()


def test_truncated_sde_approaches_second_order_as_the_box_grows():
    """The truncated Schwinger-Dyson sum (Eq. PA_Sigma on the box, vertex cut off) at the
    first iteration, where F = Lambda^0, is the second-order self-energy restricted to the
    box; as the box grows it must approach Sigma~1 (pinned by its closed forms), with the
    truncation error falling like the GGG tail, about 1/Nnu^2.  A wrong prefactor or sign
    converges to a multiple of Sigma~1 instead."""
    devs = []
    for nu in (8, 16, 32):
        p = Params("bethe", beta=2.0, U=1.0, mu=0.0, L=1, n_nu=nu, n_Omega=nu - 1, sde="truncated")
        g = O.make_grid(p)
        res = O.iterate(p, O.zero_state(p))
        s1 = O.sigma1_second_order(g, np.zeros((1, p.n_ext), np.complex128))
        kk, kn, qk, qm = O.box_indices(g)
        lo = kn[(kn >= -2) & (kn <= 1)] - g.e_lo
        devs.append(np.abs(res.sigma_new[0, lo] - s1[0, lo]).max() / np.abs(s1[0, lo]).max())
        outside = np.ones(p.n_ext, bool)
        outside[kn - g.e_lo] = False
        assert not res.sigma_new[0, outside].any()  # zero where the truncated vertex vanishes
    assert devs[0] / devs[1] > 3 and devs[1] / devs[2] > 3, devs
    assert devs[2] < 2e-3, devs


def test_first_level_equals_second_level_until_stripes_appear():
    """From Phi = 0 the first iterate is constant in (k, k') (Sec. II.A), so its K2 vanishes
    and the first- and second-level fills agree exactly for two iterations; the stripes of
    the second iterate make them differ from the third on."""
    a, b = O.zero_state(SMALL), O.zero_state(SMALL)
    p1 = SMALL.with_(kernel_level=1)
    for _ in range(2):
        a, b = O.iterate(SMALL, a).state, O.iterate(p1, b).state
    assert np.array_equal(a.sigma, b.sigma) and np.array_equal(a.phi, b.phi)
    assert np.abs(O.iterate(SMALL, a).sigma_new - O.iterate(p1, b).sigma_new).max() > 1e-4


def test_truncated_sde_keeps_particle_hole_symmetry():
    """The truncated sum on a box symmetric under nu -> -nu keeps Re Sigma = 0 for the
    half-filled Bethe lattice (odd NOmega: symmetric bosonic box)."""
    p = BETHE_SMALL.with_(sde="truncated")
    st = O.zero_state(p)
    for _ in range(3):
        st = O.iterate(p, st).state
    assert np.abs(st.sigma.real).max() <= 1e-13 * np.abs(st.sigma).max()


# --------------------------------------------------------------------------- identities of the exact equations


def _iterated(p, its):
    st = O.zero_state(p)
    for _ in range(its):
        res = O.iterate(p, st)
        st = res.state
    return res


@pytest.mark.parametrize("p", [SMALL, SMALL_ODD])
def test_crossing_symmetry_of_F(p):
    """App. A, "Crossing symmetry": F_d(q) = F_s/2 + 3F_t/2 and F_m = -F_s/2 + F_t/2 at
    k+k'+q; F_s(q) = F_d/2 - 3F_m/2 and F_t = F_d/2 + F_m/2 at q-k-k'.  The
    partner transfers are computed here, independently of the oracle's maps."""
    res = _iterated(p, 3)
    g = O.make_grid(p)
    F = res.F
    kk, kn, qk, qm = O.box_indices(g)
    L = p.L
    checked = 0
    for Q in range(p.n_Q):
        for k in range(p.n):
            for kp in range(p.n):
                kx, ky = divmod(kk[k], L)
                px, py = divmod(kk[kp], L)
                qx, qy = divmod(qk[Q], L)
                m1 = kn[k] + kn[kp] + qm[Q] + 1
                if g.m_lo <= m1 <= g.m_hi:
                    Q1 = (((kx + px + qx) % L) * L + (ky + py + qy) % L) * p.n_Omega + m1 - g.m_lo
                    assert abs(F[0, Q, k, kp] - 0.5 * F[2, Q1, k, kp] - 1.5 * F[3, Q1, k, kp]) < 1e-13
                    assert abs(F[1, Q, k, kp] + 0.5 * F[2, Q1, k, kp] - 0.5 * F[3, Q1, k, kp]) < 1e-13
                    checked += 1
                m2 = qm[Q] - kn[k] - kn[kp] - 1
                if g.m_lo <= m2 <= g.m_hi:
                    Q2 = (((qx - kx - px) % L) * L + (qy - ky - py) % L) * p.n_Omega + m2 - g.m_lo
                    assert abs(F[2, Q, k, kp] - 0.5 * F[0, Q2, k, kp] + 1.5 * F[1, Q2, k, kp]) < 1e-13
                    assert abs(F[3, Q, k, kp] - 0.5 * F[0, Q2, k, kp] - 0.5 * F[1, Q2, k, kp]) < 1e-13
    assert checked > p.n_Q * p.n  # a substantial part of the box has its partner in the box


def test_crossing_symmetry_of_aux_vertex():
    """F~ obeys the same crossing relations at all arguments, inside and outside
    the box (Sec. II.B builds F~ from the parquet equations with kernels)."""
    p = SMALL
    res = _iterated(p, 3)
    g = O.make_grid(p)
    K = O.extract_kernels(g, res.state.phi)
    rng = np.random.default_rng(5)
    k, kp, q = (rng.integers(0, g.nk, 400) for _ in range(3))
    n, np_ = rng.integers(-12, 12, 400), rng.integers(-12, 12, 400)
    m = rng.integers(-5, 5, 400)
    l0 = O.lambda0(p.U)
    Ft = [O.aux_vertex_minus_lambda0(g, K, r, k, n, kp, np_, q, m) + l0[r] for r in range(4)]
    q1 = g.kadd(g.kadd(k, kp), q)
    m1 = n + np_ + m + 1
    Ft1 = [O.aux_vertex_minus_lambda0(g, K, r, k, n, kp, np_, q1, m1) + l0[r] for r in range(4)]
    assert np.abs(Ft[0] - 0.5 * Ft1[2] - 1.5 * Ft1[3]).max() < 1e-13
    assert np.abs(Ft[1] + 0.5 * Ft1[2] - 0.5 * Ft1[3]).max() < 1e-13


@pytest.mark.parametrize("p", [SMALL, SMALL_ODD])
def test_pauli_principle_at_zero_transfer_frequency(p):
    """App. A, crossing relations: Psi_t^{k,k'}(q) = -Psi_t^{k,q-k'}(q), so F_t is odd
    and F_s even under k' -> q - k'.  At w = 0 the box maps onto itself, so it
    holds to rounding at every iteration."""
    res = _iterated(p, 3)
    g = O.make_grid(p)
    kk, kn, qk, qm = O.box_indices(g)
    for Q in np.where(qm == 0)[0]:
        kp2 = g.ksub(qk[Q], kk) * p.n_nu + (qm[Q] - kn - 1) - g.n_lo
        for r, sgn in ((3, -1.0), (2, 1.0)):
            assert np.abs(res.F[r, Q] - sgn * res.F[r, Q][:, kp2]).max() < 1e-13
            assert np.abs(res.phi_new[r, Q] - sgn * res.phi_new[r, Q][:, kp2]).max() < 1e-13


def test_particle_hole_symmetry_square_lattice():
    """At half filling on the square lattice Sigma(k + (pi,pi), i nu) = -Sigma(k, i nu)*."""
    p = SMALL
    res = _iterated(p, 3)
    L = p.L
    sh = [((ik // L + L // 2) % L) * L + (ik % L + L // 2) % L for ik in range(L * L)]
    s = res.state.sigma
    assert np.abs(s[sh] + s.conj()).max() < 1e-14 * np.abs(s).max() + 1e-16


def test_particle_hole_symmetry_bethe():
    """At half filling of the symmetric Bethe DOS, Sigma(i nu) is purely imaginary and odd."""
    res = _iterated(BETHE_SMALL, 4)
    s = res.state.sigma[0]
    assert np.abs(s.real).max() < 1e-14
    assert np.abs(s + s[::-1]).max() < 1e-14


# --------------------------------------------------------------------------- converged solution


@pytest.fixture(scope="module")
def bethe_converged():
    res, its = O.solve(BETHE_SMALL, 200, 1e-10)
    assert its < 200
    return res


def test_bse_fixed_point_by_direct_inversion(bethe_converged):
    """At the fixed point F = Gamma + Phi with Phi = s Gamma X F, so
    F_r = [1 - s_r Gamma_r diag(X_r)]^-1 Gamma_r (App. A, Eqs. PA_F_G and PA_F_Phi);
    checked by a dense LU solve per (r, Q)."""
    res = bethe_converged
    for r in range(4):
        X = res.X_ph if r < 2 else res.X_pp
        for Q in range(res.F.shape[1]):
            A = np.eye(res.F.shape[2]) - O.BSE_SIGN[r] * res.gamma[r, Q] * X[Q][None, :]
            F = np.linalg.solve(A, res.gamma[r, Q])
            assert np.abs(F - res.F[r, Q]).max() < 1e-7 * np.abs(res.F[r, Q]).max()


def test_high_frequency_tail(bethe_converged):
    """The regulated self-energy keeps the tail nu Im Sigma(i nu) -> -U^2 n(1-n) = -U^2/4
    at half filling (Sec. III.A); the plain box-truncated Eq. PA_Sigma misses it."""
    p = BETHE_SMALL
    g = O.make_grid(p)
    s = bethe_converged.state.sigma[0]
    n = np.arange(g.e_lo, g.e_hi + 1)
    tail = g.nu(n) * s.imag
    assert abs(tail[-1] + p.U**2 / 4) < 0.01 * p.U**2 / 4
    assert abs(tail[0] + p.U**2 / 4) < 0.01 * p.U**2 / 4


def test_regulated_sigma_decomposes_the_plain_sum():
    """With a kernel-term box equal to the vertex box, Sigma~2 + Sigma_dF equals the
    plain Eq. PA_Sigma summed on the box minus its Lambda^0 part (Sec. II.B splits
    Sigma into Sigma~ and a dF remainder); the plain sum is brute force here."""
    p = SMALL_ODD.with_(sigma2_factor=1)
    res0 = _iterated(p, 2)
    st = res0.state
    g = O.make_grid(p)
    G = O.Propagator(g, st.sigma)
    K = O.extract_kernels(g, st.phi)
    gam, F = O.assemble(g, st.phi, K, O.lambda0(p.U))
    s2 = O.sigma2_kernel_terms(g, G, K)
    s3 = O.sigma_delta_F(g, G, F, K, O.lambda0(p.U))
    l0 = O.lambda0(p.U)
    N, T = g.nk, g.T
    kk, kn, qk, qm = O.box_indices(g)
    for k in range(0, p.n, 5):
        tot = 0.0
        for Q in range(p.n_Q):
            for kp in range(p.n):
                ph = (G(g.kadd(kk[k], qk[Q]), kn[k] + qm[Q]) * G(g.kadd(kk[kp], qk[Q]), kn[kp] + qm[Q])
                      * G(kk[kp], kn[kp]))
                pp = (G(g.ksub(qk[Q], kk[kp]), qm[Q] - kn[kp] - 1) * G(g.ksub(qk[Q], kk[k]), qm[Q] - kn[k] - 1)
                      * G(kk[kp], kn[kp]))
                fph = (F[0, Q, k, kp] - l0[0]) - (F[1, Q, k, kp] - l0[1])
                fpp = (F[2, Q, k, kp] - l0[2]) + (F[3, Q, k, kp] - l0[3])
                tot += ph * fph + pp * fpp
        want = -(p.U / 4) * (T / N) ** 2 * tot
        e = kn[k] - g.e_lo
        assert abs(s2[kk[k], e] + s3[kk[k], e] - want) < 1e-13 * max(1.0, abs(want))


def test_dF_vanishes_where_every_lookup_is_a_fill():
    """F~ matches F at and beyond the box boundary (Sec. II.B): where every crossed
    lookup leaves the box, F - F~ reduces to the own-channel Phi - Phi~ (and
    Lambda - Lambda^0 = 0 in the parquet approximation)."""
    p = SMALL
    res = _iterated(p, 3)
    g = O.make_grid(p)
    st_prev = _iterated(p, 2).state
    K = O.extract_kernels(g, st_prev.phi)
    kk, kn, qk, qm = O.box_indices(g)
    found = 0
    for Q in range(p.n_Q):
        for k in range(p.n):
            for kp in range(p.n):
                n, np_, m = kn[k], kn[kp], qm[Q]
                outA = not (g.m_lo <= np_ - n <= g.m_hi and g.n_lo <= n + m <= g.n_hi)
                outB = not (g.m_lo <= n + np_ + m + 1 <= g.m_hi)
                if outA and outB:
                    for r in (0, 1):
                        ft = O.aux_vertex_minus_lambda0(g, K, r, kk[k], n, kk[kp], np_, qk[Q], m) + O.lambda0(p.U)[r]
                        own_dev = st_prev.phi[r, Q, k, kp] - O.kernel_value(
                            g, K, r, (kk[k], n), (kk[kp], np_), (qk[Q], m))
                        assert abs(res.F[r, Q, k, kp] - ft - own_dev) < 1e-13
                    found += 1
    assert found > 0


def _vertex_correction(p):
    res = _iterated(p, 3)
    g = O.make_grid(p)
    G = O.Propagator(g, res.state.sigma)
    K = O.extract_kernels(g, res.state.phi)
    gam, F = O.assemble(g, res.state.phi, K, O.lambda0(p.U))
    return O.sigma2_kernel_terms(g, G, K) + O.sigma_delta_F(g, G, F, K, O.lambda0(p.U))


@pytest.mark.parametrize("p", [
    Params("bethe", beta=5.0, U=1.0, mu=0.0, L=1, n_nu=8, n_Omega=7, mix=1.0),
    Params("square", beta=2.5, U=1.0, mu=0.4, L=2, n_nu=6, n_Omega=5, mix=1.0),
])
def test_vertex_changes_by_one_order_per_iteration(p):
    """Undamped iteration from Phi = 0 (Sec. II, the perturbative start): the first iterate has
    F = Lambda0 (order U), the second adds the s U X U Phi's (exactly order U^2), the third the
    next order (U^3).  So (F2 - F1) / U^2 is the same at every U and (F3 - F2) / U^3 tends to a
    constant as U -> 0; a term entering at the wrong order breaks one of the two."""
    r2, r3 = [], []
    for U in (0.2, 0.1, 0.05):
        q = p.with_(U=U)
        st, F = O.zero_state(q), []
        for _ in range(3):
            res = O.iterate(q, st)
            st = res.state
            F.append(res.F)
        r2.append(np.abs(F[1] - F[0]).max() / U**2)
        r3.append(np.abs(F[2] - F[1]).max() / U**3)
    assert max(r2) / min(r2) < 1 + 1e-9
    assert max(r3) / min(r3) < 1.02


def test_third_order_cancels_in_the_symmetric_impurity_problem():
    """Sigma - Sigma^(2)[G] comes from the order-U^2 Phi's in F.  In the
    particle-hole symmetric single-site problem the third-order self-energy
    vanishes (the ph and pp contributions cancel), so the correction scales as
    U^4; a wrong sign or factor in any channel term leaves a U^3 part."""
    r = [np.abs(_vertex_correction(BETHE_SMALL.with_(U=U))).max() / U**4 for U in (0.2, 0.1, 0.05)]
    assert max(r) < 1.03 * min(r)


def test_third_order_survives_away_from_half_filling():
    """Away from half filling (square lattice, mu = 0.4) the same correction is of order U^3."""
    base = Params("square", beta=2.5, U=1.0, mu=0.4, L=2, n_nu=6, n_Omega=5)
    r = [np.abs(_vertex_correction(base.with_(U=U))).max() / U**3 for U in (0.2, 0.1, 0.05)]
    assert max(r) < 1.03 * min(r)


def test_susceptibility_first_order_rpa():
    """With the first-iteration vertex F = Lambda = (U, -U, 2U, 0), chi_m = chi0 + U chi0^2 and
    chi_d = chi0 - U chi0^2: the first-order terms of the RPA forms chi0/(1 -+ U chi0),
    with chi0 = -(T/N) sum_k G0(k) G0(k+q) summed here with the test's own G0; in the
    particle-particle channels, with chi0pp = -(T/N) sum_k G0(k) G0(q-k),
    chi_s = chi0pp - 2U chi0pp^2 and chi_t = chi0pp (F_t = 0)."""
    p = SMALL_ODD
    res = O.iterate(p, O.zero_state(p))
    chi = O.susceptibility(res.F, res.X_ph, res.X_pp)
    L, T, N = p.L, 1.0 / p.beta, p.L * p.L
    n_lo, m_lo = -p.n_nu // 2, -(p.n_Omega // 2)
    for iq in range(N):
        qx, qy = divmod(iq, L)
        for im in range(p.n_Omega):
            m = m_lo + im
            b = bpp = 0.0
            for ik in range(N):
                kx, ky = divmod(ik, L)
                for n in range(n_lo, n_lo + p.n_nu):
                    gk = _g0_square(p, 2 * np.pi * kx / L, 2 * np.pi * ky / L, n)
                    b += gk * _g0_square(p, 2 * np.pi * (kx + qx) / L, 2 * np.pi * (ky + qy) / L, n + m)
                    # q - k: bosonic m minus fermionic n is the fermionic index m - n - 1
                    bpp += gk * _g0_square(p, 2 * np.pi * (qx - kx) / L, 2 * np.pi * (qy - ky) / L, m - n - 1)
            chi0, chi0pp = -T / N * b, -T / N * bpp
            Q = iq * p.n_Omega + im
            assert abs(chi[1, Q] - (chi0 + p.U * chi0**2)) < 1e-13
            assert abs(chi[0, Q] - (chi0 - p.U * chi0**2)) < 1e-13
            assert abs(chi[2, Q] - (chi0pp - 2 * p.U * chi0pp**2)) < 1e-13
            assert abs(chi[3, Q] - chi0pp) < 1e-13


# --------------------------------------------------------------------------- tabulated Lambda


def _lambda_tables(p, nl, seed):
    """Seeded local tables of all four channels on |m| <= nl, n, n' in [-nl, nl - 1]."""
    rng = np.random.default_rng(seed)
    return {r: (0.3 * p.U * (rng.standard_normal((2 * nl + 1, 2 * nl, 2 * nl))
                             + 1j * rng.standard_normal((2 * nl + 1, 2 * nl, 2 * nl))), nl)
            for r in range(4)}


def test_lambda_table_of_constants_equals_scalar_lambda():
    """A table holding one constant per channel over the whole box is the scalar Lambda:
    two iterations with the table and with the scalar agree to rounding."""
    p = SMALL_ODD
    c = np.array([1.3 + 0.2j, -0.7, 2.1 - 0.1j, 0.4j])
    nl = max(p.n_nu, p.n_Omega)
    tabs = {r: (np.full((2 * nl + 1, 2 * nl, 2 * nl), c[r]), nl) for r in range(4)}
    lam_t = O.lambda_tabulated(p, tabs)
    a = b = O.zero_state(p)
    for _ in range(2):
        ra, rb = O.iterate(p, a, lam=lam_t), O.iterate(p, b, lam=c)
        a, b = ra.state, rb.state
    assert np.abs(a.phi - b.phi).max() <= 1e-13 * np.abs(b.phi).max()
    assert np.abs(a.sigma - b.sigma).max() <= 1e-13 * np.abs(b.sigma).max()


def test_lambda_table_first_iteration_closed_form():
    """From Phi = 0 the kernels vanish, so Gamma_r = F_r = Lambda_r and the first iterate is
    Phi_r(Q) = alpha s_r Lambda_r(Q) diag(X_r(Q)) Lambda_r(Q) (Eq. PA_F_Phi).  Lambda is
    rebuilt here element by element from the table (inside |m| <= nl, |n|, |n'| in range;
    (U, -U, 2U, 0) outside), with a table smaller than the box so both cases occur."""
    p = Params("square", beta=2.0, U=1.1, mu=0.0, L=2, n_nu=6, n_Omega=5)
    nl = 2
    tabs = _lambda_tables(p, nl, seed=7)
    res = O.iterate(p, O.zero_state(p), lam=O.lambda_tabulated(p, tabs))
    l0 = [p.U, -p.U, 2 * p.U, 0.0]
    s_r = [1.0, 1.0, -0.5, 0.5]
    n_lo, m_lo = -p.n_nu // 2, -(p.n_Omega // 2)
    for r in range(4):
        lam = np.empty((p.n_Q, p.n, p.n), dtype=np.complex128)
        for Q in range(p.n_Q):
            m = m_lo + Q % p.n_Omega
            for k in range(p.n):
                n = n_lo + k % p.n_nu
                for kp in range(p.n):
                    npr = n_lo + kp % p.n_nu
                    if abs(m) <= nl and -nl <= n < nl and -nl <= npr < nl:
                        lam[Q, k, kp] = tabs[r][0][m + nl, n + nl, npr + nl]
                    else:
                        lam[Q, k, kp] = l0[r]
        X = res.X_ph if r < 2 else res.X_pp
        expect = p.mix * s_r[r] * np.einsum("qab,qb,qbc->qac", lam, X, lam)
        assert np.abs(res.state.phi[r] - expect).max() <= 1e-12 * np.abs(expect).max(), r
        assert np.abs(res.F[r] - lam).max() <= 1e-14 * np.abs(lam).max(), r
