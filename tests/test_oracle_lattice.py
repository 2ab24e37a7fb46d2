"""Pins of the oracle's momentum arithmetic on lattices where k + q and k - q differ.

On a 2x2 lattice every momentum is its own negative, so a sign slip in a momentum
argument (k + q for k - q, q - k' for k' - q) cannot change any result there.  The pins
below run on 3x3 and 4x4 lattices.  Most of them also thread a uniform vector potential
A through the torus: the Peierls phase turns the dispersion into
eps_k = -2t [cos(kx + Ax) + cos(ky + Ay)], which is not even in k, so G(k) != G(-k) and
even the sums over a full Brillouin zone see every momentum sign.  Each relation checked
here holds for any dispersion: the second-order diagram (Sec. II.B), the worked first
iteration (Sec. II.A), crossing symmetry and the Pauli principle of the full vertex
(App. A), the split of the regulated self-energy (Sec. II.B, Eq. PA_Sigma), and the
first-order susceptibility.  Particle-hole symmetry is checked with the plain
dispersion on the 4x4 lattice, which holds the nesting vector (pi, pi).

The tests compute every momentum themselves from the coordinates (ix, iy) of the index
ik = ix * L + iy; they take from the oracle only the quantities under test.
"""
import numpy as np
import pytest

from oracle import parquet_oracle as O
from paper_1510_03330_gb300.workloads import Params

A_FLUX = (0.37, 0.91)
P3 = Params("square", beta=2.5, U=1.3, mu=0.1, L=3, n_nu=4, n_Omega=5)
P3_EVEN = Params("square", beta=2.0, U=1.1, mu=-0.2, L=3, n_nu=4, n_Omega=4, hop=0.8)


def flux_eps(p, ix, iy):
    kx, ky = 2 * np.pi * np.asarray(ix) / p.L, 2 * np.pi * np.asarray(iy) / p.L
    return -2.0 * p.hop * (np.cos(kx + A_FLUX[0]) + np.cos(ky + A_FLUX[1]))


@pytest.fixture
def flux(monkeypatch):
    """The oracle's square lattice with the vector potential A_FLUX in its hopping."""
    orig = O.make_grid

    def make(p):
        g = orig(p)
        if p.lattice == "square":  # the Peierls phase added to the oracle's own momentum labels
            g.eps = -2.0 * p.hop * (np.cos(g.kx + A_FLUX[0]) + np.cos(g.ky + A_FLUX[1]))
        return g

    monkeypatch.setattr(O, "make_grid", make)


def fermi(e, beta):
    return 0.5 * (1.0 - np.tanh(0.5 * beta * e))


def coords(p, ik):
    return divmod(int(ik), p.L)


def idx(p, x, y):
    return (x % p.L) * p.L + (y % p.L)


def g0(p, ix, iy, n):
    nu = (2 * n + 1) * np.pi / p.beta
    return 1.0 / (1j * nu + p.mu - flux_eps(p, ix, iy))


def iterated(p, its):
    st = O.zero_state(p)
    for _ in range(its):
        res = O.iterate(p, st)
        st = res.state
    return res


def test_flux_dispersion_breaks_inversion():
    """Precondition of every flux pin: eps_k != eps_-k somewhere on the 3x3 lattice."""
    p = P3
    e = np.array([[flux_eps(p, x, y) for y in range(3)] for x in range(3)])
    e_neg = np.array([[flux_eps(p, -x, -y) for y in range(3)] for x in range(3)])
    assert np.abs(e - e_neg).max() > 0.5


@pytest.mark.parametrize("L,mu", [(3, 0.15), (4, -0.3)])
def test_second_order_closed_form_with_flux(flux, L, mu):
    """Sigma~1 (the second-order diagram, Sec. II.B) of the free propagators equals
    (U^2/N^2) sum_{a,b} [(1-f_a)(1-f_b) f_c + f_a f_b (1-f_c)] / (i nu - e_a - e_b + e_c)
    with c = a + b - k: a sign slip in the real-space transform (G(-r, beta - tau)) or in
    one of its phases exchanges k and -k, which the flux makes visible."""
    p = Params("square", beta=2.0, U=1.1, mu=mu, L=L, n_nu=4, n_Omega=5, hop=0.6)
    g = O.make_grid(p)
    s1 = O.sigma1_second_order(g, np.zeros((L * L, p.n_ext), complex))
    N = L * L
    e = np.array([flux_eps(p, *coords(p, i)) for i in range(N)]) - mu
    f = fermi(e, p.beta)
    n = np.arange(p.n_ext) - (p.n_Omega // 2) - p.n_nu // 2
    nu = (2 * n + 1) * np.pi / p.beta
    for ik in range(N):
        kx, ky = coords(p, ik)
        ref = np.zeros_like(nu, dtype=complex)
        for ia in range(N):
            ax, ay = coords(p, ia)
            for ib in range(N):
                bx, by = coords(p, ib)
                ic = idx(p, ax + bx - kx, ay + by - ky)
                num = (1 - f[ia]) * (1 - f[ib]) * f[ic] + f[ia] * f[ib] * (1 - f[ic])
                ref += num / (1j * nu - e[ia] - e[ib] + e[ic])
        ref *= p.U**2 / N**2
        assert np.abs(s1[ik] - ref).max() < 1e-11 * np.abs(ref).max(), ik


@pytest.mark.parametrize("p", [P3, P3_EVEN])
def test_first_iteration_closed_form_with_flux(flux, p):
    """Worked first iteration of Sec. II.A on the 3x3 lattice: Phi_d = Phi_m =
    U^2 (T/N) sum G0(k'') G0(k''+q), Phi_s = -2 U^2 (T/N) sum G0(k'') G0(q-k''), Phi_t = 0,
    the bubbles summed here with the test's own G0 and momentum arithmetic.  With the flux
    sum G0(k'')G0(k''+q) != sum G0(k'')G0(k''-q), so the bubbles' momentum signs are pinned."""
    res = O.iterate(p, O.zero_state(p))
    T, N = 1.0 / p.beta, p.L * p.L
    n_lo, m_lo = -p.n_nu // 2, -(p.n_Omega // 2)
    sep = 0.0
    for iq in range(N):
        qx, qy = coords(p, iq)
        for im in range(p.n_Omega):
            m = m_lo + im
            ph = pp = ph_wrong = 0.0
            for ik in range(N):
                kx, ky = coords(p, ik)
                for n in range(n_lo, n_lo + p.n_nu):
                    gk = g0(p, kx, ky, n)
                    ph += gk * g0(p, kx + qx, ky + qy, n + m)
                    ph_wrong += gk * g0(p, kx - qx, ky - qy, n + m)
                    pp += gk * g0(p, qx - kx, qy - ky, m - n - 1)
            sep = max(sep, abs(ph - ph_wrong))
            Q = iq * p.n_Omega + im
            want = [p.U**2 * T / N * ph, p.U**2 * T / N * ph, -2 * p.U**2 * T / N * pp, 0.0]
            for r in range(4):
                assert np.abs(res.phi_new[r, Q] - want[r]).max() < 1e-13 * max(1.0, abs(want[0])), (Q, r)
    assert sep > 1e-3  # the pin separates k + q from k - q


def _crossing_partners(p, g, k, kp, Q):
    """Transfers k + k' + q and q - k - k' (frequencies and momenta), computed here."""
    kk, kn, qk, qm = O.box_indices(g)
    kx, ky = coords(p, kk[k])
    px, py = coords(p, kk[kp])
    qx, qy = coords(p, qk[Q])
    m1 = kn[k] + kn[kp] + qm[Q] + 1
    m2 = qm[Q] - kn[k] - kn[kp] - 1
    Q1 = idx(p, kx + px + qx, ky + py + qy) * p.n_Omega + m1 - g.m_lo if g.m_lo <= m1 <= g.m_hi else None
    Q2 = idx(p, qx - kx - px, qy - ky - py) * p.n_Omega + m2 - g.m_lo if g.m_lo <= m2 <= g.m_hi else None
    return Q1, Q2


@pytest.mark.parametrize("p", [P3, P3_EVEN])
def test_crossing_symmetry_with_flux(flux, p):
    """App. A, "Crossing symmetry", after three iterations (stripes and fills present):
    F_d(q) = F_s/2 + 3F_t/2 and F_m = -F_s/2 + F_t/2 at k+k'+q; F_s(q) = F_d/2 - 3F_m/2 and
    F_t = F_d/2 + F_m/2 at q-k-k', the partner transfers computed here.  A sign slip in any
    of the four crossed maps of the parquet equations (A-D) breaks one of them."""
    res = iterated(p, 3)
    g = O.make_grid(p)
    F = res.F
    scale = np.abs(F).max()
    checked = 0
    for Q in range(p.n_Q):
        for k in range(p.n):
            for kp in range(p.n):
                Q1, Q2 = _crossing_partners(p, g, k, kp, Q)
                if Q1 is not None:
                    assert abs(F[0, Q, k, kp] - 0.5 * F[2, Q1, k, kp] - 1.5 * F[3, Q1, k, kp]) < 1e-13 * scale
                    assert abs(F[1, Q, k, kp] + 0.5 * F[2, Q1, k, kp] - 0.5 * F[3, Q1, k, kp]) < 1e-13 * scale
                    checked += 1
                if Q2 is not None:
                    assert abs(F[2, Q, k, kp] - 0.5 * F[0, Q2, k, kp] + 1.5 * F[1, Q2, k, kp]) < 1e-13 * scale
                    assert abs(F[3, Q, k, kp] - 0.5 * F[0, Q2, k, kp] - 0.5 * F[1, Q2, k, kp]) < 1e-13 * scale
                    checked += 1
    assert checked > p.n_Q * p.n


@pytest.mark.parametrize("p", [P3, P3_EVEN])
def test_spin_rotation_crossing_with_flux(flux, p):
    """SU(2) symmetry with the exchange of the two outgoing legs (the ph <-> ph-bar crossing,
    transfer q <-> k' - k), after three iterations with the inversion-breaking flux:
      F_d(k, k'; q) = -F_d(k, k+q; k'-k)/2 - 3 F_m(k, k+q; k'-k)/2,
      F_m(k, k'; q) = -F_d(k, k+q; k'-k)/2 +   F_m(k, k+q; k'-k)/2,
    wherever k+q and k'-k are in the box.  It is not one of the printed crossing relations:
    the parquet equations produce it through maps A and C and the d/m coefficients, so a wrong
    leg or transfer there, or a wrong coefficient of Phi_d, Phi_m in Gamma_d, Gamma_m, breaks it.
    The partner arguments are computed here."""
    res = iterated(p, 3)
    g = O.make_grid(p)
    F = res.F
    scale = np.abs(F).max()
    kk, kn, qk, qm = O.box_indices(g)
    where = {(int(kk[i]), int(kn[i])): i for i in range(p.n)}
    checked = 0
    for Q in range(p.n_Q):
        qx, qy = coords(p, qk[Q])
        for k in range(p.n):
            kx, ky = coords(p, kk[k])
            kq = where.get((idx(p, kx + qx, ky + qy), int(kn[k] + qm[Q])))
            if kq is None:
                continue
            for kp in range(p.n):
                px, py = coords(p, kk[kp])
                m = int(kn[kp] - kn[k])
                if not g.m_lo <= m <= g.m_hi:
                    continue
                Q2 = idx(p, px - kx, py - ky) * p.n_Omega + m - g.m_lo
                fd, fm = F[0, Q2, k, kq], F[1, Q2, k, kq]
                assert abs(F[0, Q, k, kp] - (-0.5 * fd - 1.5 * fm)) < 1e-13 * scale
                assert abs(F[1, Q, k, kp] - (-0.5 * fd + 0.5 * fm)) < 1e-13 * scale
                checked += 1
    assert checked > p.n_Q * p.n


def test_pauli_principle_with_flux(flux):
    """F_t odd and F_s even under k' -> q - k' at transfer frequency 0 (App. A), with
    q - k' computed here: a slip in the momentum of a crossed leg breaks it."""
    p = P3
    res = iterated(p, 3)
    g = O.make_grid(p)
    kk, kn, qk, qm = O.box_indices(g)
    found = 0
    for Q in np.where(qm == 0)[0]:
        qx, qy = coords(p, qk[Q])
        kp2 = np.array([idx(p, qx - kk[j] // p.L, qy - kk[j] % p.L) * p.n_nu + (-kn[j] - 1) - g.n_lo
                        for j in range(p.n)])
        for r, sgn in ((3, -1.0), (2, 1.0)):
            scale = np.abs(res.F[r, Q]).max()
            assert np.abs(res.F[r, Q] - sgn * res.F[r, Q][:, kp2]).max() < 1e-13 * max(scale, 1.0)
            assert np.abs(res.phi_new[r, Q] - sgn * res.phi_new[r, Q][:, kp2]).max() < 1e-13 * max(scale, 1.0)
        found += 1
    assert found == p.L * p.L


def test_regulated_sigma_decomposes_the_plain_sum_with_flux(flux):
    """With a kernel-term box equal to the vertex box, Sigma~2 + Sigma_dF equals the plain
    Eq. PA_Sigma on the box minus its Lambda^0 part (Sec. II.B), the plain sum written out
    here with its own momenta k + q, k' + q, q - k', q - k: pins the weights of both."""
    p = P3_EVEN.with_(sigma2_factor=1)
    st = iterated(p, 2).state
    g = O.make_grid(p)
    G = O.Propagator(g, st.sigma)
    K = O.extract_kernels(g, st.phi)
    lam = O.lambda0(p.U)
    _, F = O.assemble(g, st.phi, K, lam)
    s2 = O.sigma2_kernel_terms(g, G, K)
    s3 = O.sigma_delta_F(g, G, F, K, lam)
    N, T = g.nk, g.T
    kk, kn, qk, qm = O.box_indices(g)
    for k in range(0, p.n, 3):
        kx, ky = coords(p, kk[k])
        tot = 0.0
        for Q in range(p.n_Q):
            qx, qy = coords(p, qk[Q])
            m = qm[Q]
            for kp in range(p.n):
                px, py = coords(p, kk[kp])
                npr = kn[kp]
                ph = G(idx(p, kx + qx, ky + qy), kn[k] + m) * G(idx(p, px + qx, py + qy), npr + m) * G(kk[kp], npr)
                pp = (G(idx(p, qx - px, qy - py), m - npr - 1) * G(idx(p, qx - kx, qy - ky), m - kn[k] - 1)
                      * G(kk[kp], npr))
                fph = (F[0, Q, k, kp] - lam[0]) - (F[1, Q, k, kp] - lam[1])
                fpp = (F[2, Q, k, kp] - lam[2]) + (F[3, Q, k, kp] - lam[3])
                tot += ph * fph + pp * fpp
        want = -(p.U / 4) * (T / N) ** 2 * tot
        e = kn[k] - g.e_lo
        assert abs(s2[kk[k], e] + s3[kk[k], e] - want) < 1e-13 * max(1.0, abs(want)), k


def test_susceptibility_first_order_with_flux(flux):
    """chi from the first-iteration vertex F = (U, -U, 2U, 0): chi_m = chi0 + U chi0^2,
    chi_d = chi0 - U chi0^2, chi_s = chi0pp - 2U chi0pp^2, chi_t = chi0pp, the bubbles
    chi0 = -(T/N) sum G0(k) G0(k+q), chi0pp = -(T/N) sum G0(k) G0(q-k) summed here."""
    p = P3
    res = O.iterate(p, O.zero_state(p))
    chi = O.susceptibility(res.F, res.X_ph, res.X_pp)
    T, N = 1.0 / p.beta, p.L * p.L
    n_lo, m_lo = -p.n_nu // 2, -(p.n_Omega // 2)
    for iq in range(N):
        qx, qy = coords(p, iq)
        for im in range(p.n_Omega):
            m = m_lo + im
            b = bpp = 0.0
            for ik in range(N):
                kx, ky = coords(p, ik)
                for n in range(n_lo, n_lo + p.n_nu):
                    gk = g0(p, kx, ky, n)
                    b += gk * g0(p, kx + qx, ky + qy, n + m)
                    bpp += gk * g0(p, qx - kx, qy - ky, m - n - 1)
            chi0, chi0pp = -T / N * b, -T / N * bpp
            Q = iq * p.n_Omega + im
            assert abs(chi[1, Q] - (chi0 + p.U * chi0**2)) < 1e-13
            assert abs(chi[0, Q] - (chi0 - p.U * chi0**2)) < 1e-13
            assert abs(chi[2, Q] - (chi0pp - 2 * p.U * chi0pp**2)) < 1e-13
            assert abs(chi[3, Q] - chi0pp) < 1e-13


def test_particle_hole_symmetry_4x4():
    """Half filling on the 4x4 lattice, which holds the nesting vector (pi, pi):
    Sigma(k + (pi, pi), i nu) = -Sigma(k, i nu)* after three iterations (stripes and fills
    present), and the point group of the plain dispersion maps Sigma(k) onto Sigma(-k) and
    Sigma(ky, kx)."""
    p = Params("square", beta=2.0, U=1.4, mu=0.0, L=4, n_nu=4, n_Omega=3)
    s = iterated(p, 3).state.sigma
    L = p.L
    sh = [idx(p, ik // L + 2, ik % L + 2) for ik in range(L * L)]
    neg = [idx(p, -(ik // L), -(ik % L)) for ik in range(L * L)]
    swp = [idx(p, ik % L, ik // L) for ik in range(L * L)]
    scale = np.abs(s).max()
    assert np.abs(s[sh] + s.conj()).max() < 1e-13 * scale
    assert np.abs(s[neg] - s).max() < 1e-13 * scale
    assert np.abs(s[swp] - s).max() < 1e-13 * scale
    # the momentum dependence is real: Sigma differs between k = 0 and k = (pi, pi)
    assert np.abs(s[0] - s[idx(p, 2, 2)]).max() > 1e-3 * scale


# --------------------------------------------------------------------------- density and mu search


@pytest.mark.parametrize("L,mu", [(3, 0.35), (4, -0.8), (4, 0.0)])
def test_density_of_the_free_lattice_is_the_fermi_sum(flux, L, mu):
    """With Sigma = 0 the density is (2/N) sum_k f(eps_k - mu), the flux lattice included:
    checks the closed-form tails (1/2 and -beta c2/4) and the remainder sum."""
    p = Params("square", beta=3.0, U=1.0, mu=mu, L=L, n_nu=4, n_Omega=3, hop=0.9)
    n = O.density(p, np.zeros((L * L, p.n_ext), complex))
    e = np.array([flux_eps(p, *coords(p, i)) for i in range(L * L)])
    ref = 2.0 * np.mean(fermi(e - mu, p.beta))
    assert abs(n - ref) < 1e-9, (n, ref)


def test_density_is_monotone_and_half_filled_at_mu_zero():
    """At half filling of the plain lattice (mu = 0, particle-hole symmetric Sigma after three
    iterations) n = 1; n(mu) increases with mu at fixed Sigma; find_mu inverts it."""
    p = Params("square", beta=2.0, U=1.4, mu=0.0, L=4, n_nu=4, n_Omega=3)
    sig = iterated(p, 3).state.sigma
    assert abs(O.density(p, sig) - 1.0) < 1e-12
    ns = [O.density(p.with_(mu=m), sig) for m in (-1.0, -0.3, 0.2, 0.9)]
    assert all(b > a for a, b in zip(ns, ns[1:])), ns
    for target in (0.8, 1.15):
        mu = O.find_mu(p, sig, target)
        assert abs(O.density(p.with_(mu=mu), sig) - target) < 1e-11


def test_fixed_density_iteration_holds_the_density():
    """An iteration at fixed density (p.density) sets mu on the state's Sigma before the
    Dyson step: the G of that iteration holds the target filling; away from half filling
    the second-order self-energy acquires a real part."""
    p = Params("square", beta=2.5, U=1.2, mu=0.0, L=3, n_nu=4, n_Omega=3, density=0.85)
    st = O.zero_state(p)
    for _ in range(2):
        res = O.iterate(p, st)
        assert abs(O.density(p.with_(mu=res.mu, density=0.0), st.sigma) - 0.85) < 1e-11
        st = res.state
    assert res.mu < 0 and np.abs(st.sigma.real).max() > 1e-4
