"""Plain FP64 CPU oracle of one self-consistent parquet iteration.

TEST INFRASTRUCTURE.  Only the tests, the package smoke check and the
benchmark's CPU-baseline leg may import this module.  It shares no code with
the CUDA solver; both take their inputs from ``workloads``.

It follows Li, Wentzell, Pudleiner, Thunstroem and Held, "Efficient
implementation of the parquet equations -- role of the reducible vertex
function and its kernel approximation" (arXiv:1510.03330), step by step, in
the paper's notation, with numpy as the only library:

  Dyson equation           App. A, "Self-energy from the full vertex", Eq. PA_Dyson
  bubbles G G              App. A, Eq. PA_F_Phi (the G G between Gamma and F)
  kernel functions K1, K2  Sec. II.A, first- and second-level kernel approximation
  parquet equations        Sec. II, Eq. PA_F; App. A, Eqs. PA_Gamma_dm, PA_Gamma_st
  Bethe-Salpeter equation  App. A, Eq. PA_F_Phi
  auxiliary vertex F~      Sec. II.B, Eq. auxiliary_function
  regulated self-energy    Sec. II.B (Sigma = Sigma~1 + Sigma~2 + sum of G G G dF)
  Schwinger-Dyson equation App. A, Eq. PA_Sigma

Readings taken where the paper is silent or garbled (each is also listed in
the design notes):
  * The momentum sums of Eq. PA_Sigma carry one 1/N each: (T/N)^2/4, not T^2/(4N).
  * Channel signs of the BSE: s_d = s_m = +1, s_t = +1/2, s_s = -1/2.
  * K1_r(Q): mean of Phi_r(Q) over the four corners of the frequency box,
    averaged over the momenta of both legs.  K2row_r(k;Q) / K2col_r(k';Q): mean
    over the lower and upper frequency edge of the other leg (momentum
    averaged) minus K1.  Out of the box a superscript contributes no K2 term;
    a transfer outside the bosonic box contributes 0.
  * F~ is the parquet equation evaluated with level-2 kernels only, with
    Lambda^0 = (U, -U, 2U, 0); Lambda - Lambda^0 belongs to dF.
  * Sigma~2 sums k' over sigma2_factor x Nnu fermionic and q over
    sigma2_factor x NOmega bosonic frequencies (all momenta).
  * Sigma beyond its stored range is c1/(i nu) with c1 = -<nu Im Sigma> at the
    two outer stored frequencies (momentum averaged).
  * Jacobi update from the state (Phi, Sigma), linear mixing of both.
  * Ablations of Sec. II.A/B selected by Params: kernel_level 1 keeps K1 only;
    edge_rule "lower" reads K2 at the lower frequency edge alone (K1 at the lower
    corner); sde "truncated" sums Eq. PA_Sigma on the box with the vertex cut off
    there (Sigma = 0 outside the box).

Every function is pinned by the tests (closed forms, limits, invariants, stored
closed-form values); chi in all four channels by its first-order expansion at
the first-iteration vertex; the density by the Fermi-function sum of the free
lattice and particle-hole symmetry.

Array layout: Phi[r, Q, k, k'] with r in (d, m, s, t), Q = iq*NOmega + (m-m_lo),
k = ik*Nnu + (n-n_lo); Sigma[ik, n-e_lo] on the extended range.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

D, M, S, T_ = 0, 1, 2, 3
CH = "dmst"

# BSE channel factors (App. A, Eq. PA_F_Phi): + T/N for d and m, +T/2N for t, -T/2N for s.
BSE_SIGN = np.array([1.0, 1.0, -0.5, 0.5])

# Parquet equations for Gamma_r (App. A, Eqs. PA_Gamma_dm and PA_Gamma_st):
# for each channel, (coefficient, source channel, argument map) of the four
# crossed reducible vertices.  Maps:
#   A: Phi^{k,k+q}(k'-k)   B: Psi^{k,k'}(k+k'+q)   C: Phi^{k,q-k'}(k'-k)   D: Phi^{k,k'}(q-k-k')
PARQUET_TERMS = {
    D: [(-0.5, D, "A"), (-1.5, M, "A"), (0.5, S, "B"), (1.5, T_, "B")],
    M: [(-0.5, D, "A"), (0.5, M, "A"), (-0.5, S, "B"), (0.5, T_, "B")],
    S: [(0.5, D, "C"), (-1.5, M, "C"), (0.5, D, "D"), (-1.5, M, "D")],
    T_: [(-0.5, D, "C"), (-0.5, M, "C"), (0.5, D, "D"), (0.5, M, "D")],
}


def lambda0(U):
    """Parquet approximation of the fully irreducible vertex, (U, -U, 2U, 0) (Sec. II.A)."""
    return np.array([U, -U, 2.0 * U, 0.0], dtype=np.complex128)


def lambda_tabulated(p, tables):
    """Fully irreducible vertex with a tabulated local part, over the whole box.

    Sec. III.A extends the parquet approximation by a Lambda computed on a small
    frequency box and supplemented by its lowest-order value (U, -U, 2U, 0) outside.
    tables maps a channel r (0..3 = d, m, s, t) to (table, n_lambda) with
    table[m + n_lambda][n + n_lambda][n' + n_lambda] = Lambda_r^{nu_n, nu_n'}(omega_m)
    for |m| <= n_lambda and n, n' in [-n_lambda, n_lambda - 1] (local: no momentum
    dependence).  Returns four arrays [Q][k][k'] in the channel conventions of F_r.
    """
    g = make_grid(p)
    kk, kn, qk, qm = box_indices(g)
    l0 = lambda0(p.U)
    m, n, npr = qm[:, None, None], kn[None, :, None], kn[None, None, :]
    out = []
    for r in range(4):
        arr = np.full((p.n_Q, p.n, p.n), l0[r], dtype=np.complex128)
        if r in tables:
            tab, nl = tables[r]
            tab = np.asarray(tab, dtype=np.complex128)
            assert tab.shape == (2 * nl + 1, 2 * nl, 2 * nl)
            inside = (np.abs(m) <= nl) & (n >= -nl) & (n < nl) & (npr >= -nl) & (npr < nl)
            vals = tab[np.clip(m + nl, 0, 2 * nl), np.clip(n + nl, 0, 2 * nl - 1), np.clip(npr + nl, 0, 2 * nl - 1)]
            arr = np.where(inside, vals, arr)
        out.append(arr)
    return out


# ----------------------------------------------------------------------------- grids


@dataclass
class Grid:
    p: object
    T: float
    nk: int
    n_lo: int
    n_hi: int
    m_lo: int
    m_hi: int
    e_lo: int
    e_hi: int
    bf_lo: int
    bf_hi: int
    bb_lo: int
    bb_hi: int
    kx: np.ndarray
    ky: np.ndarray
    eps: np.ndarray

    def kadd(self, a, b):
        L = self.p.L
        return ((a // L + b // L) % L) * L + (a % L + b % L) % L

    def kneg(self, a):
        L = self.p.L
        return ((-(a // L)) % L) * L + (-(a % L)) % L

    def ksub(self, a, b):
        return self.kadd(a, self.kneg(b))

    def nu(self, n):
        return (2 * np.asarray(n) + 1) * np.pi / self.p.beta

    def w(self, m):
        return 2 * np.asarray(m) * np.pi / self.p.beta


def make_grid(p) -> Grid:
    L = p.L
    ik = np.arange(L * L)
    kx = 2 * np.pi * (ik // L) / L
    ky = 2 * np.pi * (ik % L) / L
    if p.lattice == "square":
        eps = -2.0 * p.hop * (np.cos(kx) + np.cos(ky))  # Eq. Hubbard
    else:
        if L != 1:
            raise ValueError("the Bethe lattice is single-site (L = 1)")
        eps = np.zeros(1)
    n_lo, n_hi = -p.n_nu // 2, p.n_nu // 2 - 1
    m_lo = -(p.n_Omega // 2)
    m_hi = m_lo + p.n_Omega - 1
    f = p.sigma2_factor
    bb_lo = -((f * p.n_Omega) // 2)
    return Grid(
        p=p, T=1.0 / p.beta, nk=L * L, n_lo=n_lo, n_hi=n_hi, m_lo=m_lo, m_hi=m_hi,
        e_lo=m_lo + n_lo, e_hi=m_hi + n_hi, bf_lo=-(f * p.n_nu) // 2, bf_hi=(f * p.n_nu) // 2 - 1,
        bb_lo=bb_lo, bb_hi=bb_lo + f * p.n_Omega - 1, kx=kx, ky=ky, eps=eps,
    )


# ----------------------------------------------------------------------------- one-particle


def g0_inverse(g: Grid, ik, n):
    """Inverse non-interacting propagator at momentum index ik and fermionic index n.

    Square lattice: i nu + mu - eps_k (Eq. PA_Dyson without Sigma).  Bethe lattice:
    inverse of the semicircular Hilbert transform (2/D^2)(i nu - i sgn(nu) sqrt(nu^2+D^2)),
    used as the fixed Weiss function of the single-site solve (Sec. III.A).
    """
    p = g.p
    nu = g.nu(n)
    if p.lattice == "square":
        return 1j * nu + p.mu - g.eps[ik]
    Dh = p.hop
    g0 = (2.0 / Dh**2) * (1j * nu - 1j * np.sign(nu) * np.sqrt(nu * nu + Dh * Dh))
    return 1.0 / g0 + 0.0 * ik


def sigma_tail_c1(g: Grid, sigma):
    """Coefficient c1 of Sigma ~ c1/(i nu) read off the two outer stored frequencies."""
    nu_lo, nu_hi = g.nu(g.e_lo), g.nu(g.e_hi)
    c = -(nu_lo * sigma[:, 0].imag + nu_hi * sigma[:, -1].imag) / 2.0
    return float(np.mean(c))


def sigma_at(g: Grid, sigma, c1, ik, n):
    """Sigma(k) on the stored extended range, c1/(i nu) beyond it."""
    ik = np.asarray(ik)
    n = np.asarray(n)
    inside = (n >= g.e_lo) & (n <= g.e_hi)
    e = np.clip(n - g.e_lo, 0, g.e_hi - g.e_lo)
    tail = c1 / (1j * g.nu(n))
    return np.where(inside, sigma[ik, e], tail)


def green(g: Grid, sigma, c1, ik, n):
    """Dyson equation G(k) = [G0(k)^-1 - Sigma(k)]^-1 (Eq. PA_Dyson)."""
    return 1.0 / (g0_inverse(g, ik, n) - sigma_at(g, sigma, c1, ik, n))


class Propagator:
    """G on a fermionic range wide enough for every sum of one iteration."""

    def __init__(self, g: Grid, sigma):
        self.g = g
        self.c1 = sigma_tail_c1(g, sigma)
        f_lo = min(g.e_lo + g.bb_lo, g.bf_lo + g.bb_lo, g.bb_lo - g.bf_hi - 1, g.bb_lo - g.e_hi - 1, g.bf_lo)
        f_hi = max(g.e_hi + g.bb_hi, g.bf_hi + g.bb_hi, g.bb_hi - g.bf_lo - 1, g.bb_hi - g.e_lo - 1, g.bf_hi)
        self.lo, self.hi = f_lo, f_hi
        ik = np.arange(g.nk)[:, None]
        n = np.arange(f_lo, f_hi + 1)[None, :]
        self.table = green(g, sigma, self.c1, ik, n)
        self.sigma = sigma

    def __call__(self, ik, n):
        n = np.asarray(n)
        assert n.min() >= self.lo and n.max() <= self.hi
        return self.table[ik, n - self.lo]


# ----------------------------------------------------------------------------- bubbles


def box_indices(g: Grid):
    """Momentum and frequency of every compound index of the vertex box."""
    p = g.p
    k = np.arange(p.n)
    q = np.arange(p.n_Q)
    return (k // p.n_nu, g.n_lo + k % p.n_nu, q // p.n_Omega, g.m_lo + q % p.n_Omega)


def bubbles(g: Grid, G: Propagator):
    """X_ph(Q,k) = (T/N) G(k) G(k+q) and X_pp(Q,k) = (T/N) G(k) G(q-k) (Eq. PA_F_Phi)."""
    kk, kn, qk, qm = box_indices(g)
    c = g.T / g.nk
    Gk = G(kk, kn)[None, :]
    Gkq = G(g.kadd(kk[None, :], qk[:, None]), kn[None, :] + qm[:, None])
    Gqk = G(g.ksub(qk[:, None], kk[None, :]), qm[:, None] - kn[None, :] - 1)
    return c * Gk * Gkq, c * Gk * Gqk


# ----------------------------------------------------------------------------- kernel functions


def extract_kernels(g: Grid, phi):
    """Kernel functions of the reducible vertex (Sec. II.A).

    K1[r, Q]: first-level kernel, the background of Phi_r(Q), taken at the four
    corners of the frequency box (far from the diagonal and the stripes).
    K2row[r, Q, k], K2col[r, Q, k']: second-level kernels minus K1, Phi_r at the
    two frequency edges of the other leg; the level-2 approximation is
    K1 + K2row(k) + K2col(k').

    Ablations of the same section (Params.edge_rule, Params.kernel_level): with
    edge_rule "lower" the second-level kernels are Phi_r at the lower frequency edge
    of the other leg alone, as in the paper's example of one edge, and K1 the corner
    at the lower edges of both legs; with kernel_level 1 only the background is kept
    (first-level approximation, K2 = 0).
    """
    p = g.p
    nk, nn = g.nk, p.n_nu
    v = phi.reshape(4, p.n_Q, nk, nn, nk, nn)
    edges = [0] if getattr(p, "edge_rule", "both") == "lower" else [0, nn - 1]
    ne = len(edges)
    K1 = sum(v[:, :, :, a, :, b].mean(axis=(2, 3)) for a in edges for b in edges) / (ne * ne)
    rows = sum(v[:, :, :, :, :, b].mean(axis=4) for b in edges) / ne  # (4, Q, k, n)
    cols = sum(v[:, :, :, a, :, :].mean(axis=2) for a in edges) / ne  # (4, Q, k', n')
    K2row = rows.reshape(4, p.n_Q, p.n) - K1[:, :, None]
    K2col = cols.reshape(4, p.n_Q, p.n) - K1[:, :, None]
    if getattr(p, "kernel_level", 2) == 1:
        K2row = np.zeros_like(K2row)
        K2col = np.zeros_like(K2col)
    return K1, K2row, K2col


# ----------------------------------------------------------------------------- parquet equations


def crossed_args(g: Grid, kind, k, n, kp, np_, q, m):
    """Row leg, column leg and transfer of the crossed vertices in Eq. PA_F.

    Momenta add modulo the lattice; Matsubara indices follow from
    nu_n = (2n+1) pi T and w_m = 2 m pi T, e.g. k + k' + q -> m = n + n' + m + 1.
    """
    if kind == "own":
        return (k, n), (kp, np_), (q, m)
    if kind == "A":  # Phi^{k,k+q}(k'-k)
        return (k, n), (g.kadd(k, q), n + m), (g.ksub(kp, k), np_ - n)
    if kind == "B":  # Psi^{k,k'}(k+k'+q)
        return (k, n), (kp, np_), (g.kadd(g.kadd(k, kp), q), n + np_ + m + 1)
    if kind == "C":  # Phi^{k,q-k'}(k'-k)
        return (k, n), (g.ksub(q, kp), m - np_ - 1), (g.ksub(kp, k), np_ - n)
    if kind == "D":  # Phi^{k,k'}(q-k-k')
        return (k, n), (kp, np_), (g.ksub(g.ksub(q, k), kp), m - n - np_ - 1)
    raise ValueError(kind)


def _flat(g: Grid, leg):
    kk, nn = leg
    inb = (nn >= g.n_lo) & (nn <= g.n_hi)
    return kk * g.p.n_nu + np.clip(nn - g.n_lo, 0, g.p.n_nu - 1), inb


def _flatQ(g: Grid, tr):
    qq, mm = tr
    inb = (mm >= g.m_lo) & (mm <= g.m_hi)
    return qq * g.p.n_Omega + np.clip(mm - g.m_lo, 0, g.p.n_Omega - 1), inb


def kernel_value(g: Grid, K, x, a, b, tr):
    """Level-2 kernel approximation of Phi_x^{a,b}(tr) (Sec. II.A):
    K1(tr) + K2row(a;tr) + K2col(b;tr), a K2 term only where its leg lies in the
    box, and 0 for a transfer outside the bosonic box."""
    K1, K2r, K2c = K
    ai, ain = _flat(g, a)
    bi, bin_ = _flat(g, b)
    qi, qin = _flatQ(g, tr)
    val = K1[x, qi] + np.where(ain, K2r[x, qi, ai], 0) + np.where(bin_, K2c[x, qi, bi], 0)
    return np.where(qin, val, 0)


def vertex_value(g: Grid, phi, K, x, a, b, tr):
    """Phi_x^{a,b}(tr): the stored value inside the box, else the kernel fill
    (Sec. II.A, "supplementing the reducible vertex functions with the
    corresponding kernel functions whenever their arguments exceed the
    parameter space")."""
    ai, ain = _flat(g, a)
    bi, bin_ = _flat(g, b)
    qi, qin = _flatQ(g, tr)
    stored = phi[x, qi, ai, bi]
    return np.where(ain & bin_ & qin, stored, kernel_value(g, K, x, a, b, tr))


def parquet_gamma(g: Grid, r, lam_r, lookup, k, n, kp, np_, q, m):
    """Gamma_r = Lambda_r + sum_i c_i Phi_{x_i}[crossed args] (Eqs. PA_Gamma_dm, PA_Gamma_st)."""
    out = lam_r + np.zeros(np.broadcast(k, n, kp, np_, q, m).shape, dtype=np.complex128)
    for coef, x, kind in PARQUET_TERMS[r]:
        a, b, tr = crossed_args(g, kind, k, n, kp, np_, q, m)
        out = out + coef * lookup(x, a, b, tr)
    return out


def assemble(g: Grid, phi, K, lam, Qs=None, ks=None):
    """Gamma_r and F_r = Gamma_r + Phi_r (Eqs. PA_F, PA_F_G) on the box, or on the
    transfer slices Qs and row legs ks only (all columns k')."""
    p = g.p
    kk, kn, qk, qm = box_indices(g)
    Qs = np.arange(p.n_Q) if Qs is None else np.asarray(Qs)
    ks = np.arange(p.n) if ks is None else np.asarray(ks)
    q3, k3, kp3 = qk[Qs][:, None, None], kk[ks][None, :, None], kk[None, None, :]
    m3, n3, np3 = qm[Qs][:, None, None], kn[ks][None, :, None], kn[None, None, :]
    lookup = lambda x, a, b, tr: vertex_value(g, phi, K, x, a, b, tr)  # noqa: E731
    gamma = np.empty((4, Qs.size, ks.size, p.n), dtype=np.complex128)
    for r in range(4):
        lam_r = lam[r][Qs][:, ks] if np.ndim(lam[r]) == 3 else lam[r]  # tabulated or scalar
        gamma[r] = parquet_gamma(g, r, lam_r, lookup, k3, n3, kp3, np3, q3, m3)
    # the selected slices and rows only (a broadcast state is never materialised whole)
    return gamma, gamma + phi[np.ix_(np.arange(4), Qs, ks)]


def aux_vertex_minus_lambda0(g: Grid, K, r, k, n, kp, np_, q, m):
    """F~_r - Lambda^0_r at arbitrary arguments (Sec. II.B, Eq. auxiliary_function,
    written with the level-2 kernels for all four channels)."""
    lookup = lambda x, a, b, tr: kernel_value(g, K, x, a, b, tr)  # noqa: E731
    own = kernel_value(g, K, r, (k, n), (kp, np_), (q, m))
    return parquet_gamma(g, r, 0.0, lookup, k, n, kp, np_, q, m) + own


# ----------------------------------------------------------------------------- Bethe-Salpeter


def bse(gamma, F, X_ph, X_pp):
    """Phi_r(Q) = s_r Gamma_r(Q) diag(X_r(Q)) F_r(Q) (Eq. PA_F_Phi), one matrix product per (r, Q)."""
    out = np.empty_like(gamma)
    for r in range(4):
        X = X_ph if r < 2 else X_pp
        out[r] = BSE_SIGN[r] * np.matmul(gamma[r] * X[:, None, :], F[r])
    return out


# ----------------------------------------------------------------------------- self-energy


def sde_weights(g: Grid, G: Propagator, k, n, kp, np_, q, m):
    """G(k+q) G(k'+q) G(k') and G(q-k') G(q-k) G(k') of Eq. PA_Sigma."""
    Gkp = G(kp, np_)
    ph = G(g.kadd(k, q), n + m) * G(g.kadd(kp, q), np_ + m) * Gkp
    pp = G(g.ksub(q, kp), m - np_ - 1) * G(g.ksub(q, k), m - n - 1) * Gkp
    return ph, pp


def sigma_delta_F(g: Grid, G: Propagator, F, K, lam, ks=None):
    """Box part of the regulated self-energy (Sec. II.B):
    -(U/4)(T/N)^2 sum_{k',q in box} [GGG (dF_d - dF_m) + GGG (dF_s + dF_t)], dF = F - F~,
    for every k of the box, or for the row legs ks given F[:, :, ks, :]."""
    p = g.p
    kk, kn, qk, qm = box_indices(g)
    ks = np.arange(p.n) if ks is None else np.asarray(ks)
    q3, k3, kp3 = qk[:, None, None], kk[ks][None, :, None], kk[None, None, :]
    m3, n3, np3 = qm[:, None, None], kn[ks][None, :, None], kn[None, None, :]
    l0 = lambda0(p.U)
    dF = [F[r] - l0[r] - aux_vertex_minus_lambda0(g, K, r, k3, n3, kp3, np3, q3, m3) for r in range(4)]
    ph, pp = sde_weights(g, G, k3, n3, kp3, np3, q3, m3)
    tot = (ph * (dF[D] - dF[M]) + pp * (dF[S] + dF[T_])).sum(axis=(0, 2))  # over q and k'
    pref = -(p.U / 4.0) * (g.T / g.nk) ** 2
    out = np.zeros((g.nk, p.n_ext), dtype=np.complex128)
    out[kk[ks], kn[ks] - g.e_lo] = pref * tot
    return out


def sigma_truncated(g: Grid, G: Propagator, F):
    """Eq. PA_Sigma summed on the vertex box with the vertex cut off at its boundary,
    the direct truncation that Sec. II.B regulates and Sec. III contrasts with:
    -(U/4)(T/N)^2 sum_{k',q in box} [G(k+q)G(k'+q)G(k')(F_d - F_m) + G(q-k')G(q-k)G(k')(F_s + F_t)]
    for every k of the box; zero for k outside it, where the truncated vertex vanishes."""
    p = g.p
    kk, kn, qk, qm = box_indices(g)
    q3, k3, kp3 = qk[:, None, None], kk[None, :, None], kk[None, None, :]
    m3, n3, np3 = qm[:, None, None], kn[None, :, None], kn[None, None, :]
    ph, pp = sde_weights(g, G, k3, n3, kp3, np3, q3, m3)
    tot = (ph * (F[D] - F[M]) + pp * (F[S] + F[T_])).sum(axis=(0, 2))  # over q and k'
    out = np.zeros((g.nk, p.n_ext), dtype=np.complex128)
    out[kk, kn - g.e_lo] = -(p.U / 4.0) * (g.T / g.nk) ** 2 * tot
    return out


def sigma2_kernel_terms(g: Grid, G: Propagator, K, outputs=None, chunk_elems=1 << 22):
    """Sigma~2 (Sec. II.B): Eq. PA_Sigma with F~ - Lambda^0, summed directly over
    k' and q on the box enlarged sigma2_factor times, for every k of the
    extended range (or the listed (ik, n) outputs)."""
    p = g.p
    bf = np.arange(g.bf_lo, g.bf_hi + 1)
    bb = np.arange(g.bb_lo, g.bb_hi + 1)
    kp = np.repeat(np.arange(g.nk), bf.size)[None, None, :]
    np_ = np.tile(bf, g.nk)[None, None, :]
    q = np.repeat(np.arange(g.nk), bb.size)[None, :, None]
    m = np.tile(bb, g.nk)[None, :, None]
    pref = -(p.U / 4.0) * (g.T / g.nk) ** 2
    if outputs is None:
        outputs = [(ik, n) for ik in range(g.nk) for n in range(g.e_lo, g.e_hi + 1)]
    outputs = np.asarray(outputs, dtype=np.int64).reshape(-1, 2)
    out = np.zeros((g.nk, p.n_ext), dtype=np.complex128)
    step = max(1, chunk_elems // (kp.size * q.size))
    for s0 in range(0, len(outputs), step):
        ik = outputs[s0:s0 + step, 0][:, None, None]
        nn = outputs[s0:s0 + step, 1][:, None, None]
        ph, pp = sde_weights(g, G, ik, nn, kp, np_, q, m)
        f = [aux_vertex_minus_lambda0(g, K, r, ik, nn, kp, np_, q, m) for r in range(4)]
        val = (ph * (f[D] - f[M]) + pp * (f[S] + f[T_])).sum(axis=(1, 2))
        out[ik[:, 0, 0], nn[:, 0, 0] - g.e_lo] = pref * val
    return out


def tau_nodes(p):
    """Composite Gauss-Legendre nodes and weights on [0, beta]."""
    x, w = np.polynomial.legendre.leggauss(p.tau_order)
    h = p.beta / p.tau_panels
    a = np.arange(p.tau_panels)[:, None] * h
    tau = (a + 0.5 * h * (x[None, :] + 1.0)).ravel()
    wt = np.tile(0.5 * h * w, p.tau_panels)
    return tau, wt


def tail_moments(g: Grid, c1):
    """c2(k), c3(k) of G(k) = 1/(i nu) + c2/(i nu)^2 + c3/(i nu)^3 + O(nu^-4)."""
    p = g.p
    if p.lattice == "square":
        a = g.eps - p.mu
        return a, a * a + c1
    return np.zeros(1), np.full(1, p.hop**2 / 4.0 + c1)


def green_tau(g: Grid, sigma, c1, tau):
    """G(k, tau) for 0 < tau < beta from its Matsubara sum, with the 1/(i nu)^j
    tails (j = 1, 2, 3) transformed analytically: -1/2, tau/2 - beta/4, tau(beta-tau)/4."""
    p = g.p
    Mc = p.tau_matsubara
    n = np.arange(-Mc, Mc)
    iv = 1j * g.nu(n)
    c2, c3 = tail_moments(g, c1)
    ik = np.arange(g.nk)[:, None]
    Gk = green(g, sigma, c1, ik, n[None, :])
    R = Gk - (1.0 / iv[None, :] + c2[:, None] / iv[None, :] ** 2 + c3[:, None] / iv[None, :] ** 3)
    E = np.exp(-1j * np.outer(g.nu(n), tau))  # (n, tau)
    Gt = g.T * (R @ E)
    b = p.beta
    Gt = Gt - 0.5 + c2[:, None] * (tau / 2 - b / 4)[None, :] + c3[:, None] * (tau * (b - tau) / 4)[None, :]
    return Gt


def sigma1_second_order(g: Grid, sigma):
    """Sigma~1: the second-order diagram with Lambda^0 (Sec. II.B), evaluated for
    all frequencies in imaginary time: Sigma(r, tau) = -U^2 G(r,tau)^2 G(-r,-tau)
    with G(-r,-tau) = -G(-r, beta-tau), then transformed back to the extended range."""
    p = g.p
    c1 = sigma_tail_c1(g, sigma)
    tau, wt = tau_nodes(p)
    Gkt = green_tau(g, sigma, c1, tau)  # (k, tau)
    # real space: G(r, tau) = (1/N) sum_k e^{i k r} G(k, tau)
    rx, ry = g.kx * p.L / (2 * np.pi), g.ky * p.L / (2 * np.pi)  # site coordinates share the index layout
    phase = np.exp(1j * (np.outer(rx, g.kx) + np.outer(ry, g.ky)))  # (r, k)
    Grt = phase @ Gkt / g.nk
    rneg = g.kneg(np.arange(g.nk))
    Gm = Grt[rneg][:, ::-1]  # G(-r, beta - tau): the nodes are symmetric about beta/2
    Srt = p.U**2 * Grt**2 * Gm
    n = np.arange(g.e_lo, g.e_hi + 1)
    Ef = np.exp(1j * np.outer(tau, g.nu(n))) * wt[:, None]  # (tau, n)
    Sr = Srt @ Ef  # (r, n)
    return phase.conj().T @ Sr  # (k, n)


# ----------------------------------------------------------------------------- iteration


@dataclass
class State:
    phi: np.ndarray  # (4, N_Q, n, n) complex128
    sigma: np.ndarray  # (N, n_ext) complex128


@dataclass
class IterationResult:
    state: State
    gamma: np.ndarray
    F: np.ndarray
    X_ph: np.ndarray
    X_pp: np.ndarray
    sigma_new: np.ndarray
    phi_new: np.ndarray
    max_dsigma: float
    K: tuple
    mu: float = 0.0


def zero_state(p) -> State:
    return State(np.zeros((4, p.n_Q, p.n, p.n), np.complex128), np.zeros((p.n_k, p.n_ext), np.complex128))


def iterate(p, state: State, lam=None) -> IterationResult:
    """One Jacobi parquet iteration from (Phi, Sigma) (Sec. II): Dyson, bubbles,
    kernel functions, parquet equations, regulated Schwinger-Dyson, BSE, mixing.
    With p.density > 0 the chemical potential is first set so that the state's G holds
    that many electrons per site (find_mu); the result's params carry it."""
    if getattr(p, "density", 0.0) > 0.0:
        p = p.with_(mu=find_mu(p, state.sigma, p.density), density=0.0)
    g = make_grid(p)
    lam = lambda0(p.U) if lam is None else lam
    G = Propagator(g, state.sigma)
    X_ph, X_pp = bubbles(g, G)
    K = extract_kernels(g, state.phi)
    gamma, F = assemble(g, state.phi, K, lam)
    if getattr(p, "sde", "regulated") == "truncated":
        sigma_new = sigma_truncated(g, G, F)
    else:
        s1 = sigma1_second_order(g, state.sigma)
        s2 = sigma2_kernel_terms(g, G, K)
        s3 = sigma_delta_F(g, G, F, K, lam)
        sigma_new = s1 + s2 + s3
    phi_new = bse(gamma, F, X_ph, X_pp)
    a = p.mix
    nxt = State(a * phi_new + (1 - a) * state.phi, a * sigma_new + (1 - a) * state.sigma)
    dmax = float(np.abs(sigma_new - state.sigma).max())
    return IterationResult(nxt, gamma, F, X_ph, X_pp, sigma_new, phi_new, dmax, K, p.mu)


def density(p, sigma):
    """Electron density per site (both spins) of G = [i nu + mu - eps_k - Sigma(k)]^-1 with the
    state's Sigma (App. A, Eq. PA_Dyson; square lattice):
    n = (2T/N) sum_k sum_nu G(k, i nu) e^{i nu 0+}.  The 1/(i nu) and 1/(i nu)^2 tails are summed
    in closed form (T sum_nu e^{i nu 0+}/(i nu) = 1/2, T sum_nu 1/(i nu)^2 = -beta/4), the rest
    over n in [-M, M-1] with M = tau_matsubara (its terms fall off as 1/nu^3 and cancel pairwise
    to leading order)."""
    g = make_grid(p)
    if p.lattice != "square":
        raise ValueError("the density is defined for the lattice solve (the Bethe solve has a fixed G0)")
    c1 = sigma_tail_c1(g, sigma)
    M = p.tau_matsubara
    n = np.arange(-M, M)
    iv = 1j * g.nu(n)
    ik = np.arange(g.nk)[:, None]
    G = green(g, sigma, c1, ik, n[None, :])
    c2 = (g.eps - p.mu)[:, None]
    rest = (G - 1.0 / iv[None, :] - c2 / iv[None, :] ** 2).sum(axis=1).real * g.T
    per_spin = 0.5 - c2[:, 0] * p.beta / 4.0 + rest
    return float(2.0 * per_spin.mean())


def find_mu(p, sigma, n_target, tol=1e-13, lo=-20.0, hi=20.0):
    """Chemical potential with density(mu) = n_target at fixed Sigma, by bisection (n(mu) is
    increasing); mu is the Hartree-shifted one of the solve (mu = 0 at half filling)."""
    f = lambda mu: density(p.with_(mu=mu), sigma) - n_target  # noqa: E731
    a, b = lo, hi
    fa = f(a)
    for _ in range(200):
        m = 0.5 * (a + b)
        fm = f(m)
        if (fm > 0) == (fa > 0):
            a, fa = m, fm
        else:
            b = m
        if b - a < tol:
            break
    return 0.5 * (a + b)


def susceptibility(F, X_ph, X_pp):
    """chi_r(Q) = -sum_k X_r(Q,k) - sum_{k,k'} X_r(Q,k) F_r^{k,k'}(Q) X_r(Q,k')
    (App. A, "Notations": chi from F and the bare bubble, summed over the box)."""
    out = np.empty((4, F.shape[1]), dtype=np.complex128)
    for r in range(4):
        X = X_ph if r < 2 else X_pp
        out[r] = -X.sum(axis=1) - np.einsum("qk,qkl,ql->q", X, F[r], X)
    return out


def solve(p, max_iter, tol, state=None):
    """Iterate to max|Sigma_new - Sigma| < tol or max_iter iterations."""
    st = zero_state(p) if state is None else state
    res = None
    for it in range(max_iter):
        res = iterate(p, st)
        st = res.state
        if res.max_dsigma < tol:
            return res, it + 1
    return res, max_iter
