"""Writes the stored expected values under tests/golden/ from closed forms of the paper,
evaluated here with numpy and scipy only (neither the oracle nor the CUDA path is used).
The paper prints no numerical tables (its results are plots), so the fixtures are its
worked example and its second-order limit evaluated at the parameters named in each file.

    python tests/golden/make_golden.py
"""
from __future__ import annotations

import os

import numpy as np
from scipy import integrate
from scipy.interpolate import CubicSpline

HERE = os.path.dirname(os.path.abspath(__file__))


def fermi(e, beta):
    return 0.5 * (1.0 - np.tanh(0.5 * beta * e))


def bethe_ipt(beta=5.0, U=1.0, D=1.0, nmax=8, ntau=801):
    """Second-order self-energy of the half-filled Bethe lattice (semicircular DOS of
    half-bandwidth D): Sigma(i nu_n) = U^2 int_0^beta e^{i nu_n tau} G0(tau)^3 d tau with
    G0(tau) = -int rho(e) e^{-e tau} f(-e) de (Sec. II.B: Sigma~1 is the second-order diagram;
    at the first iteration from Phi = 0 the regulated Sigma equals it)."""
    rho = lambda e: 2.0 / (np.pi * D * D) * np.sqrt(max(D * D - e * e, 0.0))  # noqa: E731
    ts = np.linspace(0.0, beta, ntau)
    g0 = np.array([-integrate.quad(lambda e: rho(e) * np.exp(-e * t) * fermi(-e, beta), -D, D, epsabs=1e-13)[0]
                   for t in ts])
    sp = CubicSpline(ts, U * U * g0**3)
    out = []
    for n in range(nmax):
        nu = (2 * n + 1) * np.pi / beta
        re = integrate.quad(lambda t: np.cos(nu * t) * sp(t), 0, beta, limit=400, epsabs=1e-13)[0]
        im = integrate.quad(lambda t: np.sin(nu * t) * sp(t), 0, beta, limit=400, epsabs=1e-13)[0]
        out.append((n, re, im))
    return out


def first_iteration_square(L=2, beta=3.0, U=1.5, mu=0.0, t=1.0, n_nu=8, n_omega=8):
    """The worked first iteration of Sec. II.A: with F = Gamma = (U, -U, 2U, 0),
    Phi_d = Phi_m = U^2 (T/N) sum_k'' G0(k'') G0(k''+q), Phi_s = -2 U^2 (T/N) sum_k''
    G0(k'') G0(q-k''), Phi_t = 0, the sum over the momenta and the fermionic box
    n'' in [-Nnu/2, Nnu/2 - 1]; G0(k, i nu) = 1/(i nu + mu - eps_k), eps_k = -2t(cos kx + cos ky);
    q = (q-vector, m) with m in [-floor(NOmega/2), ...]."""
    T, N = 1.0 / beta, L * L
    ks = [(2 * np.pi * x / L, 2 * np.pi * y / L) for x in range(L) for y in range(L)]

    def g0(ki, n):
        kx, ky = ks[ki]
        return 1.0 / (1j * (2 * n + 1) * np.pi * T + mu + 2 * t * (np.cos(kx) + np.cos(ky)))

    def kadd(a, b):
        return ((a // L + b // L) % L) * L + (a % L + b % L) % L

    def kneg(a):
        return ((L - a // L) % L) * L + (L - a % L) % L

    nlo, mlo = -n_nu // 2, -(n_omega // 2)
    rows = []
    for iq in range(N):
        for mi in range(n_omega):
            m = mlo + mi
            ph = pp = 0.0
            for kk in range(N):
                for n in range(nlo, nlo + n_nu):
                    ph += g0(kk, n) * g0(kadd(kk, iq), n + m)
                    pp += g0(kk, n) * g0(kadd(iq, kneg(kk)), m - n - 1)
            rows.append((iq * n_omega + mi, U * U * T / N * ph, -2.0 * U * U * T / N * pp))
    return rows


def second_order_square(L=3, beta=2.0, U=1.1, mu=0.15, t=0.8, n_nu=6, n_omega=5):
    """Second-order self-energy of the free square lattice (Sec. II.B: Sigma~1, and the regulated
    Sigma of the first iteration from Phi = 0) with Fermi functions:
    Sigma(k, i nu) = (U^2/N^2) sum_{a,b} [(1-f_a)(1-f_b) f_c + f_a f_b (1-f_c)] / (i nu - e_a - e_b + e_c),
    c = a + b - k, e = eps - mu, on the extended range e in [m_lo + n_lo, m_hi + n_hi]."""
    N = L * L
    ks = [(x, y) for x in range(L) for y in range(L)]
    e = np.array([-2 * t * (np.cos(2 * np.pi * x / L) + np.cos(2 * np.pi * y / L)) - mu for x, y in ks])
    f = fermi(e, beta)
    nlo, mlo = -n_nu // 2, -(n_omega // 2)
    ns = np.arange(mlo + nlo, mlo + n_omega - 1 + nlo + n_nu)
    nu = (2 * ns + 1) * np.pi / beta
    rows = []
    for ik, (kx, ky) in enumerate(ks):
        s = np.zeros(ns.size, dtype=complex)
        for ia, (ax, ay) in enumerate(ks):
            for ib, (bx, by) in enumerate(ks):
                ic = ((ax + bx - kx) % L) * L + (ay + by - ky) % L
                s += ((1 - f[ia]) * (1 - f[ib]) * f[ic] + f[ia] * f[ib] * (1 - f[ic])) / (1j * nu - e[ia] - e[ib] + e[ic])
        s *= U * U / N**2
        rows += [(ik, int(n), v.real, v.imag) for n, v in zip(ns, s)]
    return rows


def write(name, header, rows):
    with open(os.path.join(HERE, name), "w") as f:
        for line in header:
            f.write("# " + line + "\n")
        for r in rows:
            f.write(" ".join(f"{v:.17g}" if isinstance(v, float) else str(v) for v in r) + "\n")


def main():
    write("bethe_second_order_b5_u1.txt",
          ["Second-order self-energy of the half-filled Bethe lattice, D = 1, beta = 5, U = 1:",
           "Sigma(i nu_n) = U^2 int_0^beta e^{i nu_n tau} G0(tau)^3 dtau (Sec. II.B, Sigma~1; Sec. III.A, Bethe G0),",
           "the regulated Sigma of the first iteration from Phi = 0.  scipy quadrature; columns: n, Re, Im."],
          [(n, re, im) for n, re, im in bethe_ipt()])
    rows = first_iteration_square()
    write("first_iteration_square2_b3_u1p5.txt",
          ["Worked first iteration of Sec. II.A on the 2x2 square lattice, t = 1, beta = 3, U = 1.5, mu = 0,",
           "Nnu = NOmega = 8: Phi_d = Phi_m = U^2 (T/N) sum G0 G0(k''+q), Phi_s = -2 U^2 (T/N) sum G0 G0(q-k''),",
           "Phi_t = 0, constant in (k, k').  Columns: Q = q-index * NOmega + (m - m_lo), Re Phi_d, Im Phi_d, Re Phi_s, Im Phi_s."],
          [(Q, d.real, d.imag, s.real, s.imag) for Q, d, s in rows])
    rows = first_iteration_square(L=3, beta=2.0, U=1.1, mu=0.15, t=0.8, n_nu=6, n_omega=5)
    write("first_iteration_square3_b2_u1p1_mu0p15.txt",
          ["Worked first iteration of Sec. II.A on the 3x3 square lattice, t = 0.8, beta = 2, U = 1.1, mu = 0.15,",
           "Nnu = 6, NOmega = 5 (same formulas as the 2x2 file; on 3x3, k + q and k - q are different points).",
           "Columns: Q = q-index * NOmega + (m - m_lo), Re Phi_d, Im Phi_d, Re Phi_s, Im Phi_s."],
          [(Q, d.real, d.imag, s.real, s.imag) for Q, d, s in rows])
    write("second_order_square3_b2_u1p1_mu0p15.txt",
          ["Second-order self-energy of the free 3x3 square lattice, t = 0.8, beta = 2, U = 1.1, mu = 0.15,",
           "Nnu = 6, NOmega = 5: (U^2/N^2) sum_{a,b} [(1-f_a)(1-f_b) f_c + f_a f_b (1-f_c)]/(i nu - e_a - e_b + e_c),",
           "c = a + b - k (Sec. II.B: Sigma~1, the regulated Sigma of the first iteration from Phi = 0).",
           "Columns: k-index (ix * L + iy), n, Re Sigma, Im Sigma."],
          second_order_square())


if __name__ == "__main__":
    main()
