"""Solver parameters, the named Hubbard workloads, and seeded synthetic states.

This module holds parameters and random draws only: no step of the parquet
method is computed here.  Both the CUDA path (through the C-ABI) and the FP64
CPU oracle take their inputs from it, so a parity test feeds the two sides the
same numbers.

Grid conventions (Sec. II and App. A, "Notations"): a compound fermionic index
k = (k-vector, n) has the Matsubara index n fastest; a compound bosonic index
Q = (q-vector, m) has m fastest.  The vertex box holds n in [-Nnu/2, Nnu/2-1]
and m in [m_lo, m_lo+NOmega-1] with m_lo = -floor(NOmega/2).  The self-energy
is stored on the extended fermionic range of NOmega+Nnu-1 frequencies that the
bubbles G(k+q), G(q-k) reach.
"""
from __future__ import annotations

from dataclasses import dataclass, replace

import numpy as np

BETHE = "bethe"
SQUARE = "square"

FP64 = "fp64"
SPLIT_TF32X3 = "split_tf32x3"
SPLIT_BF16X3 = "split_bf16x3"
SPLIT_BF16X6 = "split_bf16x6"
SPLIT_FP16X3 = "split_fp16x3"


@dataclass(frozen=True)
class Params:
    """Physical and numerical parameters of one parquet solve.

    lattice   "bethe" (single-site, semicircular DOS of half-bandwidth ``hop``)
              or "square" (eps_k = -2 hop (cos kx + cos ky) on an L x L grid).
    beta, U, mu   inverse temperature, Hubbard U, chemical potential (mu=0 is
              half filling, the Hartree shift being absorbed in mu).
    L         linear momentum grid size (1 for the single-site solve).
    n_nu, n_Omega   fermionic / bosonic Matsubara frequencies per argument.
    mix       linear mixing weight alpha of the new iterate.
    sigma2_factor   size of the kernel-term summation box relative to the
              vertex box (Sec. II.B: "two or three times larger").
    tau_panels, tau_order, tau_matsubara   quadrature of the second-order
              self-energy: Gauss-Legendre panels on [0, beta], nodes per panel,
              and the Matsubara cut (n in [-M, M-1]) of the G(tau) sums.
    kernel_level   2: the fill uses K1 + K2 (second level); 1: K1 only (Sec. II.A).
    edge_rule      "both": K2 from the mean of the lower and upper frequency edges of
              the other leg; "lower": the lower edge alone (Sec. II.A).
    sde       "regulated": Sigma = Sigma~1 + Sigma~2 + the box sum of F - F~ (Sec. II.B);
              "truncated": Eq. PA_Sigma on the box with the vertex cut off there.
    density   0: mu is fixed; > 0 (square lattice): electrons per site (both spins) to hold,
              mu being searched at the start of every iteration on the state's Sigma.
    """

    lattice: str
    beta: float
    U: float
    mu: float
    L: int
    n_nu: int
    n_Omega: int
    hop: float = 1.0
    mix: float = 0.5
    sigma2_factor: int = 3
    tau_panels: int = 64
    tau_order: int = 16
    tau_matsubara: int = 2048
    kernel_level: int = 2
    edge_rule: str = "both"
    sde: str = "regulated"
    density: float = 0.0

    @property
    def n_k(self) -> int:
        return self.L * self.L

    @property
    def n(self) -> int:
        return self.n_k * self.n_nu

    @property
    def n_Q(self) -> int:
        return self.n_k * self.n_Omega

    @property
    def n_ext(self) -> int:
        return self.n_Omega + self.n_nu - 1

    def with_(self, **kw) -> "Params":
        return replace(self, **kw)


# Named workloads (Hubbard model, Sec. III and App. A).
CONFIGS = {
    # single-site parquet approximation on the Bethe lattice, D = 1
    "bethe_u1_b10": Params(BETHE, beta=10.0, U=1.0, mu=0.0, L=1, n_nu=32, n_Omega=31, hop=1.0),
    # 2D square lattice, 4x4 momenta: BSE matrices of 256 x 256
    "square4_u2_b5": Params(SQUARE, beta=5.0, U=2.0, mu=0.0, L=4, n_nu=16, n_Omega=16),
    # 2D square lattice, 8x8 momenta: BSE matrices of 1024 x 1024
    "square8_u2_b4": Params(SQUARE, beta=4.0, U=2.0, mu=0.0, L=8, n_nu=16, n_Omega=16),
    # large single solve: 8x8 momenta, 24 frequencies: BSE matrices of 1536 x 1536
    "square8_u3_b8_nu24": Params(SQUARE, beta=8.0, U=3.0, mu=0.0, L=8, n_nu=24, n_Omega=24),
    # the large solve's frequency box on the 4x4 lattice (n = 384, 0.45 GB of Phi): a small
    # case of the same kernels for profiling captures
    "square4_u3_b8_nu24": Params(SQUARE, beta=8.0, U=3.0, mu=0.0, L=4, n_nu=24, n_Omega=24),
    # BSE matrices of the 8x8 workload's size (n = 1024) on 64 transfer slices (4x4 momenta,
    # Nnu = 64, NOmega = 1; 0.5 GB of Phi): the n = 1024 products for profiling captures
    "square4_nu64_om1": Params(SQUARE, beta=4.0, U=2.0, mu=0.0, L=4, n_nu=64, n_Omega=1),
}


def batch_draw(seed: int = 1510, count: int = 64) -> list[Params]:
    """The seeded batch of uneven solves: square lattices with L ~ U{2..6}, Nnu ~ U{8, 16, 24, 32}
    (NOmega = Nnu), U ~ U[0.5, 3], beta ~ U[2, 10], half filling; numpy PCG64 with the given seed,
    drawn in the order (L, Nnu, U, beta) solve by solve."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for _ in range(count):
        L = int(rng.integers(2, 7))
        nu = int(rng.choice([8, 16, 24, 32]))
        U = float(rng.uniform(0.5, 3.0))
        beta = float(rng.uniform(2.0, 10.0))
        out.append(Params(SQUARE, beta=beta, U=U, mu=0.0, L=L, n_nu=nu, n_Omega=nu))
    return out


def device_bytes_planes(p: Params, precision: str = SPLIT_FP16X3) -> int:
    """Device memory of a single-pass solve with operand planes: Phi (complex64, 8 bytes per
    element) and the BSE operand planes (Gamma X 8 bytes, F 8 bytes for FP16x3 or 12 for BF16x3
    per element; rows padded to 8 elements), plus the one-particle and self-energy tables
    (bounded by 128 MB at the default quadrature)."""
    ld = (p.n + 7) // 8 * 8
    ops = 16 if precision == SPLIT_FP16X3 else 20
    return 4 * p.n_Q * p.n * (8 * p.n + ops * ld) + (128 << 20)


def random_state(p: Params, seed: int, amplitude: float | None = None):
    """Seeded synthetic reducible vertex and self-energy of the paper's shape.

    Phi[r, Q, k, k'] (r = d, m, s, t) is a background that decays as 1/(1+w^2)
    in the transfer frequency plus row and column stripes and a small noise,
    the structure Sec. II.A describes for the reducible vertex; Sigma[k_vec, e]
    on the extended range is -i c/nu plus noise.  Returns (Phi, Sigma) as
    complex128 arrays.
    """
    rng = np.random.default_rng(seed)
    amp = (p.U * p.U * 0.2) if amplitude is None else amplitude
    m = np.arange(p.n_Omega) - p.n_Omega // 2
    w = 2.0 * np.pi * m / p.beta
    decay = 1.0 / (1.0 + w * w)
    decay_Q = np.tile(decay, p.n_k)  # Q = (q, m), m fastest

    def cplx(*shape):
        return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)

    back = amp * cplx(4, p.n_Q) * decay_Q[None, :]
    row = 0.3 * amp * cplx(4, p.n_Q, p.n) * decay_Q[None, :, None]
    col = 0.3 * amp * cplx(4, p.n_Q, p.n) * decay_Q[None, :, None]
    noise = 0.05 * amp * cplx(4, p.n_Q, p.n, p.n)
    phi = back[:, :, None, None] + row[:, :, :, None] + col[:, :, None, :] + noise

    e = np.arange(p.n_ext) - (p.n_Omega // 2) - p.n_nu // 2
    nu = (2 * e + 1) * np.pi / p.beta
    sig = (-1j * 0.25 * p.U * p.U / nu)[None, :] * (1.0 + 0.1 * rng.standard_normal((p.n_k, p.n_ext)))
    sig = sig + 0.02 * p.U * cplx(p.n_k, p.n_ext)
    return phi.astype(np.complex128), sig.astype(np.complex128)
