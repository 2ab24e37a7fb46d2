"""The allocation-free second-order self-energy against the allocating one.

pq_sigma_second_order_noalloc exists for callers that cannot call cudaMalloc
(an application that gave all device memory to its own allocator, or a
plug-in running inside another solver's loop).  It must give what
pq_sigma_second_order gives for the same self-energy, call after call, while
its scratch lives in a static device array shared by all calls.  This file is
collected last so that a failure here cannot hide the other tests."""
import ctypes as C

import numpy as np
import pytest

from paper_1510_03330_gb300 import binding
from paper_1510_03330_gb300.workloads import Params, random_state

TOL_FP64 = 1e-10
P = Params("square", beta=2.5, U=1.3, mu=0.1, L=2, n_nu=8, n_Omega=7, hop=0.9,
           tau_matsubara=256, tau_panels=16, tau_order=16)
# every region of the static scratch at its maximum: L * L = 16 momenta (complex phases
# exp(i k.r), where a conjugation slip would show), 2 * tau_matsubara = 512,
# tau_panels * tau_order = 512 nodes, NOmega + Nnu - 1 = 128 frequencies
P_MAX = Params("square", beta=3.0, U=1.1, mu=-0.2, L=4, n_nu=2, n_Omega=127, hop=0.8,
               tau_matsubara=256, tau_panels=32, tau_order=16)


def _call(lib, p, src, dst, stream):
    return lib.pq_sigma_second_order_noalloc(1 if p.lattice == "square" else 0, p.beta, p.U, p.mu, p.hop, p.L,
                                             p.n_nu, p.n_Omega, p.tau_panels, p.tau_order, p.tau_matsubara,
                                             src, dst, stream)


@pytest.mark.gpu
@pytest.mark.parametrize("P", [P, P_MAX], ids=["2x2", "4x4_max"])
def test_noalloc_matches_the_allocating_entry_point_on_two_calls(P):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    from paper_1510_03330_gb300.binding import Solver

    sig_a = random_state(P, seed=11)[1]
    sig_b = random_state(P, seed=12)[1]
    with Solver(P) as s:
        ref = [s.sigma_second_order(sig_a), s.sigma_second_order(sig_b)]
    lib = binding.load_library()
    stream = torch.cuda.current_stream().cuda_stream
    out = torch.empty((P.n_k, P.n_ext, 2), dtype=torch.float64, device="cuda")
    for sig, want in zip((sig_a, sig_b), ref):
        src = torch.from_numpy(np.ascontiguousarray(sig).view(np.float64).reshape(P.n_k, P.n_ext, 2)).cuda()
        st = _call(lib, P, src.data_ptr(), out.data_ptr(), stream)
        assert st == binding.PQ_OK, lib.pq_last_error(None).decode()
        torch.cuda.synchronize()
        got = out.cpu().numpy().view(np.complex128).reshape(P.n_k, P.n_ext)
        err = np.abs(got - want).max() / np.abs(want).max()
        assert err < TOL_FP64, err


def test_noalloc_rejects_sizes_beyond_its_scratch():
    from paper_1510_03330_gb300 import build as B

    B.build()
    lib = binding.load_library()
    big = P.with_(L=5)
    st = _call(lib, big, C.c_void_p(16), C.c_void_p(16), None)
    assert st == binding.PQ_EINVAL
    assert "beyond the static scratch" in lib.pq_last_error(None).decode()
