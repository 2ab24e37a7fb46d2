"""Failure detection through the C ABI, with no GPU fault: every failure is made on the host
(an allocator that returns NULL, a tolerance that cannot be met, an iteration that diverges)
or by a bounded device wait that is made to run out (a barrier nothing arrives at).  The
contexts report the documented status and are left valid or poisoned as the header states."""
import ctypes as C

import numpy as np
import pytest

from oracle import parquet_oracle as O
from paper_1510_03330_gb300.workloads import FP64, SPLIT_FP16X3, Params

pytestmark = pytest.mark.gpu
SMALL = Params("square", beta=2.5, U=1.2, mu=0.0, L=2, n_nu=6, n_Omega=5)


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


@pytest.mark.parametrize("fail_after", [0, 3, 20])
def test_allocator_returning_null_gives_enomem_with_byte_count(gpu, fail_after):
    """A caller's allocator that returns NULL after fail_after allocations: pq_init returns
    PQ_ENOMEM, names the bytes the solve needs, and hands every block it got back."""
    from paper_1510_03330_gb300 import binding as B

    torch = gpu
    lib = B.load_library()
    live = {}

    def alloc(nbytes, _ctx):
        if len(live) >= fail_after:
            return None
        t = torch.empty(int(nbytes), dtype=torch.uint8, device="cuda")
        live[t.data_ptr()] = t
        return t.data_ptr()

    def free(ptr, _nbytes, _ctx):
        live.pop(int(ptr))

    fa, ff = B.ALLOC_FN(alloc), B.FREE_FN(free)
    o = B.default_options()
    o.precision = B.PRECISION[FP64]
    o.dev_alloc, o.dev_free = fa, ff
    h = C.c_void_p()
    st = lib.pq_init(C.byref(h), 1, SMALL.beta, SMALL.U, SMALL.mu, SMALL.L, SMALL.n_nu, SMALL.n_Omega, C.byref(o))
    msg = lib.pq_last_error(None).decode()
    assert st == B.PQ_ENOMEM, (st, msg)
    assert "needs" in msg and "bytes" in msg
    need = int(msg.split("needs")[1].split("bytes")[0])
    assert need > 16 * 4 * SMALL.n_Q * SMALL.n**2  # at least one complex128 copy of Phi
    assert not live  # everything allocated before the failure was released
    assert not h.value


def test_max_iterations_give_enotconv_with_a_valid_state():
    """A tolerance that cannot be met: PQ_ENOTCONV after max_iter iterations, and the state is
    that of max_iter oracle iterations (the context stays usable)."""
    from paper_1510_03330_gb300.binding import PQ_ENOTCONV, Solver

    p = SMALL
    st = O.zero_state(p)
    for _ in range(3):
        res = O.iterate(p, st)
        st = res.state
    with Solver(p) as s:
        its, d, conv = s.iterate(2, tol=1e-300)
        assert not conv and its == 2 and s.last_status == PQ_ENOTCONV
        its, d, conv = s.iterate(1, tol=1e-300)
        assert rel(s.sigma(), st.sigma) < 1e-10
        assert abs(d - res.max_dsigma) < 1e-10 * res.max_dsigma


def test_wait_timeout_poisons_the_context():
    """A bounded device wait made to run out (50 ms on a barrier nothing arrives at) sets the
    timeout flag: PQ_ETIMEOUT, the context is poisoned (PQ_ESTATE after), and the GPU context
    of the process stays usable: a new solve on the same device runs and matches the oracle."""
    from paper_1510_03330_gb300.binding import PQ_ESTATE, PQ_ETIMEOUT, ParquetError, Solver

    with Solver(SMALL, precision=SPLIT_FP16X3) as s:
        s.iterate(1)
        assert s.selftest_wait_timeout(50) == PQ_ETIMEOUT
        assert "gave up" in s.lib.pq_last_error(s.h).decode()
        with pytest.raises(ParquetError) as e:
            s.iterate(1)
        assert e.value.status == PQ_ESTATE
        with pytest.raises(ParquetError) as e:
            s.sigma()
        assert e.value.status == PQ_ESTATE
    res = O.iterate(SMALL, O.zero_state(SMALL))
    with Solver(SMALL) as t:
        t.iterate(1)
        assert rel(t.sigma(), res.state.sigma) < 1e-10


def test_divergence_detection_stops_a_diverging_iteration():
    """The single-site parquet approximation at U = 6, beta = 2 without damping (alpha = 1)
    diverges (the large-U failure of Sec. III): with diverge_window = 2, pq_iterate stops with
    PQ_EDIVERGED after the first iteration whose max|dSigma| grew for the second time in a row
    to more than 10x the larger of its first two values, found here from the oracle's own
    sequence, and keeps a valid state equal to the oracle's after as many iterations."""
    from paper_1510_03330_gb300.binding import PQ_EDIVERGED, Solver

    p = Params("bethe", beta=2.0, U=6.0, mu=0.0, L=1, n_nu=8, n_Omega=7, mix=1.0)
    st = O.zero_state(p)
    ds, states = [], []
    for _ in range(10):
        res = O.iterate(p, st)
        st = res.state
        ds.append(res.max_dsigma)
        states.append(st.sigma)
    grown, stop = 0, None
    for i in range(1, len(ds)):
        grown = grown + 1 if ds[i] > ds[i - 1] else 0
        if grown >= 2 and ds[i] > 10.0 * max(ds[:2]):
            stop = i + 1
            break
    assert stop is not None and stop < 10
    with Solver(p, diverge_window=2) as s:
        its, d, conv = s.iterate(50, tol=1e-8)
        assert s.last_status == PQ_EDIVERGED and not conv
        assert its == stop, (its, stop, ds)
        assert abs(d - ds[stop - 1]) < 1e-8 * ds[stop - 1]
        assert rel(s.sigma(), states[stop - 1]) < 1e-9
    # without detection the same run goes on to max_iter
    with Solver(p) as s:
        its, d, conv = s.iterate(stop + 1, tol=1e-8)
        assert its == stop + 1 and not conv
