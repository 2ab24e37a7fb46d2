"""GPU parity of batched solves (pq_batch_*): every member of a batch must follow the
same iteration as the same solve iterated alone, whichever grouped-kernel candidate
(tile width, schedule order) runs an iteration and once the iteration is replayed
from the captured graph; one member is also checked against the FP64 oracle."""
import numpy as np
import pytest

from oracle import parquet_oracle as O
from paper_1510_03330_gb300.workloads import FP64, SPLIT_BF16X3, SPLIT_FP16X3, Params

PLANE = {SPLIT_FP16X3: (1e-6, 2e-6), SPLIT_BF16X3: (5e-6, 1.5e-5)}

pytestmark = pytest.mark.gpu

MEMBERS = [
    Params("square", beta=3.0, U=1.5, mu=0.0, L=2, n_nu=8, n_Omega=8),            # n = 32
    Params("square", beta=2.0, U=1.0, mu=0.3, L=3, n_nu=8, n_Omega=7, hop=0.8),   # n = 72
    Params("bethe", beta=4.0, U=1.0, mu=0.0, L=1, n_nu=10, n_Omega=9),            # n = 10 (rows padded)
    Params("square", beta=2.5, U=2.0, mu=0.0, L=3, n_nu=16, n_Omega=8),           # n = 144: two row tiles
]


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
@pytest.mark.parametrize("tile_cols,order", [(0, -1), (64, 1), (128, 0)])
def test_batch_members_follow_their_own_iteration(tile_cols, order, precision):
    from paper_1510_03330_gb300.binding import Batch, Solver

    iters = 7  # with tuning: a warm-up and four candidate iterations, then the captured graph
    alone = [Solver(p, precision=precision) for p in MEMBERS]
    for s in alone:
        s.iterate(iters)
    mem = [Solver(p, precision=precision) for p in MEMBERS]
    with Batch(mem, tile_cols=tile_cols, order=order, time_steps=True) as b:
        for _ in range(iters):
            d = b.iterate(1)
        cfg = b.config()
        t = b.times()
    assert cfg["tile_cols"] in (64, 128) and cfg["order"] in (0, 1), cfg
    if tile_cols:
        assert cfg["tile_cols"] == tile_cols and cfg["order"] == order
    else:
        assert all(x > 0 for x in cfg["tuned_ms"]), cfg
    assert t["bse"] > 0 and t["iteration"] >= t["bse"]
    assert np.all(np.isfinite(d)) and np.all(d > 0)
    # the grouped launch may use another tile width than the members alone (another order of
    # the FP32 sums), so the two agree to the format's accuracy, not to the bit
    tol, tol_phi = PLANE[precision]
    for p, a, m in zip(MEMBERS, alone, mem):
        assert rel(m.sigma(), a.sigma()) < tol, p
        assert rel(all_phi(m, p), all_phi(a, p)) < tol_phi, p
        assert rel(m.chi(1), a.chi(1)) < tol, p
    for s in alone + mem:
        s.close()


@pytest.mark.parametrize("precision", list(PLANE))
def test_batch_large_member_keeps_its_own_products(precision):
    """A member with n >= 512 runs its products in its own launch inside the batch graph (the
    grouped launch holds only the small members); every member still follows its own iteration,
    and a batch of large members only has no grouped launch to tune."""
    from paper_1510_03330_gb300.binding import Batch, Solver

    big = Params("square", beta=2.0, U=1.0, mu=0.0, L=4, n_nu=32, n_Omega=2)  # n = 512
    members = [MEMBERS[1], big, MEMBERS[3]]
    iters = 7
    alone = [Solver(p, precision=precision) for p in members]
    for s in alone:
        s.iterate(iters)
    mem = [Solver(p, precision=precision) for p in members]
    with Batch(mem, time_steps=True) as b:
        for _ in range(iters):
            d = b.iterate(1)
        cfg = b.config()
        t = b.times()
    assert cfg["tile_cols"] in (64, 128) and t["bse"] > 0, (cfg, t)
    assert np.all(np.isfinite(d)) and np.all(d > 0)
    tol, tol_phi = PLANE[precision]
    for p, a, m in zip(members, alone, mem):
        assert rel(m.sigma(), a.sigma()) < tol, p
        assert rel(all_phi(m, p), all_phi(a, p)) < tol_phi, p
    with Batch([mem[1]]) as b:
        b.iterate(2)
        assert b.config()["tile_cols"] == -1
    alone[1].iterate(2)
    assert rel(mem[1].sigma(), alone[1].sigma()) < tol
    for s in alone + mem:
        s.close()


def test_batch_more_members_than_the_shared_table():
    """65 grouped members: more than the grouped kernel keeps in shared memory (64), so the
    CTAs search the problem table in global memory; members at both ends of the table and
    across the boundary follow their own iteration."""
    from paper_1510_03330_gb300.binding import Batch, Solver

    tol, tol_phi = PLANE[SPLIT_FP16X3]
    members = [MEMBERS[i % 2].with_(U=1.0 + 0.01 * i) for i in range(65)]
    check = [0, 1, 63, 64]
    iters = 7
    alone = [Solver(members[i], precision=SPLIT_FP16X3) for i in check]
    for s in alone:
        s.iterate(iters)
    mem = [Solver(p, precision=SPLIT_FP16X3) for p in members]
    with Batch(mem, tile_cols=128, order=0) as b:
        d = b.iterate(iters)
    assert np.all(np.isfinite(d)) and np.all(d > 0)
    for i, a in zip(check, alone):
        p = members[i]
        assert rel(mem[i].sigma(), a.sigma()) < tol, i
        assert rel(all_phi(mem[i], p), all_phi(a, p)) < tol_phi, i
    for s in alone + mem:
        s.close()


@pytest.mark.parametrize("precision", list(PLANE))
def test_batch_member_matches_oracle(precision):
    from paper_1510_03330_gb300.binding import Batch, Solver

    tol, tol_phi = PLANE[precision]
    p = MEMBERS[1]
    st = O.zero_state(p)
    mem = [Solver(q, precision=precision) for q in MEMBERS]
    with Batch(mem) as b:
        for it in range(3):
            res = O.iterate(p, st)
            st = res.state
            b.iterate(1)
        assert rel(mem[1].sigma(), st.sigma) < tol
        assert rel(all_phi(mem[1], p), st.phi) < tol_phi
        chi = O.susceptibility(res.F, res.X_ph, res.X_pp)
        assert rel(mem[1].chi(1), chi[1]) < tol
    for s in mem:
        s.close()


def test_batch_refusals():
    from paper_1510_03330_gb300.binding import Batch, ParquetError, Solver

    p = MEMBERS[0]
    with Solver(p, precision=FP64) as f, pytest.raises(ParquetError):
        Batch([f])
    with Solver(MEMBERS[1], precision=SPLIT_BF16X3, q_chunk=2) as c, pytest.raises(ParquetError):
        Batch([c])  # several passes per iteration
    with Solver(p, precision=SPLIT_BF16X3) as x, Solver(p, precision=SPLIT_FP16X3) as y, pytest.raises(ParquetError):
        Batch([x, y])  # one operand format per batch
    s = Solver(p, precision=SPLIT_FP16X3)
    b = Batch([s])
    with pytest.raises(ParquetError):
        s.iterate(1)  # the batch owns the iteration
    with pytest.raises(ParquetError):
        Batch([s])    # already in a batch
    b.iterate(2)
    b.close()
    s.iterate(1)      # free again
    s.close()
