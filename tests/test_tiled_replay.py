"""CPU replay of the tiled BF16x3 assembly's index arithmetic (no GPU): for small lattices it
walks every CTA, step and thread of the kernel's schedule -- the gathers of each step, the
d/m stores, and the s/t stores with the per-thread delay line of the single-pass kernel --
and checks that every source and destination lies inside its buffer and that every output
element (r, Q, k, k') is written exactly once.  The geometry (block count G, rows per sweep,
tile strides, shared-memory budget) restates the launch geometry of the kernel; this is the
check that was run on the CPU before the kernel's first launch."""
import numpy as np
import pytest

TT = 256
SMEM_TWO_PER_SM = (228 * 1024) // 2 - 1024 - 4480


def geometry(L, nnu, nom, fused):
    def a128(x):
        return (x + 127) // 128 * 128

    def geo(G):
        hb, upr = nnu // 4, G * nnu // 4
        if upr > TT:
            return None
        sweeps = (nom + TT // upr - 1) // (TT // upr)
        rows = (nom + sweeps - 1) // sweeps
        if fused and rows < nom:
            return None
        if nom > 256 or nnu + 6 > 256:
            return None
        sh = 2 if G > 1 else 0        # R block a starts a * sh words into its rows
        RS = nnu + 2 * max(G - 1, 1)  # R rows = TMA box width
        RA = (nom * RS + 15) // 16 * 16
        BW = nnu + 2
        PW = G * BW
        PPW = G * nnu + 2  # P tile: adjacent blocks, padded rows
        sm = a128(2 * G * RA * 8)
        sm = a128(sm + 2 * nom * PPW * 8)
        sm = a128(sm + 2 * nom * PW * 8)
        sm = a128(sm + 2 * G * nom * 8)
        if fused:
            sm = a128(sm + 16 * 8 * hb * rows * (G * (G - 1) // 2))
        return dict(G=G, hb=hb, upr=upr, rows=rows, RS=RS, RA=RA, BW=BW, PW=PW, PPW=PPW, sh=sh, smem=sm + 8)

    cands = [c for c in (geo(G) for G in (4, 2, 1) if L % G == 0) if c and c["smem"] <= 200 * 1024]
    if not cands:
        return None
    two = [c for c in cands if c["smem"] <= SMEM_TWO_PER_SM]
    return (two or cands)[0]


def replay(L, nnu, nom, fused, q_chunk=None):
    nk = L * L
    n, nQ = nk * nnu, nk * nom
    ld = (n + 7) // 8 * 8

    def kadd(a, b):
        return ((a // L + b // L) % L) * L + (a % L + b % L) % L

    def kneg(a):
        return ((L - a // L) % L) * L + (L - a % L) % L

    def ksub(a, b):
        return kadd(a, kneg(b))

    c = geometry(L, nnu, nom, fused)
    assert c is not None
    G, hb, upr, rows = c["G"], c["hb"], c["upr"], c["rows"]
    RS, RA, BW, PW, PPW, sh = c["RS"], c["RA"], c["BW"], c["PW"], c["PPW"], c["sh"]
    assert PPW <= PW and PPW % 2 == 0 and RS % 2 == 0 and RS % 4 == 2 and RA % 16 == 0
    ring_n = hb * rows
    ring_sz = 8 * ring_n * (G * (G - 1) // 2)
    chan = nQ * n * n
    passes = [(0, nk)] if fused else [(qb, min(q_chunk, nk - qb)) for qb in range(0, nk, q_chunk)]
    for qb, nq in passes:
        ochan = nq * nom * n * ld
        seen = np.zeros((4, nq * nom, n, n), dtype=np.int32)
        for k in range(n):
            ik = k // nnu
            for j in range(nk // G):
                p0 = j * G
                ring = {}
                for step in range(nk if fused else 2 * nq):
                    do_dm = fused or step % 2 == 0
                    do_st = fused or step % 2 == 1
                    qt = step if fused else qb + step // 2
                    for b in range(G):  # the step table and the gathers of block b
                        pb = p0 + b
                        qs_ = qt if do_dm else ksub(ksub(qt, ik), pb)
                        xg = kadd(kadd(ik, pb), qt) if do_dm else qt
                        for x in range(2):
                            # R: one TMA box (x0 .. x0 + RS, row k, slabs z .. z + nom) of the
                            # channel-x Phi viewed as [4 nQ][n][n]; its Nnu columns start b*sh in
                            x0 = kadd(ik, qs_) * nnu - b * sh
                            z = x * nQ + ksub(pb, ik) * nom
                            assert x0 % 2 == 0  # 16-byte aligned innermost coordinate
                            assert 0 <= x0 + b * sh and x0 + b * sh + nnu <= n  # the wanted columns
                            assert 0 <= z and z + nom <= 4 * nQ and 0 <= k < n
                            dst = (x * G + b) * RA
                            assert dst % 16 == 0 and dst + nom * RS <= 2 * G * RA  # 128-byte aligned
                            assert b * sh + nnu <= RS
                        for mt in range(nom):
                            for x in range(2):
                                # S: one copy per block; P: one copy per block on s/t steps
                                src = (x + 2) * chan + ((xg * nom + mt) * n + k) * n + pb * nnu
                                assert src + nnu <= 4 * chan and src % 2 == 0
                                dst = (x * nom + mt) * PW + b * BW
                                assert dst % 2 == 0 and dst + nnu <= 2 * nom * PW
                                if not do_dm:
                                    src = x * chan + ((qs_ * nom + mt) * n + k) * n + pb * nnu
                                    assert src + nnu <= 4 * chan and src % 2 == 0
                                    dst = (x * nom + mt) * PPW + b * nnu
                                    assert dst % 2 == 0 and dst + nnu <= (x * nom + mt + 1) * PPW
                    if do_dm:
                        # P on d/m steps: the G blocks of a row share their transfer qt and are
                        # adjacent in Phi and in the tile, so one copy moves the whole row
                        for mt in range(nom):
                            for x in range(2):
                                src = x * chan + ((qt * nom + mt) * n + k) * n + p0 * nnu
                                assert src + G * nnu <= 4 * chan and src % 2 == 0
                                assert p0 * nnu + G * nnu <= n  # within one row of Phi
                                dst = (x * nom + mt) * PPW
                                assert dst % 2 == 0 and dst + G * nnu <= (x * nom + mt + 1) * PPW
                    for tid in range(upr * rows):
                        cu, row0 = tid % upr, tid // upr
                        a = cu // hb
                        col0 = p0 * nnu + 4 * cu
                        assert col0 % 4 == 0 and col0 + 4 <= n
                        for mi in range(row0, nom, rows):
                            if do_dm:
                                Q = qt * nom + mi
                                o = ((Q - qb * nom) * n + k) * ld + col0
                                assert 0 <= o and o + 4 <= ochan
                                seen[0:2, Q - qb * nom, k, col0:col0 + 4] += 1
                            if not do_st:
                                continue
                            Qp = (kadd(kadd(ik, p0 + a), qt) if fused else qt) * nom + mi
                            if not fused:
                                seen[2:4, Qp - qb * nom, k, col0:col0 + 4] += 1
                                continue
                            qy = qt % L
                            slot = 8 * ring_n * (a * (a - 1) // 2) + row0 * hb + cu % hb
                            if a > 0 and qy >= a:  # block a of the row whose block 0 is produced now
                                Qr, cols = ring.pop((tid, qy % a))
                                assert Qr == kadd(kadd(ik, p0), qt) * nom + mi
                                assert slot + 8 * ring_n * (qy % a) + 7 * ring_n < ring_sz
                                seen[2:4, Qr, k, cols:cols + 4] += 1
                            if a == 0 or qy + a >= L:
                                seen[2:4, Qp, k, col0:col0 + 4] += 1
                            else:
                                assert slot + 8 * ring_n * (qy % a) + 7 * ring_n < ring_sz
                                ring[(tid, qy % a)] = (Qp, col0)
                assert not ring
        assert seen.min() == 1 and seen.max() == 1


@pytest.mark.parametrize("L,nnu,nom,fused,q_chunk", [
    (4, 8, 8, True, None),    # G = 4 with the delay line
    (2, 8, 8, True, None),    # G = 2
    (3, 8, 7, True, None),    # G = 1, odd NOmega
    (1, 12, 9, True, None),   # Bethe (one momentum)
    (4, 8, 8, False, 3),      # two-gather passes, ragged last pass
    (2, 24, 24, False, 3),    # Nnu = 24: G chosen by the shared-memory budget, two row sweeps
    (4, 24, 6, True, None),   # 30-word R boxes, 24 threads per row
    (2, 32, 9, True, None),   # Nnu = 32: 34-word R boxes, odd NOmega
])
def test_tiled_schedule_in_bounds_and_exactly_once(L, nnu, nom, fused, q_chunk):
    replay(L, nnu, nom, fused, q_chunk)


def test_bench_block_geometry():
    """The 8x8, Nnu = NOmega = 16 launch: G = 4, one sweep of 16 rows, two CTAs per SM."""
    c = geometry(8, 16, 16, True)
    assert (c["G"], c["rows"], c["upr"]) == (4, 16, 16)
    assert c["smem"] <= SMEM_TWO_PER_SM
    c24 = geometry(8, 24, 24, False)  # the n = 1536 solve, in passes
    assert c24["G"] == 2 and c24["smem"] <= SMEM_TWO_PER_SM
