"""The connection-row scan with chunk masks (refine.cu `k_dense_best`),
restated lane by lane on the host: reading only the chunks a row's mask
marks gives the same proposal as reading the whole row, for any mask that
covers every nonzero entry, in both proposal variants.

A warp scans a row of K entries as int4 groups; lane l takes groups l, l+32,
... (whole row) or, chunk by chunk in increasing order, groups q0 + l, q0 +
l + 32, ... of each marked chunk of cw / 4 groups. Each lane keeps the first
best candidate it meets (larger gain; in the variant the first adjacent
partition seeds it), then the lanes reduce by (larger gain, lower id). An
entry outside every marked chunk is 0, and a partition with conn 0 is never
taken, so the two scans see the same candidates, each lane in increasing
partition order.
"""
import numpy as np
import pytest


def _better(s1, m1, s2, m2):
    if m1 < 0:
        return False
    if m2 < 0:
        return True
    return s1 > s2 or (s1 == s2 and m1 < m2)


def _lane_visit(bs, bk, p, c, T, ok, nonpos):
    g = c - T
    if (g > bs or (nonpos and bk < 0 and c > 0)) and c > 0 and ok:
        return g, p
    return bs, bk


def _reduce(lanes):
    bs, bk = lanes[0]
    for s2, m2 in lanes[1:]:
        if _better(s2, m2, bs, bk):
            bs, bk = s2, m2
    return bs, bk


def scan_full(C, K, T, ok, nonpos):
    lanes = []
    nq = (K + 3) // 4
    for lane in range(32):
        bs, bk = 0, -1
        for q in range(lane, nq, 32):
            for u in range(4):
                p = 4 * q + u
                if p < K:
                    bs, bk = _lane_visit(bs, bk, p, C[p], T, ok[p], nonpos)
        lanes.append((bs, bk))
    return _reduce(lanes)


def scan_chunks(C, K, T, ok, nonpos, mask, cw):
    lanes = []
    nq = (K + 3) // 4
    for lane in range(32):
        bs, bk = 0, -1
        m = mask
        while m:
            c = (m & -m).bit_length() - 1
            m &= m - 1
            q0 = c * (cw // 4)
            q1 = min(q0 + cw // 4, nq)
            for q in range(q0 + lane, q1, 32):
                for u in range(4):
                    p = 4 * q + u
                    if p < K:
                        bs, bk = _lane_visit(bs, bk, p, C[p], T, ok[p], nonpos)
        lanes.append((bs, bk))
    return _reduce(lanes)


def chunk_width(Kp):
    cw = 32
    while cw * 64 < Kp:
        cw <<= 1
    return cw


@pytest.mark.parametrize("K", [1, 5, 31, 64, 200, 1000, 4536, 9011])
@pytest.mark.parametrize("nonpos", [0, 1])
def test_chunked_scan_equals_full_scan(K, nonpos):
    rng = np.random.Generator(np.random.PCG64(K * 2 + nonpos))
    Kp = (K + 3) & ~3
    cw = chunk_width(Kp)
    assert (Kp + cw - 1) // cw <= 64
    for trial in range(40):
        C = np.zeros(Kp, np.int64)
        # a few clusters of adjacent partitions, gains with ties
        for _ in range(int(rng.integers(0, 4))):
            a = int(rng.integers(0, K))
            b = min(K, a + int(rng.integers(1, 12)))
            C[a:b] = rng.integers(0, 6, size=b - a)
        T = int(rng.integers(-2, 5))
        ok = rng.random(Kp) < 0.8
        nz = {int(p) // cw for p in np.flatnonzero(C[:K] > 0)}
        extra = {int(x) for x in rng.integers(0, (Kp + cw - 1) // cw, size=int(rng.integers(0, 3)))}
        mask = 0
        for c in nz | extra:
            mask |= 1 << c
        assert scan_chunks(C, K, T, ok, nonpos, mask, cw) == scan_full(C, K, T, ok, nonpos)


def test_chunk_width_and_bits():
    for Kp in [4, 128, 2048, 2052, 4096, 4536, 9012, 1 << 16]:
        cw = chunk_width(Kp)
        assert cw >= 32 and cw & (cw - 1) == 0 and cw % 4 == 0
        assert (Kp - 1) // cw < 64                    # every partition's bit fits a 64-bit mask
        assert cw == 32 or (cw // 2) * 64 < Kp        # the smallest such width
