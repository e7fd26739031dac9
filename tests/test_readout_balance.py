"""Arithmetic of the balanced forward readout launch, checked on the CPU.

The launch splits U = row_blocks x npair units into G contiguous ranges
[floor(U b / G), floor(U (b + 1) / G)); a row block cut between blocks sums
each segment into the plane given by its position among the row block's
segments, which the device derives from the count of block boundaries at or
below a unit, cnt(v) = ceil((v + 1) G / U), and the host sizes the workspace
with planes = 2 + (npair - 1) // floor(U / G).  These tests enumerate the
segments directly (block by block, unit by unit) and check that the derived
positions are exactly 0 .. nseg - 1 for every row block, that nseg is what
the device computes, and that it never exceeds the host's plane count.
"""
import random

import pytest


def cnt(v, G, U):
    return ((v + 1) * G + U - 1) // U


def segments_direct(rblocks, npair, G):
    """{row block: [(block, first unit, end unit)]} by walking each block's range."""
    U = rblocks * npair
    out = {}
    for b in range(G):
        u, u1 = U * b // G, U * (b + 1) // G
        while u < u1:
            rbk = u // npair
            ue = min(u1, (rbk + 1) * npair)
            out.setdefault(rbk, []).append((b, u, ue))
            u = ue
    return out


def check(rblocks, npair, G):
    U = rblocks * npair
    minblk = U // G
    assert minblk >= 2  # the host uses the balanced launch only then
    planes = 2 + (npair - 1) // minblk
    segs = segments_direct(rblocks, npair, G)
    assert sorted(segs) == list(range(rblocks))
    covered = 0
    for rbk, ss in segs.items():
        rs, re = rbk * npair, (rbk + 1) * npair
        nseg_dev = 1 + cnt(re - 1, G, U) - cnt(rs, G, U)
        assert nseg_dev == len(ss) <= planes
        ords = [cnt(u, G, U) - cnt(rs, G, U) for _, u, _ in ss]
        assert ords == list(range(len(ss)))
        assert ss[0][1] == rs and ss[-1][2] == re
        assert all(a[2] == b[1] for a, b in zip(ss, ss[1:]))  # contiguous, no unit twice
        covered += sum(e - u for _, u, e in ss)
    assert covered == U


@pytest.mark.parametrize("rblocks,npair,G", [(256, 16, 304), (192, 4, 304), (256, 16, 456), (128, 32, 152),
                                             (1000, 3, 608), (17, 40, 304)])
def test_balanced_segments_named_workloads(rblocks, npair, G):
    if rblocks * npair < 2 * G:
        pytest.skip("the host keeps the grid launch below two units per block")
    check(rblocks, npair, G)


def test_balanced_segments_random():
    rng = random.Random(7)
    n = 0
    while n < 400:
        G = rng.randint(1, 700)
        npair = rng.randint(1, 40)
        rblocks = rng.randint(1, 4 * G)
        if rblocks * npair < 2 * G:
            continue
        check(rblocks, npair, G)
        n += 1


def test_plane_count_2d256():
    """256 rows, 16 coil pairs, 304 resident blocks: three planes."""
    U, G = 256 * 16, 304
    assert 2 + 15 // (U // G) == 3
    segs = segments_direct(256, 16, G)
    assert max(len(v) for v in segs.values()) == 3
