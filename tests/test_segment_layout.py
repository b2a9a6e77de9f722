"""Layout of the parallel-in-y slab substitution (hz_segment_layout; host
logic, no GPU): the segments tile both elimination chains of the twisted block
LU, the groups of the two-level carries tile each half's segments, and the
carry equations the kernels use (in-group carries from a zero group start,
group boundary chains through in-group prefix products, one fix-up product per
segment start) reproduce the sequential segment carries on that layout."""

import math

import numpy as np
import pytest

import paper_1412_0464_gb300 as hz

CASES = [(ny, P, cap) for ny in (3, 4, 5, 7, 10, 33, 64, 101, 219, 300, 1039, 2059)
         for P, cap in ((0, 304), (0, 152), (2, 304), (5, 304), (24, 304), (300, 304))
         if P <= ny - 1]


@pytest.fixture(scope="module", autouse=True)
def _built():
    hz.build()


@pytest.mark.parametrize("ny,P,cap", CASES)
def test_segments_tile_both_chains(ny, P, cap):
    lay = hz.segment_layout(ny, P, cap)
    mid, S0, seg = lay["mid"], lay["S0"], lay["seg"]
    assert mid == (ny - 1) // 2
    assert lay["P"] == len(seg) and 1 <= S0 < lay["P"]
    if P == 0:
        assert lay["P"] <= max(cap, 2) and lay["P"] <= ny - 1
        want = min(2 * round(ny ** (2.0 / 3.0)), max(cap, 2), ny - 1)
        assert abs(lay["P"] - want) <= 1
    # top chain: rows 0 .. mid-1 upwards; bottom chain: rows ny-1 .. mid+1 downwards
    rows = 0
    for q in range(S0):
        first, n, d, _ = seg[q]
        assert d == 1 and n >= 1 and first == rows
        rows += n
    assert rows == mid
    rows = ny - 1
    for q in range(S0, lay["P"]):
        first, n, d, _ = seg[q]
        assert d == -1 and n >= 1 and first == rows
        rows -= n
    assert rows == mid
    # segment lengths within a chain differ by at most one
    for sl in (seg[:S0, 1], seg[S0:, 1]):
        assert sl.max() - sl.min() <= 1


@pytest.mark.parametrize("ny,P,cap", CASES)
def test_groups_tile_each_half(ny, P, cap):
    lay = hz.segment_layout(ny, P, cap)
    S0, Pn, G0, NG, seg, grp = lay["S0"], lay["P"], lay["G0"], lay["NG"], lay["seg"], lay["grp"]
    assert NG == len(grp) and 1 <= G0 < NG
    for half, (s_first, nh, g_first, ng) in enumerate(((0, S0, 0, G0), (S0, Pn - S0, G0, NG - G0))):
        assert ng == max(1, min(nh, round(math.sqrt(nh))))
        nxt = s_first
        sizes = []
        for c in range(ng):
            lo, hi, h, idx = grp[g_first + c]
            assert (lo, h, idx) == (nxt, half, c) and hi >= lo
            assert all(seg[q, 3] == g_first + c for q in range(lo, hi + 1))
            sizes.append(hi - lo + 1)
            nxt = hi + 1
        assert nxt == s_first + nh
        assert max(sizes) - min(sizes) <= 1


@pytest.mark.parametrize("ny,P", [(33, 0), (101, 0), (219, 24), (1039, 0), (2059, 0), (300, 300)])
def test_two_level_carries_reproduce_the_sequential_carries(ny, P):
    """Forward carry Y_s = yhat_s + Phi_s Y_{s-1} (first segment of a half: its
    own yhat) and backward carry X_s = xhat_s + Psi_s X_{s+1} (last segment of
    a half: from x_m) along each half, with random W x W transfer matrices."""
    assert _carry_mismatches(ny, P, planted=False) == 0


@pytest.mark.parametrize("ny,P", [(101, 0), (1039, 0)])
def test_planted_boundary_mistake_is_caught(ny, P):
    """The check is not vacuous: a fix-up that reads the wrong group boundary
    (the segment's own group instead of the previous one) fails it."""
    assert _carry_mismatches(ny, P, planted=True) > 0


def _carry_mismatches(ny, P, planted):
    lay = hz.segment_layout(ny, P, 304)
    Pn, S0, G0, NG, seg, grp = lay["P"], lay["S0"], lay["G0"], lay["NG"], lay["seg"], lay["grp"]
    rng = np.random.default_rng(ny + Pn)
    W = 3
    Phi = rng.standard_normal((Pn, W, W)) * 0.5
    Psi = rng.standard_normal((Pn, W, W)) * 0.5
    yhat = rng.standard_normal((Pn, W))
    xhat = rng.standard_normal((Pn, W))
    xm = rng.standard_normal(W)
    halves = ((0, S0), (S0, Pn - S0))
    Y, X = np.zeros((Pn, W)), np.zeros((Pn, W))
    for s_first, nh in halves:
        v = yhat[s_first]
        Y[s_first] = v
        for q in range(s_first + 1, s_first + nh):
            v = yhat[q] + Phi[q] @ v
            Y[q] = v
        v = xm
        for q in range(s_first + nh - 1, s_first - 1, -1):
            v = xhat[q] + Psi[q] @ v
            X[q] = v
    # in-group prefix products (forward for groups after the first of a half, backward for all)
    PhiP, PsiP = {}, {}
    for lo, hi, half, c in grp:
        if c != 0:
            M = Phi[lo]
            PhiP[lo] = M
            for q in range(lo + 1, hi + 1):
                M = Phi[q] @ M
                PhiP[q] = M
        M = Psi[hi]
        PsiP[hi] = M
        for q in range(hi - 1, lo - 1, -1):
            M = Psi[q] @ M
            PsiP[q] = M
    # in-group carries from a zero group start
    lf, lb = yhat.copy(), xhat.copy()
    for lo, hi, _, _ in grp:
        for q in range(lo + 1, hi + 1):
            lf[q] = yhat[q] + Phi[q] @ lf[q - 1]
        for q in range(hi - 1, lo - 1, -1):
            lb[q] = xhat[q] + Psi[q] @ lb[q + 1]
    # group boundary chains: true group ends (forward) and starts (backward)
    Tf, Tb = np.zeros((NG, W)), np.zeros((NG, W))
    for half, (g_first, ng) in enumerate(((0, G0), (G0, NG - G0))):
        v = lf[grp[g_first][1]]
        Tf[g_first] = v
        for g in range(g_first + 1, g_first + ng):
            q = grp[g][1]
            v = lf[q] + PhiP[q] @ v
            Tf[g] = v
        v = xm
        for g in range(g_first + ng - 1, g_first - 1, -1):
            q = grp[g][0]
            v = lb[q] + PsiP[q] @ v
            Tb[g] = v
    # the meeting row reads the true ends of both halves' last groups
    bad = int(not (np.allclose(Tf[G0 - 1], Y[S0 - 1]) and np.allclose(Tf[NG - 1], Y[Pn - 1])))
    # fix-up of every segment start
    prev = 0 if planted else 1
    for s in range(Pn):
        if s not in (0, S0):               # forward re-run of segment s starts from Y_{s-1}
            q = s - 1
            g = seg[q, 3]
            first_group = g == (G0 if s >= S0 else 0)
            start = lf[q] if first_group else lf[q] + PhiP[q] @ Tf[g - prev]
            bad += int(not np.allclose(start, Y[q]))
        if s not in (S0 - 1, Pn - 1):      # backward re-run of segment s starts from X_{s+1}
            q = s + 1
            g = seg[q, 3]
            last_group = g == (NG - 1 if s >= S0 else G0 - 1)
            vin = xm if last_group else Tb[g + prev]
            bad += int(not np.allclose(lb[q] + PsiP[q] @ vin, X[q]))
    return bad


def test_layout_rejects_bad_arguments():
    import ctypes
    L = hz.lib()
    c = [ctypes.c_int() for _ in range(5)]
    refs = [ctypes.byref(x) for x in c]
    assert L.hz_segment_layout(2, 0, 304, *refs, None, 0, None, 0) == hz.HZ_EINVAL   # ny < 3
    assert L.hz_segment_layout(100, 0, 304, None, *refs[1:], None, 0, None, 0) == hz.HZ_EINVAL
    seg = np.zeros((4, 4), dtype=np.int32)
    assert L.hz_segment_layout(1039, 0, 304, *refs, seg.ctypes.data, 4, None, 0) == hz.HZ_EINVAL
    assert c[1].value > 4                                               # the counts are written
