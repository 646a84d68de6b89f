"""Host logic of the tensor-core contractions (CPU): the work-unit planning
of tomo_plan_tc_units on the tile ranges of the c2 and paper-geometry
workloads and on edge cases, checked against the properties the kernels rely
on: every tile's reduction range covered exactly once, in chunk order; every
unit a multiple of the slice width and at most the table size; every CTA's
share within the equal share; empty tiles one zero-length unit each, spread."""
import numpy as np
import pytest

import oracle
import paper_2404_02844_gb300 as tomo
import workloads

TILE = 128


def fwd_adj_ranges(M, lam, band_k=10.0):
    pr = oracle.Problem(M, 2, lam, band_k, 0.0, store_F=False)
    lo, hi = pr.bands()
    D = lam.shape[0]
    fst, fen = [], []
    for t in range((D + TILE - 1) // TILE):
        a, b = lo[TILE * t:TILE * t + TILE].min(), hi[TILE * t:TILE * t + TILE].max()
        fst.append((a // 64) * 64)
        fen.append(((b + 1 + 63) // 64) * 64)
    ast, aen = [], []
    for t in range((M + TILE - 1) // TILE):
        i0, i1 = TILE * t, min(M, TILE * t + TILE) - 1
        dmin = np.searchsorted(hi, i0, side="left")
        dmax = np.searchsorted(lo, i1, side="right") - 1
        if dmin > dmax:
            ast.append(0)
            aen.append(0)
        else:
            ast.append((dmin // 64) * 64)
            aen.append(((dmax + 1 + 63) // 64) * 64)
    return (np.array(fst), np.array(fen)), (np.array(ast), np.array(aen))


def check(st, en, ctas, align=64, max_unit=1024):
    units, cta_first, nsplit = tomo.plan_tc_units(st, en, align, max_unit, ctas)
    tiles = st.shape[0]
    W = int(np.sum(np.maximum(en - st, 0)))
    share = max(align, -(-(-(-W // ctas)) // align) * align)
    n_ctas = cta_first.shape[0] - 1
    assert 1 <= n_ctas <= ctas
    assert cta_first[0] == 0 and cta_first[-1] == units.shape[0]
    assert np.all(np.diff(cta_first) >= 1) or W == 0
    # coverage per tile, in chunk order
    for t in range(tiles):
        u = units[units[:, 0] == t]
        assert u.shape[0] == nsplit[t]
        assert np.array_equal(np.sort(u[:, 1]), np.arange(nsplit[t]))
        u = u[np.argsort(u[:, 1])]
        if en[t] <= st[t]:
            assert nsplit[t] == 1 and u[0, 2] == 0 and u[0, 3] == 0
            continue
        assert u[0, 2] == st[t] and u[-1, 3] == en[t]
        assert np.all(u[1:, 2] == u[:-1, 3])
        lens = u[:, 3] - u[:, 2]
        assert np.all(lens > 0) and np.all(lens % align == 0) and np.all(lens <= max_unit)
    # shares
    for c in range(n_ctas):
        u = units[cta_first[c]:cta_first[c + 1]]
        assert int(np.sum(u[:, 3] - u[:, 2])) <= share
    # empty tiles spread: no CTA holds more than its fair part plus one
    n_empty = int(np.sum(en <= st))
    if n_empty:
        per = [int(np.sum((units[cta_first[c]:cta_first[c + 1], 3] == 0) &
                          (units[cta_first[c]:cta_first[c + 1], 2] == 0))) for c in range(n_ctas)]
        assert max(per) <= -(-n_empty // n_ctas) + 1
    return units, cta_first, nsplit, share


def test_c2_schedules():
    w = workloads.config_c2()
    (fs, fe), (as_, ae) = fwd_adj_ranges(w.M, w.lam)
    u, cf, ns, share = check(fs, fe, 152)
    assert share == 384 and cf.shape[0] - 1 == 140 and ns.sum() == u.shape[0]
    u, cf, ns, share = check(as_, ae, 152)
    assert cf.shape[0] - 1 == 147 and int((ae <= as_).sum()) == 4


def test_paper_geometry_schedules():
    lam = workloads.quadratic_intensities(workloads.F2_D)
    (fs, fe), (as_, ae) = fwd_adj_ranges(workloads.F2_M, lam)
    u, cf, ns, share = check(fs, fe, 76)
    assert ns.max() > 200              # long forward unions cut at the table size
    check(as_, ae, 76)


@pytest.mark.parametrize("ctas", [1, 3, 152, 10000])
def test_edge_cases(ctas):
    st = np.array([0, 64, 0, 128, 0], dtype=np.int64)
    en = np.array([640, 64, 0, 4096, 64], dtype=np.int64)     # two empty tiles
    check(st, en, ctas)
    # all tiles empty
    check(np.zeros(3, np.int64), np.zeros(3, np.int64), ctas)


def test_invalid_arguments():
    with pytest.raises(tomo.TomoError):
        tomo.plan_tc_units(np.array([0]), np.array([100]), align=64)       # not a multiple of 64
    with pytest.raises(tomo.TomoError):
        tomo.plan_tc_units(np.array([0]), np.array([128]), align=64, max_unit=100)
