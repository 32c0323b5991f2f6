"""Host analysis of the ILU(0) segment sweeps (CPU, no GPU needed): the
segments, hand-out orders and coupling counts that ms_plan_segments returns
against a plain restatement of their definition, the invariants the sweeps
rely on (chains inside a segment, no other coupling inside it, dependencies
handed out first), and the algebra of the sweeps: segments in the plan's
orders, each chain solved by a 32-lane scan of affine maps, reproduce the
oracle's ILU(0) application."""
import numpy as np
import pytest

import oracle as O
from paper_2001_01624_gb300 import geomodel as G


@pytest.fixture(scope="module")
def b():
    from paper_2001_01624_gb300 import build
    build.build()
    from paper_2001_01624_gb300 import binding
    return binding


def _rows(rowptr, col):
    n = len(rowptr) - 1
    return [set(int(k) for k in col[rowptr[i]:rowptr[i + 1]]) - {i} for i in range(n)]


def _reference(rows, max_len):
    """Segments, orders, kg and width written out from their definition."""
    n = len(rows)
    off, start = [0], 0
    for i in range(1, n):
        ok = i - start < max_len and (i - 1) in rows[i] and i in rows[i - 1]
        ok = ok and not any(start <= k <= i - 2 for k in rows[i])            # row i to an earlier row of the run
        ok = ok and not any(i in rows[r] for r in range(start, i - 1))        # an earlier row of the run to row i
        if not ok:
            off.append(i)
            start = i
    off.append(n)
    ns = len(off) - 1
    sid = np.repeat(np.arange(ns), np.diff(off))
    lf, lb = [0] * ns, [0] * ns
    kgf = kgb = 0
    for S in range(ns):
        for i in range(off[S], off[S + 1]):
            low = [k for k in rows[i] if k < off[S]]
            kgf = max(kgf, len(low))
            kgb = max(kgb, sum(1 for k in rows[i] if k >= off[S + 1]))
            for k in low:
                lf[S] = max(lf[S], lf[sid[k]] + 1)
    for S in reversed(range(ns)):
        for i in range(off[S], off[S + 1]):
            for k in rows[i]:
                if k >= off[S + 1]:
                    lb[S] = max(lb[S], lb[sid[k]] + 1)
    fwd = sorted(range(ns), key=lambda S: (lf[S], S))
    bwd = sorted(range(ns), key=lambda S: (lb[S], -S))
    width = max(max(np.bincount(lf)), max(np.bincount(lb)))
    return np.array(off), np.array(fwd), np.array(bwd), (kgf, kgb), int(width)


def _check_invariants(rows, plan, max_len):
    off = plan["seg_off"]
    n = len(rows)
    assert off[0] == 0 and off[-1] == n and np.all(np.diff(off) >= 1) and np.all(np.diff(off) <= max_len)
    ns = len(off) - 1
    sid = np.repeat(np.arange(ns), np.diff(off))
    for S in range(ns):
        a, e = off[S], off[S + 1]
        for i in range(a, e):
            if i > a:                                          # the chain, both ways
                assert (i - 1) in rows[i] and i in rows[i - 1]
            for k in rows[i]:                                  # nothing else inside the segment
                assert not (a <= k < e and abs(k - i) >= 2)
    for order, lower in ((plan["order_fwd"], True), (plan["order_bwd"], False)):
        assert sorted(order) == list(range(ns))
        pos = np.empty(ns, int)
        pos[order] = np.arange(ns)
        for S in range(ns):
            for i in range(off[S], off[S + 1]):
                for k in rows[i]:
                    if (k < off[S]) if lower else (k >= off[S + 1]):
                        assert pos[sid[k]] < pos[S]            # dependencies are handed out first


def _compare(b, rowptr, col, max_len=256):
    rows = _rows(rowptr, col)
    plan = b.ms_plan_segments(rowptr, col, max_len)
    off, fwd, bwd, kg, width = _reference(rows, max_len)
    np.testing.assert_array_equal(plan["seg_off"], off)
    np.testing.assert_array_equal(plan["order_fwd"], fwd)
    np.testing.assert_array_equal(plan["order_bwd"], bwd)
    assert plan["kg"] == kg and plan["width"] == width
    _check_invariants(rows, plan, max_len)
    return plan


@pytest.mark.parametrize("shape", [(18, 14, 7), (41, 23, 9), (5, 3, 2)])
def test_faulted_grids(b, shape):
    gm = G.faulted(*shape, seed=9, n_fault_x=1, n_fault_y=1, block=(4, 3, 2))
    A = O.assemble_tpfa(gm.grid, gm.perm).A
    plan = _compare(b, A.rowptr, A.col)
    assert 1 < len(plan["seg_off"]) - 1 < A.n                   # lines cut by faults and inactive cells


@pytest.mark.parametrize("max_len", [256, 7, 1])
def test_long_lines_are_cut(b, max_len):
    gm = G.lognormal_box(700, 3, 2, seed=4, block=(50, 3, 2))
    act = np.ones(gm.grid.N, np.uint8)
    act[5] = 0
    gm.grid.active = act
    A = O.assemble_tpfa(gm.grid, gm.perm).A
    plan = _compare(b, A.rowptr, A.col, max_len)
    lens = np.diff(plan["seg_off"])
    assert lens.max() == min(max_len, 694)
    if max_len == 1:
        assert len(lens) == A.n


def test_couplings_inside_a_line_and_one_way_couplings(b):
    """A chain of 300 rows with random extra couplings (some both ways, some
    one way, some repeated, the diagonal listed, columns unsorted)."""
    rng = np.random.default_rng(5)
    n = 300
    rows = [set() for _ in range(n)]
    for i in range(1, n):
        if rng.random() < 0.95:
            rows[i].add(i - 1)
            rows[i - 1].add(i)
    for _ in range(40):
        i, k = rng.integers(0, n, 2)
        if abs(i - k) >= 2:
            rows[i].add(int(k))
            if rng.random() < 0.5:
                rows[k].add(int(i))
    rowptr, col = [0], []
    for i in range(n):
        c = list(rows[i]) + [i] + list(rows[i])[:1]
        rng.shuffle(c)
        col += c
        rowptr.append(len(col))
    _compare(b, np.array(rowptr), np.array(col))


def test_single_row_and_errors(b):
    plan = b.ms_plan_segments(np.array([0, 1]), np.array([0]))
    assert list(plan["seg_off"]) == [0, 1] and plan["kg"] == (0, 0) and plan["width"] == 1
    rp, cl = np.array([0, 2, 4]), np.array([0, 1, 0, 1])
    for bad in (dict(max_len=0), dict(max_len=257)):
        with pytest.raises(b.MsError):
            b.ms_plan_segments(rp, cl, **bad)
    with pytest.raises(b.MsError):
        b.ms_plan_segments(rp, np.array([0, 1, 0, 2]))                 # column out of range
    with pytest.raises(b.MsError):
        b.ms_plan_segments(np.array([0, 2, 1]), cl)                    # decreasing rowptr


def _lane_scan(a, B, bwd):
    """One warp's solve of the chain x_p = B_p + a_p x_(p-1) (bwd: x_(p+1)):
    each of 32 lanes composes the affine maps of its run of rows, the
    compositions are scanned across the lanes (distances 1, 2, 4, 8, 16), and
    each lane applies its scanned input."""
    L = len(a)
    C = (L + 31) // 32
    A, Bc = np.ones(32), np.zeros(32)
    runs = [range(l * C, min(l * C + C, L)) for l in range(32)]
    for l in range(32):
        for p in (reversed(runs[l]) if bwd else runs[l]):
            Bc[l] = a[p] * Bc[l] + B[p]
            A[l] = a[p] * A[l]
    d = 1
    while d < 32:
        An, Bn = A.copy(), Bc.copy()
        for l in range(32):
            src = l + d if bwd else l - d
            if 0 <= src < 32:
                Bn[l] = A[l] * Bc[src] + Bc[l]
                An[l] = A[l] * A[src]
        A, Bc, d = An, Bn, 2 * d
    x = np.zeros(L)
    for l in range(32):
        src = l + 1 if bwd else l - 1
        v = Bc[src] if 0 <= src < 32 else 0.0
        for p in (reversed(runs[l]) if bwd else runs[l]):
            v = a[p] * v + B[p]
            x[p] = v
    return x


@pytest.mark.parametrize("case", ["faulted", "long_lines"])
def test_segment_scans_solve_the_ilu_triangles(b, case):
    """The segment plan and the chain scans reproduce the oracle's ILU(0)
    application (Sec. 6.4 "Smooth": L y = r, then U z = y): segments taken
    in the plan's hand-out orders, couplings leaving a segment gathered from
    segments already solved, each chain solved by the lane scan."""
    if case == "faulted":
        gm = G.faulted(41, 23, 9, seed=9, n_fault_x=1, n_fault_y=1, block=(4, 3, 2))
        max_len = 256
    else:
        gm = G.lognormal_box(700, 3, 2, seed=4, block=(50, 3, 2))
        act = np.ones(gm.grid.N, np.uint8)
        act[5] = 0
        gm.grid.active = act
        max_len = 64
    Ap, _ = O.pin(O.assemble_tpfa(gm.grid, gm.perm).A, None, 0)
    lu = O.ilu0(Ap)
    r = np.random.default_rng(3).standard_normal(Ap.n)
    plan = b.ms_plan_segments(Ap.rowptr, Ap.col, max_len)
    off = plan["seg_off"]
    row = [(Ap.col[Ap.rowptr[i]:Ap.rowptr[i + 1]], lu[Ap.rowptr[i]:Ap.rowptr[i + 1]]) for i in range(Ap.n)]
    d = np.array([v[c == i][0] for i, (c, v) in enumerate(row)])
    y = np.full(Ap.n, np.nan)
    for S in plan["order_fwd"]:
        a0, e0 = off[S], off[S + 1]
        a, B = np.zeros(e0 - a0), np.zeros(e0 - a0)
        for p, i in enumerate(range(a0, e0)):
            s = r[i]
            for k, v in zip(*row[i]):
                if k == i - 1 and i > a0:
                    a[p] = -v
                elif k < a0:
                    assert not np.isnan(y[k])          # handed out before
                    s -= v * y[k]
            B[p] = s
        y[a0:e0] = _lane_scan(a, B, bwd=False)
    z = np.full(Ap.n, np.nan)
    for S in plan["order_bwd"]:
        a0, e0 = off[S], off[S + 1]
        a, B = np.zeros(e0 - a0), np.zeros(e0 - a0)
        for p, i in enumerate(range(a0, e0)):
            s = y[i]
            for k, v in zip(*row[i]):
                if k == i + 1 and i + 1 < e0:
                    a[p] = -v / d[i]
                elif k >= e0:
                    assert not np.isnan(z[k])
                    s -= v * z[k]
            B[p] = s / d[i]
        z[a0:e0] = _lane_scan(a, B, bwd=True)
    zr = O.ilu0_apply(Ap, lu, r)
    assert np.abs(z - zr).max() <= 1e-12 * np.abs(zr).max()
