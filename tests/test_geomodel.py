"""The seeded synthetic inputs follow their stated recipe (CPU): sizes and cell
dimensions, lognormal statistics after re-standardisation, Kz = 0.1 Kx where
stated, binary 1 mD / 1000 mD channels, fault faces replaced by displaced
non-neighbour connections with multipliers in [1e-3, 1], ~8 % inactive cells
with one connected active set, clipped ensemble fields, zero-sum corner
sources, and determinism per seed."""
import numpy as np
import pytest

from paper_2001_01624_gb300 import geomodel as G

MD, FT = G.MD, G.FT


def _lnk(gm):
    return np.log(gm.perm[:, 0] / MD)


def _sources_ok(gm):
    q = gm.q
    assert abs(q.sum()) < 1e-12 and q.max() > 0 and q.min() < 0
    act = gm.grid.active_mask().astype(bool)
    assert np.all(q[~act] == 0)


def test_same_seed_same_model_other_seed_other_model():
    a, b, c = G.config1(0), G.config1(0), G.config1(1)
    assert np.array_equal(a.perm, b.perm) and not np.array_equal(a.perm, c.perm)


def test_config1_lognormal_2d():
    gm = G.config1(0)
    g = gm.grid
    assert (g.nx, g.ny, g.nz) == (60, 220, 1) and np.isclose(g.dx, 20 * FT) and np.isclose(g.dy, 10 * FT)
    z = (_lnk(gm) - np.log(100.0)) / 2.0                       # ln K = ln 100 mD + 2 z, z re-standardised
    assert abs(z.mean()) < 1e-12 and abs(z.std() - 1.0) < 1e-12
    assert np.array_equal(gm.perm[:, 0], gm.perm[:, 1]) and np.array_equal(gm.perm[:, 0], gm.perm[:, 2])
    assert gm.block == (10, 20, 1)
    _sources_ok(gm)


def test_config2_lognormal_top_channels_bottom():
    gm = G.config2(0)
    g = gm.grid
    assert (g.nx, g.ny, g.nz) == (60, 220, 85) and np.isclose(g.dz, 2 * FT) and gm.block == (10, 20, 5)
    k = gm.perm.reshape(85, 220, 60, 3)
    assert np.allclose(k[..., 2], 0.1 * k[..., 0], rtol=1e-15)
    top = np.log(k[:35, ..., 0] / MD)
    z = (top - np.log(100.0)) / 2.0
    assert abs(z.mean()) < 1e-12 and abs(z.std() - 1.0) < 1e-12
    bot = k[35:, ..., 0] / MD
    assert set(np.unique(np.round(bot, 6))) == {1.0, 1000.0}
    fac = gm.facies.reshape(85, 220, 60)
    assert np.array_equal(fac[35:] == 1, np.isclose(bot, 1000.0)) and not fac[:35].any()
    frac = (fac[35:] == 1).mean(axis=(1, 2))                   # 3..6 channels of width 4..8 per layer
    assert frac.min() > 0.03 and frac.max() < 0.9
    _sources_ok(gm)


def _connected(grid):
    from scipy.sparse import coo_matrix
    from scipy.sparse.csgraph import connected_components
    nx, ny, nz = grid.nx, grid.ny, grid.nz
    act = grid.active_mask().astype(bool)
    idx = np.arange(grid.N).reshape(nz, ny, nx)
    a, b = [], []
    for sl_a, sl_b, m in ((idx[:, :, :-1], idx[:, :, 1:], grid.mult_x), (idx[:, :-1, :], idx[:, 1:, :], grid.mult_y),
                          (idx[:-1], idx[1:], grid.mult_z)):
        keep = np.ones(sl_a.size, bool) if m is None else (m > 0)
        a.append(sl_a.ravel()[keep]); b.append(sl_b.ravel()[keep])
    if grid.nnc is not None:
        a.append(grid.nnc[:, 0]); b.append(grid.nnc[:, 1])
    a, b = np.concatenate(a), np.concatenate(b)
    e = act[a] & act[b]
    M = coo_matrix((np.ones(e.sum()), (a[e], b[e])), shape=(grid.N, grid.N))
    _, lab = connected_components(M, directed=False)
    return len(np.unique(lab[act])) == 1


def test_faulted_model():
    gm = G.faulted(60, 40, 12, seed=2, n_fault_x=2, n_fault_y=1, block=(6, 5, 3))
    g = gm.grid
    nx, ny, nz = g.nx, g.ny, g.nz
    k = gm.perm.reshape(nz, ny, nx, 3)
    assert np.allclose(k[..., 2], 0.1 * k[..., 0], rtol=1e-15)
    mx = g.mult_x.reshape(nz, ny, nx - 1)
    cut = np.flatnonzero((mx == 0).all(axis=(0, 1)))
    assert list(cut + 1) == [int(round((f + 1) * nx / 3)) for f in range(2)]      # evenly spaced planes
    assert g.nnc_mult.min() >= 1e-3 and g.nnc_mult.max() <= 1.0
    a, b = g.nnc[:, 0], g.nnc[:, 1]
    ia, ja, ka = a % nx, (a // nx) % ny, a // (nx * ny)
    ib, jb, kb = b % nx, (b // nx) % ny, b // (nx * ny)
    assert np.all(kb - ka == 2)                                                   # 2-cell throw
    assert np.all(((ib - ia == 1) & (jb == ja) & (g.nnc_axis == 0)) | ((jb - ja == 1) & (ib == ia) & (g.nnc_axis == 1)))
    inactive = 1.0 - g.active_mask().mean()
    assert 0.04 < inactive < 0.15
    assert _connected(g)
    lnk = np.log(k[..., 0])
    assert np.array_equal(gm.facies.reshape(nz, ny, nx), (lnk > np.median(lnk)).astype(np.int8))
    _sources_ok(gm)


def test_config3_size_and_inactive_fraction():
    gm = G.config3(0)
    g = gm.grid
    assert (g.nx, g.ny, g.nz) == (200, 200, 50) and g.n_nnc > 0
    inactive = 1.0 - g.active_mask().mean()
    assert 0.05 < inactive < 0.12                                                  # ~8 %
    assert gm.block == (10, 10, 5)


@pytest.mark.parametrize("m", [0, 7, 187, 255])
def test_ensemble_members(m):
    gm = G.ensemble_member(m)
    g = gm.grid
    assert 24 <= g.nx <= 96 and 24 <= g.ny <= 96 and 8 <= g.nz <= 48 and 20_000 <= g.N <= 400_000
    sig = gm.meta["sigma"]
    assert 1.0 <= sig <= 3.0 and 2.0 <= gm.meta["corr"] <= 16.0
    z = (_lnk(gm) - np.log(100.0)) / sig
    assert z.min() >= -3.0 - 1e-9 and z.max() <= 3.0 + 1e-9                       # field clipped to +-3
    assert gm.seed == 1000 + m and gm.block == (8, 8, 4)
    _sources_ok(gm)
