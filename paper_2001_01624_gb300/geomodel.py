"""Seeded synthetic geomodels for the multiscale pressure solver.

This module produces INPUTS only: Cartesian grids, permeability fields, active
masks, fault connections, facies indicators and source terms.  It contains no
step of the solver (no transmissibility, partition, basis or solve arithmetic),
so both the CUDA path and the CPU oracle consume the same arrays without
sharing any of the method.

Conventions
-----------
* Cell ``(i, j, k)`` has grid index ``c = i + nx * (j + ny * k)`` (i fastest).
  Arrays of cell data are laid out in that order.
* ``perm`` is ``float64[N, 3]`` holding the diagonal permeability
  ``(Kx, Ky, Kz)`` in m^2 (1 mD = 9.869233e-16 m^2).  Lengths are in metres
  (1 ft = 0.3048 m).
* Face multipliers: the x-face between ``(i,j,k)`` and ``(i+1,j,k)`` has index
  ``i + (nx-1) * (j + ny * k)``; the y-face between ``(i,j,k)`` and
  ``(i,j+1,k)`` has index ``i + nx * (j + (ny-1) * k)``; the z-face between
  ``(i,j,k)`` and ``(i,j,k+1)`` has index ``i + nx * (j + ny * k)``.
  A multiplier of 0 removes the face.
* Non-neighbour connections (``nnc``) are pairs of grid indices with the axis
  whose permeability component, face area and cell length define their
  two-point transmissibility, and a multiplier.
* ``q`` is the source vector over grid cells (0 on inactive cells); it sums to
  zero (injector +, producer -), the problem statement of the paper's
  Sec. 1 / Eq. (9) with sources at opposite corners.

The permeability recipes stand in for the SPE10 and SAIGUP models, which are
not available: Gaussian-correlated lognormal fields (white noise convolved with
``exp(-r^2 / (2 l^2))`` and re-standardised), binary sinuous channel facies
with a 1000:1 contrast, and a faulted model with a 2-cell throw.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Optional

import numpy as np

MD = 9.869233e-16  # m^2 per millidarcy
FT = 0.3048        # m per foot


@dataclass
class Grid:
    nx: int
    ny: int
    nz: int
    dx: float
    dy: float
    dz: float
    active: Optional[np.ndarray] = None      # uint8 [N]; None = all active
    mult_x: Optional[np.ndarray] = None      # float64 [(nx-1)*ny*nz]
    mult_y: Optional[np.ndarray] = None      # float64 [nx*(ny-1)*nz]
    mult_z: Optional[np.ndarray] = None      # float64 [nx*ny*(nz-1)]
    nnc: Optional[np.ndarray] = None         # int32 [n, 2] grid indices
    nnc_axis: Optional[np.ndarray] = None    # int8 [n] in {0,1,2}
    nnc_mult: Optional[np.ndarray] = None    # float64 [n]

    @property
    def N(self) -> int:
        return self.nx * self.ny * self.nz

    def active_mask(self) -> np.ndarray:
        if self.active is None:
            return np.ones(self.N, dtype=np.uint8)
        return self.active

    def active_cells(self) -> np.ndarray:
        """Grid index of every active cell, ascending (natural order)."""
        return np.flatnonzero(self.active_mask()).astype(np.int32)

    def n_active(self) -> int:
        return int(self.active_mask().sum())

    @property
    def n_nnc(self) -> int:
        return 0 if self.nnc is None else int(self.nnc.shape[0])


@dataclass
class Geomodel:
    name: str
    grid: Grid
    perm: np.ndarray                 # float64 [N, 3]  (m^2)
    q: np.ndarray                    # float64 [N]      grid-indexed sources
    block: tuple                     # Cartesian coarse block (bx, by, bz)
    facies: Optional[np.ndarray] = None   # int8 [N]
    seed: int = 0
    meta: dict = field(default_factory=dict)

    def q_active(self) -> np.ndarray:
        """Sources restricted to the active cells (natural order)."""
        return np.ascontiguousarray(self.q[self.grid.active_cells()])


# --------------------------------------------------------------------------- fields
def gaussian_field(shape_zyx, corr_len, rng) -> np.ndarray:
    """Standard-normal white noise convolved with a Gaussian kernel of length
    ``corr_len`` cells per axis (axes of extent 1 are not smoothed), then
    re-standardised to mean 0 / variance 1."""
    from scipy.ndimage import gaussian_filter

    z = rng.standard_normal(shape_zyx)
    if np.isscalar(corr_len):
        corr_len = (corr_len,) * len(shape_zyx)
    sig = tuple(0.0 if n == 1 else float(c) for n, c in zip(shape_zyx, corr_len))
    f = gaussian_filter(z, sigma=sig, mode="reflect", truncate=3.0)
    s = f.std()
    f = f - f.mean()
    if s > 0:
        f = f / s
    return f


def lognormal_perm(shape_zyx, mean_md, sigma, corr_len, rng, kz_ratio=1.0, clip=None) -> np.ndarray:
    """``ln K = ln(mean_md) + sigma * z`` with z a correlated standard field,
    optionally clipped to [-clip, clip]."""
    z = gaussian_field(shape_zyx, corr_len, rng)
    if clip is not None:
        z = np.clip(z, -clip, clip)
    kx = np.exp(np.log(mean_md) + sigma * z) * MD
    k = np.empty(kx.shape + (3,), dtype=np.float64)
    k[..., 0] = kx
    k[..., 1] = kx
    k[..., 2] = kx * kz_ratio
    return k


def channel_perm(nz, ny, nx, rng, k_bg_md=1.0, k_ch_md=1000.0, kz_ratio=0.1):
    """Binary sinuous channels along y, drawn independently per layer:
    3..6 channels with centreline ``x = x0 + a sin(2 pi y / lam + phi)`` and
    integer width U{4..8} cells."""
    kx = np.full((nz, ny, nx), k_bg_md)
    fac = np.zeros((nz, ny, nx), dtype=np.int8)
    y = np.arange(ny)[:, None]
    x = np.arange(nx)[None, :]
    for k in range(nz):
        nch = int(rng.integers(3, 7))
        for _ in range(nch):
            x0 = rng.uniform(0, nx)
            a = rng.uniform(2.0, 0.15 * nx + 2.0)
            lam = rng.uniform(0.3 * ny, 1.0 * ny)
            phi = rng.uniform(0, 2 * np.pi)
            w = int(rng.integers(4, 9))
            c = x0 + a * np.sin(2 * np.pi * y / lam + phi)
            m = np.abs(x - c) < 0.5 * w
            kx[k][m] = k_ch_md
            fac[k][m] = 1
    k = np.empty((nz, ny, nx, 3))
    k[..., 0] = kx * MD
    k[..., 1] = kx * MD
    k[..., 2] = kx * MD * kz_ratio
    return k, fac


def corner_sources(grid: Grid) -> np.ndarray:
    """+1 spread over the active cells of column (0, 0, :) and -1 over those of
    column (nx-1, ny-1, :)."""
    nx, ny, nz = grid.nx, grid.ny, grid.nz
    act = grid.active_mask().astype(bool)
    q = np.zeros(grid.N)
    inj = np.array([0 + nx * (0 + ny * k) for k in range(nz)])
    prd = np.array([(nx - 1) + nx * ((ny - 1) + ny * k) for k in range(nz)])
    inj = inj[act[inj]]
    prd = prd[act[prd]]
    if len(inj) == 0 or len(prd) == 0:      # fall back to the columns of the first / last active cell
        cells = np.flatnonzero(act)
        c0, c1 = cells[0], cells[-1]
        inj = np.array([c for c in (c0 % (nx * ny) + nx * ny * k for k in range(nz)) if act[c]])
        prd = np.array([c for c in (c1 % (nx * ny) + nx * ny * k for k in range(nz)) if act[c]])
    q[inj] = 1.0 / len(inj)
    q[prd] = -1.0 / len(prd)
    return q


# --------------------------------------------------------------------------- grids
def _largest_component(grid: Grid, act: np.ndarray) -> np.ndarray:
    """Keep the largest connected set of active cells (face graph + NNC)."""
    from scipy.sparse import coo_matrix
    from scipy.sparse.csgraph import connected_components

    nx, ny, nz = grid.nx, grid.ny, grid.nz
    N = grid.N
    idx = np.arange(N).reshape(nz, ny, nx)
    rows, cols = [], []

    def add(a, b, keep):
        rows.append(a[keep].ravel())
        cols.append(b[keep].ravel())

    a, b = idx[:, :, :-1], idx[:, :, 1:]
    mx = np.ones(a.shape, bool) if grid.mult_x is None else grid.mult_x.reshape(nz, ny, nx - 1) > 0
    add(a, b, mx & act.reshape(nz, ny, nx)[:, :, :-1] & act.reshape(nz, ny, nx)[:, :, 1:])
    a, b = idx[:, :-1, :], idx[:, 1:, :]
    my = np.ones(a.shape, bool) if grid.mult_y is None else grid.mult_y.reshape(nz, ny - 1, nx) > 0
    add(a, b, my & act.reshape(nz, ny, nx)[:, :-1, :] & act.reshape(nz, ny, nx)[:, 1:, :])
    if nz > 1:
        a, b = idx[:-1], idx[1:]
        mz = np.ones(a.shape, bool) if grid.mult_z is None else grid.mult_z.reshape(nz - 1, ny, nx) > 0
        add(a, b, mz & act.reshape(nz, ny, nx)[:-1] & act.reshape(nz, ny, nx)[1:])
    if grid.nnc is not None and len(grid.nnc):
        e = grid.nnc
        keep = act[e[:, 0]] & act[e[:, 1]] & (grid.nnc_mult > 0)
        rows.append(e[keep, 0])
        cols.append(e[keep, 1])
    r = np.concatenate(rows)
    c = np.concatenate(cols)
    g = coo_matrix((np.ones(len(r)), (r, c)), shape=(N, N))
    ncomp, lab = connected_components(g, directed=False)
    lab = np.where(act, lab, -1)
    counts = np.bincount(lab[act], minlength=ncomp)
    best = int(np.argmax(counts))
    return (lab == best)


# --------------------------------------------------------------------------- configs
def homogeneous(nx, ny, nz, k_md=100.0, dx=20 * FT, dy=10 * FT, dz=2 * FT,
                block=(2, 2, 1), kz_ratio=1.0, name="homogeneous") -> Geomodel:
    grid = Grid(nx, ny, nz, dx, dy, dz)
    perm = np.empty((grid.N, 3))
    perm[:, 0] = k_md * MD
    perm[:, 1] = k_md * MD
    perm[:, 2] = k_md * MD * kz_ratio
    return Geomodel(name, grid, perm, corner_sources(grid), tuple(block))


def lognormal_box(nx, ny, nz, seed=0, sigma=2.0, corr=8.0, mean_md=100.0,
                  block=(10, 20, 5), kz_ratio=1.0, dx=20 * FT, dy=10 * FT, dz=2 * FT,
                  name="lognormal") -> Geomodel:
    rng = np.random.default_rng(seed)
    grid = Grid(nx, ny, nz, dx, dy, dz)
    k = lognormal_perm((nz, ny, nx), mean_md, sigma, corr, rng, kz_ratio)
    return Geomodel(name, grid, k.reshape(-1, 3), corner_sources(grid), tuple(block), seed=seed)


def config1(seed=0) -> Geomodel:
    """2D 60x220 lognormal (ln K ~ N(ln 100 mD, 2^2), correlation 8 cells),
    dx = 20 ft, dy = 10 ft, 6x11 coarse blocks of 10x20."""
    g = lognormal_box(60, 220, 1, seed=seed, sigma=2.0, corr=8.0, block=(10, 20, 1),
                      name="c1_2d_60x220")
    return g


def config2(seed=0) -> Geomodel:
    """3D 60x220x85: top 35 layers anisotropic lognormal (Kz = 0.1 Kx), bottom
    50 layers binary channel facies (1 mD / 1000 mD, Kz = 0.1 Kx); 10x20x5
    coarse blocks (6x11x17)."""
    nx, ny, nz = 60, 220, 85
    rng = np.random.default_rng(seed)
    grid = Grid(nx, ny, nz, 20 * FT, 10 * FT, 2 * FT)
    top = lognormal_perm((35, ny, nx), 100.0, 2.0, 8.0, rng, kz_ratio=0.1)
    bot, fac_b = channel_perm(nz - 35, ny, nx, rng)
    k = np.concatenate([top, bot], axis=0)
    fac = np.concatenate([np.zeros((35, ny, nx), np.int8), fac_b], axis=0)
    return Geomodel("c2_3d_60x220x85", grid, k.reshape(-1, 3), corner_sources(grid),
                    (10, 20, 5), facies=fac.ravel(), seed=seed)


def faulted(nx, ny, nz, seed=0, n_fault_x=3, n_fault_y=3, throw=2, inactive_pct=8.0,
            sigma=2.0, corr=8.0, block=(10, 10, 5), name="faulted") -> Geomodel:
    """Lognormal (Kz = 0.1 Kx) model with vertical faults at evenly spaced
    constant-x and constant-y planes.  Across a fault the cell (i,j,k) on the
    low side connects to the cell shifted by ``throw`` layers down on the high
    side (full overlap), with a per-fault multiplier log-uniform in [1e-3, 1].
    Cells where a second smooth field exceeds its (100 - inactive_pct)
    percentile are inactive; only the largest connected set of active cells is
    kept.  Facies = (ln K > median)."""
    rng = np.random.default_rng(seed)
    grid = Grid(nx, ny, nz, 20 * FT, 10 * FT, 2 * FT)
    k = lognormal_perm((nz, ny, nx), 100.0, sigma, corr, rng, kz_ratio=0.1)
    lnk = np.log(k[..., 0])
    fac = (lnk > np.median(lnk)).astype(np.int8)
    mult_x = np.ones((nz, ny, nx - 1))
    mult_y = np.ones((nz, ny - 1, nx))
    nnc, axis, mult = [], [], []
    idx = np.arange(grid.N).reshape(nz, ny, nx)
    fx = [int(round((f + 1) * nx / (n_fault_x + 1))) for f in range(n_fault_x)]
    fy = [int(round((f + 1) * ny / (n_fault_y + 1))) for f in range(n_fault_y)]
    for xf in fx:   # face between columns xf-1 and xf
        m = 10.0 ** rng.uniform(-3.0, 0.0)
        mult_x[:, :, xf - 1] = 0.0
        a = idx[: nz - throw, :, xf - 1]
        b = idx[throw:, :, xf]
        nnc.append(np.stack([a.ravel(), b.ravel()], 1))
        axis.append(np.zeros(a.size, np.int8))
        mult.append(np.full(a.size, m))
    for yf in fy:
        m = 10.0 ** rng.uniform(-3.0, 0.0)
        mult_y[:, yf - 1, :] = 0.0
        a = idx[: nz - throw, yf - 1, :]
        b = idx[throw:, yf, :]
        nnc.append(np.stack([a.ravel(), b.ravel()], 1))
        axis.append(np.ones(a.size, np.int8))
        mult.append(np.full(a.size, m))
    grid.mult_x = mult_x.ravel()
    grid.mult_y = mult_y.ravel()
    if nnc:
        grid.nnc = np.concatenate(nnc).astype(np.int32)
        grid.nnc_axis = np.concatenate(axis)
        grid.nnc_mult = np.concatenate(mult)
    if inactive_pct > 0:
        s = gaussian_field((nz, ny, nx), corr, rng).ravel()
        act = s <= np.percentile(s, 100.0 - inactive_pct)
        for kk in range(nz):                     # keep the source corner columns active
            act[0 + nx * ny * kk] = True
            act[(nx - 1) + nx * ((ny - 1) + ny * kk)] = True
    else:
        act = np.ones(grid.N, bool)
    act = _largest_component(grid, act)
    grid.active = act.astype(np.uint8)
    return Geomodel(name, grid, k.reshape(-1, 3), corner_sources(grid), tuple(block),
                    facies=fac.ravel(), seed=seed)


def config3(seed=0) -> Geomodel:
    """3D faulted 200x200x50 (~8 % inactive), 6 vertical faults, 2-cell throw;
    general partition 10x10x5 (20x20x10 = 4000 blocks)."""
    return faulted(200, 200, 50, seed=seed, name="c3_faulted_200x200x50")


def ensemble_member(m: int, block=(8, 8, 4)) -> Geomodel:
    """Member m of the uneven batched ensemble: nx, ny ~ U{24..96},
    nz ~ U{8..48} redrawn until 20k <= N <= 400k; correlation length
    U[2, 16] cells, sigma U[1, 3]; seed 1000 + m.  The standard field is
    clipped to +-3: with sigma near 3 its +-4.5 tails span ten orders of
    magnitude of K and can seal regions off so nearly that even a direct
    FP64 solve misses a 1e-6 relative residual."""
    rng = np.random.default_rng(1000 + m)
    while True:
        nx = int(rng.integers(24, 97))
        ny = int(rng.integers(24, 97))
        nz = int(rng.integers(8, 49))
        if 20_000 <= nx * ny * nz <= 400_000:
            break
    corr = float(rng.uniform(2.0, 16.0))
    sigma = float(rng.uniform(1.0, 3.0))
    grid = Grid(nx, ny, nz, 20 * FT, 10 * FT, 2 * FT)
    k = lognormal_perm((nz, ny, nx), 100.0, sigma, corr, rng, kz_ratio=0.1, clip=3.0)
    return Geomodel(f"c4_member_{m}", grid, k.reshape(-1, 3), corner_sources(grid),
                    tuple(block), seed=1000 + m, meta=dict(corr=corr, sigma=sigma))


def make_config(name: str, seed: int = 0) -> Geomodel:
    table = {"c1": config1, "c2": config2, "c3": config3}
    if name not in table:
        raise KeyError(name)
    return table[name](seed)
