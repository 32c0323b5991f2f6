"""CPU oracle for the multiscale multibasis pressure solver -- TEST INFRASTRUCTURE.

Plain FP64 C (``ms_oracle.c``) behind a ctypes shim, built single-threaded
(the correctness oracle) and, for timing the method on all host cores only,
with OpenMP (``use_openmp``; bitwise the same results except the rounding of
dot products and norms).  Only
``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package.  It shares
no code with the CUDA library: the two are compared on the same seeded
inputs.

What each routine follows (Klemetsdal, Moyner & Lie) and what pins it
(tests/test_oracle_pins.py):

=====================  ==========================================  ============================================
routine                paper                                       pinned by
=====================  ==========================================  ============================================
assemble_tpfa          Sec. 3 two-point flux; Eq. (9)              2-cell harmonic mean by hand; 1D closed form
                                                                   p_i = -i/T; multiplier / NNC / inactive cases;
                                                                   A 1 = 0; symmetry
pin                    problem statement (one reference cell)      dense solve equals the least-squares Neumann
                                                                   solution shifted to p_ref = 0
partition_cartesian    Sec. 5 (non-overlapping partition)          hand-counted blocks incl. ragged / empty blocks
components             Sec. 5.1 static / dynamic partitions        scipy connected_components on a masked graph
partition_dynamic      Sec. 5.1 dynamic (bins of |dp|)             hand-worked 1D example (tests/golden)
support_box            Sec. 5 requirement 2                        hand-worked boxes; Omega_j within S_j
support_hop            Sec. 5 requirement 2                        hand-worked 1D example (tests/golden)
msrsb_basis            Sec. 5.1 (MsRSB, localized iterations)      partition of unity; confinement; P >= 0;
                                                                   closed-form converged hat for two blocks in
                                                                   1D (and its 2D / 3D tensor products); values
                                                                   and increments of iterations 1 and 2 worked
                                                                   by hand on a 4-cell chain (omega, update from
                                                                   old values, renormalisation, stop test)
galerkin               Eq. (10), R = P^T                           symmetry; positive definiteness; P^T A 1 = 0
                                                                   for the unpinned A; dense P^T A P by numpy
cholesky(_solve)       coarse solve (A_c)^-1                       numpy.linalg.solve
galerkin_fv            Sec. 5, finite-volume restriction R         A_c 1 = 0 and 1^T A_c = 0 (unpinned A);
                                                                   constant basis: equals the Galerkin operator
                                                                   and -sum of the face transmissibilities
                                                                   between blocks (closed form)
lu(_solve)             coarse solve, Gaussian elimination          P A = L U; a zero leading pivot; numpy solve
partition_wells        Sec. 6.2 well bases                         hand-worked blocks; repeated cell rejected
cpr_residual /         Sec. 4 quasi-IMPES decoupling of a          Jacobian blocks against central finite
cpr_pressure           compressible two-phase step                 differences of cpr_residual; fluxes cancel in
                                                                   the sums over cells; weights cancel the
                                                                   saturation diagonal and sum to one;
                                                                   incompressible, equal densities, uniform
                                                                   state: J* = lambda_t A_tpfa / 2 (closed form)
ms_solve (FV stage)    Eq. (11) with R = block indicator           after a cycle ending in an FV coarse
                                                                   correction every block's residual sums to
                                                                   zero (local conservation); dense direct solve
ilu0 / ilu0_apply      Sec. 5.1 / 6.4 ILU(0)                       (L U)_ij = A_ij on the pattern (defining
                                                                   property); exact on tridiagonal A
ms_solve               Eq. (11) in Richardson (Sec. 5.2)           dense direct solve; identity partition
                                                                   converges in one cycle; A-norm error does not
                                                                   grow per coarse stage; first cycle with one
                                                                   and two stages worked by hand on a 4-cell
                                                                   ring (smoother before each coarse stage)
cost_model             Eq. (12)                                    sum of the itemised Sec. 6.4 counts
=====================  ==========================================  ============================================
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ms_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libms_oracle.so")
_LIB_OMP = os.path.join(_BUILD, "libms_oracle_omp.so")

OK, EINVAL, ENOMEM, ENOTCONV, ESINGULAR = 0, 1, 2, 4, 5


class OracleError(RuntimeError):
    def __init__(self, code, what):
        super().__init__(f"oracle {what} failed with status {code}")
        self.code = code


def build(force: bool = False, openmp: bool = False) -> str:
    """Compile the oracle with gcc (plain C11, -O2, no architecture flags);
    openmp=True builds the OpenMP variant used for timing."""
    os.makedirs(_BUILD, exist_ok=True)
    path = _LIB_OMP if openmp else _LIB
    if force or not os.path.exists(path) or os.path.getmtime(path) < os.path.getmtime(_SRC):
        tmp = path + f".tmp{os.getpid()}"
        extra = ["-fopenmp"] if openmp else []
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared"] + extra + ["-o", tmp, _SRC, "-lm"])
        os.replace(tmp, path)
    return path


_lib = None
_lib_omp = None
_use_omp = False


def use_openmp(on: bool = True) -> None:
    """Route later calls to the OpenMP build (timing on all host cores; its
    thread count follows OMP_NUM_THREADS) or back to the single-threaded one."""
    global _use_omp
    _use_omp = bool(on)


def openmp_threads() -> int:
    """Threads the OpenMP build runs with (builds it if needed)."""
    L = _load(True)
    L.or_threads.restype = _i
    return int(L.or_threads())

_i = C.c_int
_d = C.c_double
_pi = C.POINTER(C.c_int)
_pd = C.POINTER(C.c_double)
_ppi = C.POINTER(_pi)
_ppd = C.POINTER(_pd)
_vp = C.c_void_p


class _Stage(C.Structure):
    _fields_ = [("M", _i), ("sptr", _vp), ("scells", _vp), ("pval", _vp), ("L", _vp), ("part", _vp),
                ("piv", _vp)]


class _Adapt(C.Structure):
    _fields_ = [("schedule", _i), ("n_bins", _i), ("eps", _d), ("smoothed", _i), ("omega", _d),
                ("tol", _d), ("max_iter", _i), ("val_unpinned", _vp), ("cells", _vp),
                ("nx", _i), ("ny", _i), ("nz", _i), ("part_out", _vp), ("md_hist", _vp)]


def lib():
    return _load(_use_omp)


def _load(omp: bool):
    global _lib, _lib_omp
    cur = _lib_omp if omp else _lib
    if cur is None:
        cur = C.CDLL(build(openmp=omp))
        if omp:
            _lib_omp = cur
        else:
            _lib = cur
        L = cur
        L.or_free.argtypes = [_vp]
        L.or_tpfa_assemble.argtypes = [_i, _i, _i, _d, _d, _d, _vp, _vp, _vp, _vp, _vp, _i, _vp, _vp, _vp,
                                       _vp, _vp, _pi, _ppi, _pi, _ppi, _ppi, _ppd, _ppi, _ppi, _ppd]
        L.or_pin.argtypes = [_i, _vp, _vp, _vp, _vp, _i]
        L.or_partition_cartesian.argtypes = [_i, _i, _i, _i, _vp, _i, _i, _i, _vp, _pi]
        L.or_components.argtypes = [_i, _vp, _vp, _vp, _vp, _pi]
        L.or_partition_dynamic.argtypes = [_i, _vp, _vp, _vp, _i, _d, _vp, _pi]
        L.or_support_box.argtypes = [_i, _i, _i, _i, _vp, _vp, _vp, _vp, _i, _i, _i, _i, _ppi, _ppi]
        L.or_support_hop.argtypes = [_i, _i, _i, _i, _vp, _vp, _vp, _vp, _i, _ppi, _ppi]
        L.or_support_block.argtypes = [_i, _vp, _i, _ppi, _ppi]
        L.or_msrsb_basis.argtypes = [_i, _vp, _vp, _vp, _vp, _i, _vp, _vp, _d, _d, _i, _vp, _pi, _vp]
        L.or_constant_basis.argtypes = [_i, _vp, _vp]
        L.or_constant_basis.restype = None
        L.or_galerkin.argtypes = [_i, _vp, _vp, _vp, _i, _vp, _vp, _vp, _vp]
        L.or_cholesky.argtypes = [_i, _vp]
        L.or_cholesky_solve.argtypes = [_i, _vp, _vp, _vp]
        L.or_cholesky_solve.restype = None
        L.or_galerkin_fv.argtypes = [_i, _vp, _vp, _vp, _i, _vp, _vp, _vp, _vp, _vp]
        L.or_lu.argtypes = [_i, _vp, _vp]
        L.or_lu_solve.argtypes = [_i, _vp, _vp, _vp, _vp]
        L.or_lu_solve.restype = None
        L.or_partition_wells.argtypes = [_i, _i, _vp, _vp, _vp, _pi]
        L.or_cpr_residual.argtypes = [_i, _i, _vp, _vp, _vp, _d, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _d, _vp, _vp]
        L.or_cpr_residual.restype = None
        L.or_cpr_pressure.argtypes = [_i, _vp, _vp, _i, _vp, _vp, _vp, _d, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _d,
                                      _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]
        L.or_ilu0.argtypes = [_i, _vp, _vp, _vp, _vp]
        L.or_ilu0_apply.argtypes = [_i, _vp, _vp, _vp, _vp, _vp]
        L.or_ilu0_apply.restype = None
        L.or_ms_solve.argtypes = [_i, _vp, _vp, _vp, _i, C.POINTER(_Stage), _i, _vp, _d, _vp, _vp, _d, _i,
                                  C.POINTER(_Adapt), _pi, _vp]
        L.or_ms_gmres.argtypes = [_i, _vp, _vp, _vp, _i, C.POINTER(_Stage), _i, _vp, _d, _vp, _vp, _d, _i, _i,
                                  _pi, _vp]
        L.or_total_mobility.argtypes = [_i, _vp, _vp, _vp]
        L.or_total_mobility.restype = None
        L.or_fw_max_slope.argtypes = [_vp]
        L.or_fw_max_slope.restype = _d
        L.or_transport_step.argtypes = [_i, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _d, _d, _d, _d, _pi]
        L.or_cost_model.argtypes = [_d, _d, _d, _d, _d]
        L.or_cost_model.restype = _d
    return cur


def _p(a):
    return None if a is None else a.ctypes.data


def _take_i(ptr, n):
    out = np.ctypeslib.as_array(ptr, shape=(n,)).copy() if n > 0 else np.zeros(0, np.int32)
    lib().or_free(C.cast(ptr, _vp))
    return out.astype(np.int32, copy=False)


def _take_d(ptr, n):
    out = np.ctypeslib.as_array(ptr, shape=(n,)).copy() if n > 0 else np.zeros(0)
    lib().or_free(C.cast(ptr, _vp))
    return out


def _check(st, what):
    if st != OK:
        raise OracleError(st, what)


# ---------------------------------------------------------------------------- data types
@dataclass
class CSR:
    n: int
    rowptr: np.ndarray
    col: np.ndarray
    val: np.ndarray

    def copy(self):
        return CSR(self.n, self.rowptr.copy(), self.col.copy(), self.val.copy())

    def to_scipy(self):
        from scipy.sparse import csr_matrix
        return csr_matrix((self.val, self.col, self.rowptr), shape=(self.n, self.n))

    def dense(self):
        return self.to_scipy().toarray()


@dataclass
class System:
    A: CSR                 # unpinned TPFA matrix over active cells
    cells: np.ndarray      # grid index of each active cell
    faces: tuple           # (fa, fb, T_geometric)


@dataclass
class Basis:
    M: int
    sptr: np.ndarray       # CSC column pointers (per block)
    scells: np.ndarray     # support cells, ascending within each block
    pval: np.ndarray       # values aligned with scells
    part: np.ndarray
    iters: int = 0
    inc_hist: Optional[np.ndarray] = None

    def dense(self, n):
        P = np.zeros((n, self.M))
        for j in range(self.M):
            s, e = self.sptr[j], self.sptr[j + 1]
            P[self.scells[s:e], j] = self.pval[s:e]
        return P


# ---------------------------------------------------------------------------- routines
def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def assemble_tpfa(grid, perm, lam=None, p_prev=None) -> System:
    """Unpinned TPFA matrix over the active cells (Sec. 3, Eq. (9))."""
    L = lib()
    perm = _f64(perm).reshape(-1, 3)
    act = None if grid.active is None else np.ascontiguousarray(grid.active, dtype=np.uint8)
    mx = None if grid.mult_x is None else _f64(grid.mult_x)
    my = None if grid.mult_y is None else _f64(grid.mult_y)
    mz = None if grid.mult_z is None else _f64(grid.mult_z)
    nn = grid.n_nnc
    nnc = _i32(grid.nnc).reshape(-1) if nn else None
    nax = np.ascontiguousarray(grid.nnc_axis, dtype=np.int8) if nn else None
    nm = _f64(grid.nnc_mult) if nn else None
    lam = None if lam is None else _f64(lam)
    p_prev = None if p_prev is None else _f64(p_prev)
    n = _i(); nf = _i()
    cells = _pi(); fa = _pi(); fb = _pi(); ft = _pd(); rp = _pi(); ci = _pi(); v = _pd()
    st = L.or_tpfa_assemble(grid.nx, grid.ny, grid.nz, grid.dx, grid.dy, grid.dz, _p(act), _p(perm),
                            _p(mx), _p(my), _p(mz), nn, _p(nnc), _p(nax), _p(nm), _p(lam), _p(p_prev),
                            C.byref(n), C.byref(cells), C.byref(nf), C.byref(fa), C.byref(fb), C.byref(ft),
                            C.byref(rp), C.byref(ci), C.byref(v))
    _check(st, "tpfa_assemble")
    n = n.value; nf = nf.value
    rowptr = _take_i(rp, n + 1)
    nnz = int(rowptr[-1])
    A = CSR(n, rowptr, _take_i(ci, nnz), _take_d(v, nnz))
    return System(A, _take_i(cells, n), (_take_i(fa, nf), _take_i(fb, nf), _take_d(ft, nf)))


def pin(A: CSR, q: Optional[np.ndarray] = None, ref: int = 0):
    """Pinned copy of A (and q): row/column ``ref`` off-diagonals zeroed."""
    Ap = A.copy()
    qp = None if q is None else _f64(q).copy()
    _check(lib().or_pin(A.n, _p(Ap.rowptr), _p(Ap.col), _p(Ap.val), _p(qp), ref), "pin")
    return Ap, qp


def partition_cartesian(grid, cells, block):
    cells = _i32(cells)
    part = np.empty(len(cells), np.int32)
    M = _i()
    _check(lib().or_partition_cartesian(grid.nx, grid.ny, grid.nz, len(cells), _p(cells), int(block[0]),
                                        int(block[1]), int(block[2]), _p(part), C.byref(M)),
           "partition_cartesian")
    return part, M.value


def components(A: CSR, cls):
    cls = _i32(cls)
    part = np.empty(A.n, np.int32)
    M = _i()
    _check(lib().or_components(A.n, _p(A.rowptr), _p(A.col), _p(cls), _p(part), C.byref(M)), "components")
    return part, M.value


def partition_static(A: CSR, part_general, facies):
    """Static partition: general blocks split by facies class into connected
    components (Sec. 5.1, static partitions adapted to geology)."""
    nf = int(np.max(facies)) + 1 if len(facies) else 1
    return components(A, _i32(part_general) * nf + _i32(facies))


def partition_dynamic(A: CSR, dp, n_bins=8, eps=1e-8):
    dp = _f64(dp)
    part = np.empty(A.n, np.int32)
    M = _i()
    _check(lib().or_partition_dynamic(A.n, _p(A.rowptr), _p(A.col), _p(dp), n_bins, eps, _p(part), C.byref(M)),
           "partition_dynamic")
    return part, M.value


def support_box(grid, cells, A: CSR, part, M, block):
    cells = _i32(cells); part = _i32(part)
    sp = _pi(); sc = _pi()
    _check(lib().or_support_box(grid.nx, grid.ny, grid.nz, A.n, _p(cells), _p(A.rowptr), _p(A.col), _p(part), M,
                                int(block[0]), int(block[1]), int(block[2]), C.byref(sp), C.byref(sc)),
           "support_box")
    sptr = _take_i(sp, M + 1)
    return sptr, _take_i(sc, int(sptr[-1]))


def support_hop(grid, cells, A: CSR, part, M):
    cells = _i32(cells); part = _i32(part)
    sp = _pi(); sc = _pi()
    _check(lib().or_support_hop(grid.nx, grid.ny, grid.nz, A.n, _p(cells), _p(A.rowptr), _p(A.col), _p(part), M,
                                C.byref(sp), C.byref(sc)), "support_hop")
    sptr = _take_i(sp, M + 1)
    return sptr, _take_i(sc, int(sptr[-1]))


def support_block(part, M):
    part = _i32(part)
    sp = _pi(); sc = _pi()
    _check(lib().or_support_block(len(part), _p(part), M, C.byref(sp), C.byref(sc)), "support_block")
    sptr = _take_i(sp, M + 1)
    return sptr, _take_i(sc, int(sptr[-1]))


def msrsb_basis(A_unpinned: CSR, part, M, sptr, scells, omega=2.0 / 3.0, tol=1e-3, max_iter=500) -> Basis:
    part = _i32(part); sptr = _i32(sptr); scells = _i32(scells)
    pval = np.empty(int(sptr[-1]))
    hist = np.zeros(max(max_iter, 1))
    it = _i()
    _check(lib().or_msrsb_basis(A_unpinned.n, _p(A_unpinned.rowptr), _p(A_unpinned.col), _p(A_unpinned.val),
                                _p(part), M, _p(sptr), _p(scells), omega, tol, max_iter, _p(pval), C.byref(it),
                                _p(hist)), "msrsb_basis")
    return Basis(M, sptr, scells, pval, part, it.value, hist[: it.value].copy())


def constant_basis(part, M) -> Basis:
    sptr, scells = support_block(part, M)
    pval = np.empty(int(sptr[-1]))
    lib().or_constant_basis(M, _p(sptr), _p(pval))
    return Basis(M, sptr, scells, pval, _i32(part))


def galerkin(A: CSR, B: Basis) -> np.ndarray:
    Ac = np.empty((B.M, B.M))
    _check(lib().or_galerkin(A.n, _p(A.rowptr), _p(A.col), _p(A.val), B.M, _p(B.sptr), _p(B.scells), _p(B.pval),
                             _p(Ac)), "galerkin")
    return Ac


def cholesky(Ac) -> np.ndarray:
    L = _f64(Ac).copy()
    _check(lib().or_cholesky(L.shape[0], _p(L)), "cholesky")
    return L


def cholesky_solve(L, b):
    b = _f64(b); x = np.empty_like(b)
    lib().or_cholesky_solve(L.shape[0], _p(_f64(L)), _p(b), _p(x))
    return x


@dataclass
class FVFactor:
    """Finite-volume coarse stage: LU factors (with interchanges) of
    A_c = R A P, R the block indicator of ``part``."""
    LU: np.ndarray
    piv: np.ndarray
    part: np.ndarray


def galerkin_fv(A: CSR, B: Basis, part=None) -> np.ndarray:
    """A_c = R A P with R_ji = 1 for the cells i of block j (Sec. 5,
    finite-volume restriction); ``part`` defaults to the basis's partition."""
    part = _i32(B.part if part is None else part)
    Ac = np.empty((B.M, B.M))
    _check(lib().or_galerkin_fv(A.n, _p(A.rowptr), _p(A.col), _p(A.val), B.M, _p(B.sptr), _p(B.scells),
                                _p(B.pval), _p(part), _p(Ac)), "galerkin_fv")
    return Ac


def lu(Ac):
    """Dense LU with partial pivoting: returns (LU, piv)."""
    LU = _f64(Ac).copy()
    piv = np.zeros(LU.shape[0], np.int32)
    _check(lib().or_lu(LU.shape[0], _p(LU), _p(piv)), "lu")
    return LU, piv


def lu_solve(LU, piv, b):
    b = _f64(b); x = np.empty_like(b)
    lib().or_lu_solve(LU.shape[0], _p(_f64(LU)), _p(_i32(piv)), _p(b), _p(x))
    return x


def coarse_fv(A: CSR, B: Basis) -> FVFactor:
    """The finite-volume stage of basis B on the pinned A: factors of R A P."""
    LU, piv = lu(galerkin_fv(A, B))
    return FVFactor(LU, piv, _i32(B.part))


def partition_wells(n: int, wells: Sequence[Sequence[int]]):
    """Block w = the cells of well w; every other cell in block len(wells)."""
    wptr = np.zeros(len(wells) + 1, np.int32)
    for w, c in enumerate(wells):
        wptr[w + 1] = wptr[w] + len(c)
    wcells = _i32(np.concatenate([np.asarray(c, np.int32) for c in wells]) if wells else np.zeros(0, np.int32))
    part = np.empty(n, np.int32)
    M = _i()
    _check(lib().or_partition_wells(n, len(wells), _p(wptr), _p(wcells), _p(part), C.byref(M)), "partition_wells")
    return part, M.value


@dataclass
class LUFactor:
    """Galerkin stage of a non-symmetric A: LU factors of P^T A P."""
    LU: np.ndarray
    piv: np.ndarray


def coarse_lu(A: CSR, B: Basis) -> LUFactor:
    LU, piv = lu(galerkin(A, B))
    return LUFactor(LU, piv)


def _stage_struct(B, Lc, keep):
    if isinstance(Lc, LUFactor):
        LU, piv = _f64(Lc.LU), _i32(Lc.piv)
        keep += [B, LU, piv]
        return _Stage(B.M, _p(B.sptr), _p(B.scells), _p(B.pval), _p(LU), None, _p(piv))
    if isinstance(Lc, FVFactor):
        LU, piv, part = _f64(Lc.LU), _i32(Lc.piv), _i32(Lc.part)
        keep += [B, LU, piv, part]
        return _Stage(B.M, _p(B.sptr), _p(B.scells), _p(B.pval), _p(LU), _p(part), _p(piv))
    Lc = _f64(Lc)
    keep += [B, Lc]
    return _Stage(B.M, _p(B.sptr), _p(B.scells), _p(B.pval), _p(Lc), None, None)


def ilu0(A: CSR) -> np.ndarray:
    lu = np.empty_like(A.val)
    _check(lib().or_ilu0(A.n, _p(A.rowptr), _p(A.col), _p(A.val), _p(lu)), "ilu0")
    return lu


def ilu0_apply(A: CSR, lu, r):
    r = _f64(r); z = np.empty_like(r)
    lib().or_ilu0_apply(A.n, _p(A.rowptr), _p(A.col), _p(_f64(lu)), _p(r), _p(z))
    return z


@dataclass
class SolveResult:
    x: np.ndarray
    iters: int
    hist: np.ndarray
    converged: bool
    dyn_part: Optional[np.ndarray] = None
    md_hist: Optional[np.ndarray] = None


def ms_solve(A: CSR, stages: Sequence[tuple], q, tol=1e-6, max_iter=500, smoother="ilu0", jac_omega=2.0 / 3.0,
             x0=None, adapt: Optional[dict] = None, lu=None) -> SolveResult:
    """Multistage Richardson solve (Eq. (11)).  ``stages`` holds (Basis, L)
    pairs with L the Cholesky factor of the stage's Galerkin A_c, or an
    FVFactor for a finite-volume stage.  ``adapt`` (optional):
    dict(schedule=1|2, n_bins, eps, smoothed, omega, tol, max_iter,
    A_unpinned, grid, cells)."""
    L = lib()
    q = _f64(q)
    x = np.zeros(A.n) if x0 is None else _f64(x0).copy()
    keep = []
    arr = (_Stage * max(len(stages), 1))()
    for s, (B, Lc) in enumerate(stages):
        arr[s] = _stage_struct(B, Lc, keep)
    sm = 0 if smoother == "ilu0" else 1
    if sm == 0 and lu is None:
        lu = ilu0(A)
    hist = np.zeros(max_iter + 1)
    it = _i()
    ad_ptr = None
    dyn_part = md_hist = None
    if adapt:
        dyn_part = np.zeros(A.n, np.int32)
        md_hist = np.zeros(max_iter, np.int32)
        Au = adapt.get("A_unpinned", A)
        grid = adapt.get("grid")
        cells = _i32(adapt.get("cells", np.arange(A.n)))
        keep += [Au, cells]
        ad = _Adapt(int(adapt.get("schedule", 2)), int(adapt.get("n_bins", 8)), float(adapt.get("eps", 1e-8)),
                    int(adapt.get("smoothed", 0)), float(adapt.get("omega", 2.0 / 3.0)),
                    float(adapt.get("basis_tol", 1e-3)), int(adapt.get("basis_max_iter", 500)),
                    _p(Au.val), _p(cells), grid.nx if grid else A.n, grid.ny if grid else 1,
                    grid.nz if grid else 1, _p(dyn_part), _p(md_hist))
        ad_ptr = C.pointer(ad)
    st = L.or_ms_solve(A.n, _p(A.rowptr), _p(A.col), _p(A.val), len(stages), arr, sm,
                       _p(lu) if lu is not None else None, jac_omega, _p(q), _p(x), tol, max_iter, ad_ptr,
                       C.byref(it), _p(hist))
    if st not in (OK, ENOTCONV):
        raise OracleError(st, "ms_solve")
    n_it = it.value
    return SolveResult(x, n_it, hist[: n_it + 1].copy(), st == OK, dyn_part,
                       None if md_hist is None else md_hist[:n_it].copy())


def ms_gmres(A: CSR, stages: Sequence[tuple], q, tol=1e-6, max_iter=500, restart=30, smoother="ilu0",
             jac_omega=2.0 / 3.0, x0=None, lu=None) -> SolveResult:
    """Restarted right-preconditioned GMRES(restart) with one multistage cycle
    (Eq. (11), zero initial guess) as the preconditioner; max_iter bounds the
    Arnoldi steps.  hist[k] is ||q - A x|| / ||q|| after step k (the GMRES
    estimate inside a restart, the true residual at its end)."""
    L = lib()
    q = _f64(q)
    x = np.zeros(A.n) if x0 is None else _f64(x0).copy()
    keep = []
    arr = (_Stage * max(len(stages), 1))()
    for s, (B, Lc) in enumerate(stages):
        arr[s] = _stage_struct(B, Lc, keep)
    sm = 0 if smoother == "ilu0" else 1
    if sm == 0 and lu is None:
        lu = ilu0(A)
    hist = np.zeros(max_iter + 1)
    it = _i()
    st = L.or_ms_gmres(A.n, _p(A.rowptr), _p(A.col), _p(A.val), len(stages), arr, sm,
                       _p(lu) if lu is not None else None, jac_omega, _p(q), _p(x), tol, max_iter, restart,
                       C.byref(it), _p(hist))
    if st not in (OK, ENOTCONV):
        raise OracleError(st, "ms_gmres")
    n_it = it.value
    return SolveResult(x, n_it, hist[: n_it + 1].copy(), st == OK, None, None)


def _fluid(fl):
    d = dict(mu_w=1.0, mu_o=3.0, n_w=2.0, n_o=2.0, s_wc=0.0, s_or=0.0)
    d.update(fl or {})
    return np.array([d["mu_w"], d["mu_o"], d["n_w"], d["n_o"], d["s_wc"], d["s_or"]])


def total_mobility(S, fluid=None):
    """lambda_t = krw/mu_w + kro/mu_o (Corey) per cell."""
    S = _f64(S)
    fl = _fluid(fluid)
    lam = np.empty(len(S))
    lib().or_total_mobility(len(S), _p(S), _p(fl), _p(lam))
    return lam


def fw_max_slope(fluid=None):
    fl = _fluid(fluid)
    return lib().or_fw_max_slope(_p(fl))


def transport_step(A_unpinned: CSR, p, q, S, dt, fluid=None, porosity=0.2, volume=1.0, cfl=0.9):
    """Explicit upstream water transport over dt with the transmissibilities of
    A_unpinned (assembled with the step's face mobilities).  Returns (S_new,
    substeps)."""
    fl = _fluid(fluid)
    S = _f64(S).copy()
    p = _f64(p)
    q = _f64(q)
    k = _i()
    st = lib().or_transport_step(A_unpinned.n, _p(A_unpinned.rowptr), _p(A_unpinned.col), _p(A_unpinned.val),
                                 _p(p), _p(q), _p(S), _p(fl), porosity, volume, cfl, dt, C.byref(k))
    if st != OK:
        raise OracleError(st, "transport_step")
    return S, k.value


CPR_DEFAULT = dict(mu_w=1e-3, mu_o=3e-3, n_w=2.0, n_o=2.0, s_wc=0.0, s_or=0.0, phi0=0.2, rho_w0=1000.0,
                   rho_o0=800.0, c_w=4.5e-10, c_o=1.5e-9, c_r=5e-10, p_ref=2e7)


def _cpr_params(params):
    d = dict(CPR_DEFAULT)
    d.update(params or {})
    return np.array([d[k] for k in ("mu_w", "mu_o", "n_w", "n_o", "s_wc", "s_or", "phi0", "rho_w0", "rho_o0",
                                    "c_w", "c_o", "c_r", "p_ref")])


def cpr_residual(sysm: System, vol, p, s, p0, s0, qw, qo, dt, params=None):
    """(R_w, R_o) of the compressible two-phase step (Sec. 4 reading)."""
    fa, fb, T = sysm.faces
    cp = _cpr_params(params)
    n = sysm.A.n
    Rw, Ro = np.empty(n), np.empty(n)
    args = [_f64(x) for x in (p, s, p0, s0, qw, qo)]
    lib().or_cpr_residual(n, len(fa), _p(_i32(fa)), _p(_i32(fb)), _p(_f64(T)), float(vol), _p(cp),
                          *[_p(a) for a in args], float(dt), _p(Rw), _p(Ro))
    return Rw, Ro


def cpr_pressure(sysm: System, vol, p, s, p0, s0, qw, qo, dt, params=None) -> dict:
    """Jacobian blocks, quasi-IMPES weights and the CPR pressure system
    (Sec. 4): dict(Jwp, Jop, Jstar as CSR on A's pattern; Dws, Dos, Rw, Ro,
    ww, wo, rstar as vectors)."""
    A = sysm.A
    fa, fb, T = sysm.faces
    cp = _cpr_params(params)
    n, nnz = A.n, len(A.val)
    out = {k: np.empty(nnz) for k in ("Jwp", "Jop", "Jstar")}
    out.update({k: np.empty(n) for k in ("Dws", "Dos", "Rw", "Ro", "ww", "wo", "rstar")})
    args = [_f64(x) for x in (p, s, p0, s0, qw, qo)]
    _check(lib().or_cpr_pressure(n, _p(A.rowptr), _p(A.col), len(fa), _p(_i32(fa)), _p(_i32(fb)), _p(_f64(T)),
                                 float(vol), _p(cp), *[_p(a) for a in args], float(dt),
                                 *[_p(out[k]) for k in ("Jwp", "Jop", "Dws", "Dos", "Rw", "Ro", "ww", "wo",
                                                        "Jstar", "rstar")]), "cpr_pressure")
    for k in ("Jwp", "Jop", "Jstar"):
        out[k] = CSR(n, A.rowptr, A.col, out[k])
    return out


def cost_model(N, Np, d, b, Nc):
    return lib().or_cost_model(float(N), float(Np), float(d), float(b), float(Nc))


# ---------------------------------------------------------------------------- convenience
def setup_general(gm, omega=2.0 / 3.0, tol=1e-3, max_iter=500, support="box", block=None):
    """Assemble, pin and build the general-partition stage of a geomodel.
    Returns (system, A_pinned, q_pinned, basis, A_c, L)."""
    sysm = assemble_tpfa(gm.grid, gm.perm)
    Ap, qp = pin(sysm.A, gm.q_active(), 0)
    block = gm.block if block is None else block
    part, M = partition_cartesian(gm.grid, sysm.cells, block)
    if support == "box":
        sptr, sc = support_box(gm.grid, sysm.cells, sysm.A, part, M, block)
    else:
        sptr, sc = support_hop(gm.grid, sysm.cells, sysm.A, part, M)
    B = msrsb_basis(sysm.A, part, M, sptr, sc, omega, tol, max_iter)
    Ac = galerkin(Ap, B)
    return sysm, Ap, qp, B, Ac, cholesky(Ac)
