/*
 * ms_oracle.c -- plain FP64 CPU oracle for the iterative multiscale multibasis
 * pressure solver of Klemetsdal, Moyner & Lie, "Accelerating Multiscale
 * Simulation of Complex Geomodels by Use of Dynamically Adapted Basis
 * Functions".
 *
 * TEST INFRASTRUCTURE ONLY.  This file exists to check the CUDA library
 * against an independent, slow, obviously-correct implementation.  Only the
 * test suite, the smoke check and the CPU-baseline leg of the benchmark load
 * it.  It shares no code, header, table or helper with the CUDA library.
 *
 * Every routine is double precision and follows the paper's steps in the
 * paper's order.  Where the paper is silent the routine follows one stated
 * reading (each is named in its comment).  The library is built twice: once
 * single-threaded (the correctness oracle the tests compare against) and
 * once with -fopenmp, only to time the method on all host cores.  The
 * OpenMP build splits loops whose iterations each write their own outputs
 * (rows of a product, basis columns, cells, coarse columns), which gives
 * bitwise the single-threaded results, and sums dot products and norms in
 * per-thread partial sums, which changes only their rounding.
 *
 * Memory: routines that produce variable-size results return malloc'd arrays
 * through out-pointers; release them with or_free().
 *
 * Parity: every public routine is pinned by a test against something other
 * than itself (closed forms, invariants, dense direct solves, hand-worked
 * examples); see the header of oracle/__init__.py for the list.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#define OR_PAR_FOR _Pragma("omp parallel for schedule(static)")
#define OR_PAR_FOR_DYN _Pragma("omp parallel for schedule(dynamic, 8)")
#define OR_PRAGMA(x) _Pragma(#x)
#define OR_PAR_SUM(v) OR_PRAGMA(omp parallel for schedule(static) reduction(+ : v))
#define OR_PAR_MAX(v) OR_PRAGMA(omp parallel for schedule(static) reduction(max : v))
#define OR_THREADS() omp_get_max_threads()
#define OR_TID() omp_get_thread_num()
#else
#define OR_PAR_FOR
#define OR_PAR_FOR_DYN
#define OR_PAR_SUM(v)
#define OR_PAR_MAX(v)
#define OR_THREADS() 1
#define OR_TID() 0
#endif

#define OR_OK 0
#define OR_EINVAL 1
#define OR_ENOMEM 2
#define OR_ENOTCONV 4
#define OR_ESINGULAR 5

void or_free(void *p) { free(p); }

/* Threads the loops below run on (1 in the single-threaded build). */
int or_threads(void) { return OR_THREADS(); }

static void *xmalloc(size_t n) { return malloc(n ? n : 1); }
static void *xcalloc(size_t n, size_t s) { return calloc(n ? n : 1, s ? s : 1); }

/* ------------------------------------------------------------------------ */
/* Two-point flux approximation (Sec. 3: two-point fluxes, single-point      */
/* upstream mobility) assembled into A of Eq. (9), A p = q.                  */
/*                                                                           */
/* Reading: diagonal K per cell; half transmissibility                       */
/*   t_i = K_i,axis * area / (h_axis / 2);                                   */
/* face transmissibility T = mult / (1/t_a + 1/t_b), times the face mobility */
/* (upstream cell's by the sign of p_prev_a - p_prev_b; arithmetic mean on a */
/* tie or when no previous pressure is given).  A_ii = sum_j T_ij,           */
/* A_ij = -T_ij.  Unknowns are the active cells in natural order.            */
/* ------------------------------------------------------------------------ */
typedef struct {
    int a, b;
    double t;
} or_conn;

static int conn_push(or_conn **v, int *n, int *cap, int a, int b, double t) {
    if (*n == *cap) {
        int nc = *cap ? 2 * *cap : 1024;
        or_conn *nv = (or_conn *)realloc(*v, (size_t)nc * sizeof(or_conn));
        if (!nv) return OR_ENOMEM;
        *v = nv;
        *cap = nc;
    }
    (*v)[*n].a = a;
    (*v)[*n].b = b;
    (*v)[*n].t = t;
    (*n)++;
    return OR_OK;
}

static double half_trans(const double *perm, int cell, int axis, double dx, double dy, double dz) {
    double h, area;
    if (axis == 0) { h = dx; area = dy * dz; }
    else if (axis == 1) { h = dy; area = dx * dz; }
    else { h = dz; area = dx * dy; }
    return perm[3 * (size_t)cell + axis] * area / (0.5 * h);
}

static double two_point(double ta, double tb, double mult) {
    if (!(ta > 0.0) || !(tb > 0.0) || !(mult > 0.0)) return 0.0;
    return mult / (1.0 / ta + 1.0 / tb);
}

static int cmp_int(const void *x, const void *y) {
    int a = *(const int *)x, b = *(const int *)y;
    return (a > b) - (a < b);
}

int or_tpfa_assemble(int nx, int ny, int nz, double dx, double dy, double dz,
                     const uint8_t *active, const double *perm,
                     const double *mult_x, const double *mult_y, const double *mult_z,
                     int n_nnc, const int32_t *nnc, const int8_t *nnc_axis, const double *nnc_mult,
                     const double *lambda, const double *p_prev,
                     int *n_out, int **cells_out,
                     int *nf_out, int **fa_out, int **fb_out, double **ft_out,
                     int **rowptr_out, int **col_out, double **val_out) {
    if (nx <= 0 || ny <= 0 || nz <= 0 || !(dx > 0) || !(dy > 0) || !(dz > 0) || !perm) return OR_EINVAL;
    int N = nx * ny * nz;
    for (int c = 0; c < N; ++c)
        for (int a = 0; a < 3; ++a) {
            double k = perm[3 * (size_t)c + a];
            if (!(k >= 0.0) || isinf(k)) return OR_EINVAL;
        }
    int *g2a = (int *)xmalloc((size_t)N * sizeof(int));
    int n = 0;
    for (int c = 0; c < N; ++c) g2a[c] = (!active || active[c]) ? n++ : -1;
    int *cells = (int *)xmalloc((size_t)n * sizeof(int));
    for (int c = 0; c < N; ++c)
        if (g2a[c] >= 0) cells[g2a[c]] = c;

    or_conn *cv = NULL;
    int nc = 0, cap = 0, st = OR_OK;
    for (int k = 0; k < nz && st == OR_OK; ++k)
        for (int j = 0; j < ny && st == OR_OK; ++j)
            for (int i = 0; i < nx && st == OR_OK; ++i) {
                int c = i + nx * (j + ny * k);
                if (g2a[c] < 0) continue;
                if (i + 1 < nx && g2a[c + 1] >= 0) {
                    double m = mult_x ? mult_x[i + (nx - 1) * (j + ny * k)] : 1.0;
                    if (m > 0.0) {
                        double T = two_point(half_trans(perm, c, 0, dx, dy, dz),
                                             half_trans(perm, c + 1, 0, dx, dy, dz), m);
                        st = conn_push(&cv, &nc, &cap, g2a[c], g2a[c + 1], T);
                    }
                }
                if (j + 1 < ny && g2a[c + nx] >= 0) {
                    double m = mult_y ? mult_y[i + nx * (j + (ny - 1) * k)] : 1.0;
                    if (m > 0.0) {
                        double T = two_point(half_trans(perm, c, 1, dx, dy, dz),
                                             half_trans(perm, c + nx, 1, dx, dy, dz), m);
                        st = conn_push(&cv, &nc, &cap, g2a[c], g2a[c + nx], T);
                    }
                }
                if (k + 1 < nz && g2a[c + nx * ny] >= 0) {
                    double m = mult_z ? mult_z[i + nx * (j + ny * k)] : 1.0;
                    if (m > 0.0) {
                        double T = two_point(half_trans(perm, c, 2, dx, dy, dz),
                                             half_trans(perm, c + nx * ny, 2, dx, dy, dz), m);
                        st = conn_push(&cv, &nc, &cap, g2a[c], g2a[c + nx * ny], T);
                    }
                }
            }
    for (int e = 0; e < n_nnc && st == OR_OK; ++e) {
        int ca = nnc[2 * e], cb = nnc[2 * e + 1];
        int ax = nnc_axis[e];
        if (ca < 0 || cb < 0 || ca >= N || cb >= N || ca == cb || ax < 0 || ax > 2) { st = OR_EINVAL; break; }
        if (g2a[ca] < 0 || g2a[cb] < 0 || !(nnc_mult[e] > 0.0)) continue;
        double T = two_point(half_trans(perm, ca, ax, dx, dy, dz), half_trans(perm, cb, ax, dx, dy, dz), nnc_mult[e]);
        st = conn_push(&cv, &nc, &cap, g2a[ca], g2a[cb], T);
    }
    if (st != OR_OK) { free(cv); free(g2a); free(cells); return st; }

    /* geometric face list (before mobility) */
    int *fa = (int *)xmalloc((size_t)nc * sizeof(int));
    int *fb = (int *)xmalloc((size_t)nc * sizeof(int));
    double *ft = (double *)xmalloc((size_t)nc * sizeof(double));
    for (int e = 0; e < nc; ++e) { fa[e] = cv[e].a; fb[e] = cv[e].b; ft[e] = cv[e].t; }

    /* face mobility */
    if (lambda) {
        for (int e = 0; e < nc; ++e) {
            int a = cv[e].a, b = cv[e].b;
            double lf;
            if (p_prev && p_prev[a] != p_prev[b]) lf = (p_prev[a] > p_prev[b]) ? lambda[a] : lambda[b];
            else lf = 0.5 * (lambda[a] + lambda[b]);
            cv[e].t *= lf;
        }
    }

    /* CSR: each row = diagonal + one entry per incident connection, sorted by
       column, duplicate columns summed. */
    int *cnt = (int *)xcalloc((size_t)n + 1, sizeof(int));
    for (int e = 0; e < nc; ++e) { cnt[cv[e].a]++; cnt[cv[e].b]++; }
    int *rp = (int *)xmalloc(((size_t)n + 1) * sizeof(int));
    rp[0] = 0;
    for (int i = 0; i < n; ++i) rp[i + 1] = rp[i] + cnt[i] + 1;
    int *tc = (int *)xmalloc((size_t)rp[n] * sizeof(int));
    double *tv = (double *)xmalloc((size_t)rp[n] * sizeof(double));
    int *fill = (int *)xmalloc((size_t)n * sizeof(int));
    for (int i = 0; i < n; ++i) { tc[rp[i]] = i; tv[rp[i]] = 0.0; fill[i] = rp[i] + 1; }
    for (int e = 0; e < nc; ++e) {
        int a = cv[e].a, b = cv[e].b;
        double t = cv[e].t;
        tv[rp[a]] += t;
        tv[rp[b]] += t;
        tc[fill[a]] = b; tv[fill[a]++] = -t;
        tc[fill[b]] = a; tv[fill[b]++] = -t;
    }
    /* sort within rows (insertion sort by column, carrying values) and merge */
    int *orp = (int *)xmalloc(((size_t)n + 1) * sizeof(int));
    int *oc = (int *)xmalloc((size_t)rp[n] * sizeof(int));
    double *ov = (double *)xmalloc((size_t)rp[n] * sizeof(double));
    int w = 0;
    orp[0] = 0;
    for (int i = 0; i < n; ++i) {
        int s = rp[i], e = rp[i + 1];
        for (int p = s + 1; p < e; ++p) {
            int cc = tc[p];
            double vv = tv[p];
            int q = p - 1;
            while (q >= s && tc[q] > cc) { tc[q + 1] = tc[q]; tv[q + 1] = tv[q]; --q; }
            tc[q + 1] = cc;
            tv[q + 1] = vv;
        }
        for (int p = s; p < e; ++p) {
            if (w > orp[i] && oc[w - 1] == tc[p]) ov[w - 1] += tv[p];
            else { oc[w] = tc[p]; ov[w] = tv[p]; ++w; }
        }
        orp[i + 1] = w;
    }
    free(cnt); free(rp); free(tc); free(tv); free(fill); free(cv); free(g2a);
    *n_out = n;
    *cells_out = cells;
    *nf_out = nc;
    *fa_out = fa; *fb_out = fb; *ft_out = ft;
    *rowptr_out = orp; *col_out = oc; *val_out = ov;
    return OR_OK;
}

/* Reference-cell pin (problem statement: one reference cell fixed).  Row r
 * and column r lose their off-diagonal entries; the diagonal is kept; the
 * source of row r becomes 0.  The pattern is kept (values become 0). */
int or_pin(int n, const int *rowptr, const int *col, double *val, double *q, int ref) {
    if (ref < 0 || ref >= n) return OR_EINVAL;
    for (int i = 0; i < n; ++i)
        for (int p = rowptr[i]; p < rowptr[i + 1]; ++p)
            if ((i == ref) != (col[p] == ref)) val[p] = 0.0;
    if (q) q[ref] = 0.0;
    return OR_OK;
}

/* y = A x  (CSR) */
static void csr_mv(int n, const int *rp, const int *ci, const double *v, const double *x, double *y) {
    OR_PAR_FOR
    for (int i = 0; i < n; ++i) {
        double s = 0.0;
        for (int p = rp[i]; p < rp[i + 1]; ++p) s += v[p] * x[ci[p]];
        y[i] = s;
    }
}

static int diag_pos(const int *rp, const int *ci, int i) {
    for (int p = rp[i]; p < rp[i + 1]; ++p)
        if (ci[p] == i) return p;
    return -1;
}

/* ------------------------------------------------------------------------ */
/* Coarse partitions (Sec. 5: non-overlapping partition into M blocks;      */
/* Sec. 5.1: general, static and dynamic partitions).                        */
/* ------------------------------------------------------------------------ */

/* General structured partition: block (i/bx, j/by, k/bz); empty blocks are
 * dropped and the rest numbered in increasing Cartesian block index. */
int or_partition_cartesian(int nx, int ny, int nz, int n, const int *cells, int bx, int by, int bz,
                           int *part, int *M_out) {
    if (bx <= 0 || by <= 0 || bz <= 0) return OR_EINVAL;
    int nbx = (nx + bx - 1) / bx, nby = (ny + by - 1) / by, nbz = (nz + bz - 1) / bz;
    size_t nb = (size_t)nbx * nby * nbz;
    int *map = (int *)xmalloc(nb * sizeof(int));
    for (size_t b = 0; b < nb; ++b) map[b] = -1;
    for (int a = 0; a < n; ++a) {
        int c = cells[a], i = c % nx, j = (c / nx) % ny, k = c / (nx * ny);
        map[(i / bx) + (size_t)nbx * ((j / by) + (size_t)nby * (k / bz))] = 0;
    }
    int M = 0;
    for (size_t b = 0; b < nb; ++b)
        if (map[b] == 0) map[b] = M++;
    for (int a = 0; a < n; ++a) {
        int c = cells[a], i = c % nx, j = (c / nx) % ny, k = c / (nx * ny);
        part[a] = map[(i / bx) + (size_t)nbx * ((j / by) + (size_t)nby * (k / bz))];
    }
    free(map);
    *M_out = M;
    return OR_OK;
}

/* Connected components (through the off-diagonal pattern of A) of cells of
 * equal class; components are numbered in order of their lowest cell index.
 * Used for the static partition (Cartesian block x facies class) and the
 * dynamic partition (bin of |dp|). */
int or_components(int n, const int *rowptr, const int *col, const int *cls, int *part, int *M_out) {
    int *queue = (int *)xmalloc((size_t)n * sizeof(int));
    for (int i = 0; i < n; ++i) part[i] = -1;
    int M = 0;
    for (int s = 0; s < n; ++s) {
        if (part[s] >= 0) continue;
        int head = 0, tail = 0;
        queue[tail++] = s;
        part[s] = M;
        while (head < tail) {
            int i = queue[head++];
            for (int p = rowptr[i]; p < rowptr[i + 1]; ++p) {
                int k = col[p];
                if (k != i && part[k] < 0 && cls[k] == cls[s]) { part[k] = M; queue[tail++] = k; }
            }
        }
        ++M;
    }
    free(queue);
    *M_out = M;
    return OR_OK;
}

/* Dynamic partition from the pressure update (Sec. 5.1, "Dynamic" bases:
 * cells binned by the magnitude of their pressure update).
 * Reading: v_i = log10(max(|dp_i|, eps * max|dp|)); n_bins equal-width bins
 * on [min v, max v], bin = min(floor((v - vmin) / width), n_bins - 1) (a value
 * on an edge goes to the upper bin); blocks = connected components within a
 * bin.  All-zero dp gives a single class. */
int or_partition_dynamic(int n, const int *rowptr, const int *col, const double *dp, int n_bins, double eps,
                         int *part, int *M_out) {
    if (n_bins <= 0 || !(eps > 0.0)) return OR_EINVAL;
    double amax = 0.0;
    for (int i = 0; i < n; ++i) { double a = fabs(dp[i]); if (a > amax) amax = a; }
    int *cls = (int *)xcalloc((size_t)n, sizeof(int));
    if (amax > 0.0) {
        double *v = (double *)xmalloc((size_t)n * sizeof(double));
        double vmin = INFINITY, vmax = -INFINITY;
        for (int i = 0; i < n; ++i) {
            double a = fabs(dp[i]);
            if (a < eps * amax) a = eps * amax;
            v[i] = log10(a);
            if (v[i] < vmin) vmin = v[i];
            if (v[i] > vmax) vmax = v[i];
        }
        if (vmax > vmin) {
            double w = (vmax - vmin) / n_bins;
            for (int i = 0; i < n; ++i) {
                int b = (int)floor((v[i] - vmin) / w);
                if (b > n_bins - 1) b = n_bins - 1;
                if (b < 0) b = 0;
                cls[i] = b;
            }
        }
        free(v);
    }
    int st = or_components(n, rowptr, col, cls, part, M_out);
    free(cls);
    return st;
}

/* ------------------------------------------------------------------------ */
/* Basis supports (Sec. 5, requirement 2: compact support S_j containing    */
/* block j).                                                                 */
/* ------------------------------------------------------------------------ */
typedef struct { int *ptr; int *cells; int cap; } or_lists;

static int cells_sorted_unique(int *v, int m) {
    qsort(v, (size_t)m, sizeof(int), cmp_int);
    int w = 0;
    for (int i = 0; i < m; ++i)
        if (w == 0 || v[w - 1] != v[i]) v[w++] = v[i];
    return w;
}

/* Cartesian box rule: the block's nominal index box (from the Cartesian
 * block of its cells) grown by floor(b/2) cells on each side of each axis,
 * clipped to the grid, restricted to active cells reachable from the block
 * through connections that stay inside the grown box. */
int or_support_box(int nx, int ny, int nz, int n, const int *cells, const int *rowptr, const int *col,
                   const int *part, int M, int bx, int by, int bz, int **sptr_out, int **scells_out) {
    if (bx <= 0 || by <= 0 || bz <= 0) return OR_EINVAL;
    int N = nx * ny * nz;
    int *g2a = (int *)xmalloc((size_t)N * sizeof(int));
    for (int c = 0; c < N; ++c) g2a[c] = -1;
    for (int a = 0; a < n; ++a) g2a[cells[a]] = a;
    int *first = (int *)xmalloc((size_t)M * sizeof(int));
    for (int j = 0; j < M; ++j) first[j] = -1;
    for (int a = 0; a < n; ++a)
        if (first[part[a]] < 0) first[part[a]] = a;
    int *bptr = (int *)xcalloc((size_t)M + 1, sizeof(int));     /* block member lists */
    for (int a = 0; a < n; ++a) bptr[part[a] + 1]++;
    for (int j = 0; j < M; ++j) bptr[j + 1] += bptr[j];
    int *bcell = (int *)xmalloc((size_t)n * sizeof(int));
    int *bf = (int *)xmalloc((size_t)M * sizeof(int));
    for (int j = 0; j < M; ++j) bf[j] = bptr[j];
    for (int a = 0; a < n; ++a) bcell[bf[part[a]]++] = a;
    free(bf);

    int *stamp = (int *)xmalloc((size_t)n * sizeof(int));
    for (int a = 0; a < n; ++a) stamp[a] = -1;
    int *queue = (int *)xmalloc((size_t)n * sizeof(int));
    size_t cap = (size_t)n * 4 + 16, used = 0;
    int *sc = (int *)xmalloc(cap * sizeof(int));
    int *sp = (int *)xmalloc(((size_t)M + 1) * sizeof(int));
    sp[0] = 0;
    for (int j = 0; j < M; ++j) {
        if (first[j] < 0) { sp[j + 1] = (int)used; continue; }
        int c0 = cells[first[j]];
        int I = (c0 % nx) / bx, J = ((c0 / nx) % ny) / by, K = (c0 / (nx * ny)) / bz;
        int x0 = I * bx - bx / 2, x1 = (I + 1) * bx - 1 + bx / 2;
        int y0 = J * by - by / 2, y1 = (J + 1) * by - 1 + by / 2;
        int z0 = K * bz - bz / 2, z1 = (K + 1) * bz - 1 + bz / 2;
        if (x0 < 0) x0 = 0;
        if (y0 < 0) y0 = 0;
        if (z0 < 0) z0 = 0;
        if (x1 > nx - 1) x1 = nx - 1;
        if (y1 > ny - 1) y1 = ny - 1;
        if (z1 > nz - 1) z1 = nz - 1;
        /* breadth-first search from the block inside the box */
        int head = 0, tail = 0;
        int stj = 2 * j, stv = 2 * j + 1;        /* candidate / visited stamps */
        for (int k = z0; k <= z1; ++k)
            for (int jj = y0; jj <= y1; ++jj)
                for (int i = x0; i <= x1; ++i) {
                    int a = g2a[i + nx * (jj + ny * k)];
                    if (a >= 0) stamp[a] = stj;
                }
        for (int p = bptr[j]; p < bptr[j + 1]; ++p) { stamp[bcell[p]] = stv; queue[tail++] = bcell[p]; }
        while (head < tail) {
            int i = queue[head++];
            for (int p = rowptr[i]; p < rowptr[i + 1]; ++p) {
                int k = col[p];
                if (stamp[k] == stj) { stamp[k] = stv; queue[tail++] = k; }
            }
        }
        if (used + (size_t)tail > cap) {
            while (used + (size_t)tail > cap) cap *= 2;
            int *nsc = (int *)realloc(sc, cap * sizeof(int));
            if (!nsc) { free(sc); free(sp); free(stamp); free(queue); free(g2a); free(first); free(bptr); free(bcell); return OR_ENOMEM; }
            sc = nsc;
        }
        memcpy(sc + used, queue, (size_t)tail * sizeof(int));
        int m = cells_sorted_unique(sc + used, tail);
        used += (size_t)m;
        sp[j + 1] = (int)used;
    }
    free(stamp); free(queue); free(g2a); free(first); free(bptr); free(bcell);
    *sptr_out = sp;
    *scells_out = sc;
    return OR_OK;
}

/* General-partition rule: S_j = block j plus, for every block k adjacent to
 * j, the cells i of block k with hop(i, block j) <= hop(i, c_k), where c_k
 * is the cell of block k nearest its index-space centroid (lowest index on a
 * tie) and hop counts are breadth-first distances on the connection graph
 * restricted to blocks j and k. */
int or_support_hop(int nx, int ny, int nz, int n, const int *cells, const int *rowptr, const int *col,
                   const int *part, int M, int **sptr_out, int **scells_out) {
    (void)nz;
    int *bptr = (int *)xcalloc((size_t)M + 1, sizeof(int));
    for (int a = 0; a < n; ++a) bptr[part[a] + 1]++;
    for (int j = 0; j < M; ++j) bptr[j + 1] += bptr[j];
    int *bcell = (int *)xmalloc((size_t)n * sizeof(int));
    int *bf = (int *)xmalloc((size_t)M * sizeof(int));
    for (int j = 0; j < M; ++j) bf[j] = bptr[j];
    for (int a = 0; a < n; ++a) bcell[bf[part[a]]++] = a;
    free(bf);
    /* centres */
    int *ctr = (int *)xmalloc((size_t)M * sizeof(int));
    for (int j = 0; j < M; ++j) {
        double sx = 0, sy = 0, sz = 0;
        int m = bptr[j + 1] - bptr[j];
        for (int p = bptr[j]; p < bptr[j + 1]; ++p) {
            int c = cells[bcell[p]];
            sx += c % nx; sy += (c / nx) % ny; sz += c / (nx * ny);
        }
        sx /= m; sy /= m; sz /= m;
        double best = INFINITY;
        int bi = -1;
        for (int p = bptr[j]; p < bptr[j + 1]; ++p) {      /* bcell is ascending within a block */
            int c = cells[bcell[p]];
            double ddx = c % nx - sx, ddy = (c / nx) % ny - sy, ddz = c / (nx * ny) - sz;
            double d2 = ddx * ddx + ddy * ddy + ddz * ddz;
            if (d2 < best) { best = d2; bi = bcell[p]; }
        }
        ctr[j] = bi;
    }
    int *h1 = (int *)xmalloc((size_t)n * sizeof(int));
    int *h2 = (int *)xmalloc((size_t)n * sizeof(int));
    for (int a = 0; a < n; ++a) { h1[a] = -1; h2[a] = -1; }
    int *queue = (int *)xmalloc((size_t)n * sizeof(int));
    int *nbl = (int *)xmalloc((size_t)M * sizeof(int));
    int *nbmark = (int *)xmalloc((size_t)M * sizeof(int));
    for (int j = 0; j < M; ++j) nbmark[j] = -1;
    size_t cap = (size_t)n * 4 + 16, used = 0;
    int *sc = (int *)xmalloc(cap * sizeof(int));
    int *sp = (int *)xmalloc(((size_t)M + 1) * sizeof(int));
    int *tmp = (int *)xmalloc((size_t)n * sizeof(int));
    sp[0] = 0;
    for (int j = 0; j < M; ++j) {
        int nt = 0;
        for (int p = bptr[j]; p < bptr[j + 1]; ++p) tmp[nt++] = bcell[p];
        /* adjacent blocks */
        int nn = 0;
        for (int p = bptr[j]; p < bptr[j + 1]; ++p) {
            int i = bcell[p];
            for (int q = rowptr[i]; q < rowptr[i + 1]; ++q) {
                int k = part[col[q]];
                if (k != j && nbmark[k] != j) { nbmark[k] = j; nbl[nn++] = k; }
            }
        }
        for (int t = 0; t < nn; ++t) {
            int k = nbl[t];
            /* BFS from block j restricted to blocks j, k */
            int head = 0, tail = 0;
            for (int p = bptr[j]; p < bptr[j + 1]; ++p) { h1[bcell[p]] = 0; queue[tail++] = bcell[p]; }
            while (head < tail) {
                int i = queue[head++];
                for (int q = rowptr[i]; q < rowptr[i + 1]; ++q) {
                    int c = col[q], pc = part[c];
                    if ((pc == j || pc == k) && h1[c] < 0) { h1[c] = h1[i] + 1; queue[tail++] = c; }
                }
            }
            int nvis1 = tail;
            /* BFS from c_k restricted to blocks j, k */
            int head2 = 0, tail2 = 0;
            int *qq = (int *)xmalloc((size_t)(bptr[j + 1] - bptr[j] + bptr[k + 1] - bptr[k] + 1) * sizeof(int));
            h2[ctr[k]] = 0;
            qq[tail2++] = ctr[k];
            while (head2 < tail2) {
                int i = qq[head2++];
                for (int q = rowptr[i]; q < rowptr[i + 1]; ++q) {
                    int c = col[q], pc = part[c];
                    if ((pc == j || pc == k) && h2[c] < 0) { h2[c] = h2[i] + 1; qq[tail2++] = c; }
                }
            }
            for (int p = bptr[k]; p < bptr[k + 1]; ++p) {
                int i = bcell[p];
                if (h1[i] >= 0 && (h2[i] < 0 || h1[i] <= h2[i])) tmp[nt++] = i;
            }
            for (int u = 0; u < nvis1; ++u) h1[queue[u]] = -1;
            for (int u = 0; u < tail2; ++u) h2[qq[u]] = -1;
            free(qq);
        }
        int m = cells_sorted_unique(tmp, nt);
        if (used + (size_t)m > cap) {
            while (used + (size_t)m > cap) cap *= 2;
            int *nsc = (int *)realloc(sc, cap * sizeof(int));
            if (!nsc) return OR_ENOMEM;
            sc = nsc;
        }
        memcpy(sc + used, tmp, (size_t)m * sizeof(int));
        used += (size_t)m;
        sp[j + 1] = (int)used;
    }
    free(bptr); free(bcell); free(ctr); free(h1); free(h2); free(queue); free(nbl); free(nbmark); free(tmp);
    *sptr_out = sp;
    *scells_out = sc;
    return OR_OK;
}

/* Support = the block itself (constant basis of the dynamic partitions,
 * Sec. 5.1). */
int or_support_block(int n, const int *part, int M, int **sptr_out, int **scells_out) {
    int *sp = (int *)xcalloc((size_t)M + 1, sizeof(int));
    for (int a = 0; a < n; ++a) sp[part[a] + 1]++;
    for (int j = 0; j < M; ++j) sp[j + 1] += sp[j];
    int *sc = (int *)xmalloc((size_t)n * sizeof(int));
    int *f = (int *)xmalloc((size_t)M * sizeof(int));
    for (int j = 0; j < M; ++j) f[j] = sp[j];
    for (int a = 0; a < n; ++a) sc[f[part[a]]++] = a;
    free(f);
    *sptr_out = sp;
    *scells_out = sc;
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Restriction-smoothed (MsRSB) basis functions (Sec. 5.1: general and      */
/* static partitions use MsRSB bases, computed by iterating on localized    */
/* residual equations).                                                      */
/*                                                                           */
/* Reading: P^0 = block indicator; one iteration updates every basis j on    */
/* its support from the old values,                                          */
/*     P_ij <- P_ij - omega * (A P_j)_i / A_ii      (i in S_j, 0 elsewhere), */
/* then renormalises every cell so that sum_j P_ij = 1 (requirement 3).     */
/* Stops when max |P_new - P_old| < tol or after max_iter iterations.        */
/* A is the unpinned TPFA matrix.  pval is aligned with scells (CSC).       */
/* ------------------------------------------------------------------------ */
int or_msrsb_basis(int n, const int *rowptr, const int *col, const double *val,
                   const int *part, int M, const int *sptr, const int *scells,
                   double omega, double tol, int max_iter,
                   double *pval, int *iters_out, double *inc_hist) {
    int nnzp = sptr[M];
    double *dg = (double *)xmalloc((size_t)n * sizeof(double));
    for (int i = 0; i < n; ++i) {
        int p = diag_pos(rowptr, col, i);
        if (p < 0 || !(val[p] > 0.0)) { free(dg); return OR_EINVAL; }
        dg[i] = val[p];
    }
    for (int j = 0; j < M; ++j)
        for (int e = sptr[j]; e < sptr[j + 1]; ++e) pval[e] = (part[scells[e]] == j) ? 1.0 : 0.0;
    /* entries of each cell in increasing entry order (block order), for the
       per-cell sums of the renormalisation */
    int *cp = (int *)xcalloc((size_t)n + 1, sizeof(int));
    for (int e = 0; e < nnzp; ++e) cp[scells[e] + 1]++;
    for (int i = 0; i < n; ++i) cp[i + 1] += cp[i];
    int *ce = (int *)xmalloc((size_t)nnzp * sizeof(int));
    int *f = (int *)xmalloc((size_t)n * sizeof(int));
    memcpy(f, cp, (size_t)n * sizeof(int));
    for (int e = 0; e < nnzp; ++e) ce[f[scells[e]]++] = e;
    free(f);
    const int nt = OR_THREADS();
    double *w = (double *)xcalloc((size_t)n * nt, sizeof(double));   /* one dense work vector per thread */
    double *pn = (double *)xmalloc((size_t)nnzp * sizeof(double));
    double *rs = (double *)xmalloc((size_t)n * sizeof(double));
    int it = 0;
    while (it < max_iter) {
        OR_PAR_FOR_DYN
        for (int j = 0; j < M; ++j) {
            double *wt = w + (size_t)n * OR_TID();
            for (int e = sptr[j]; e < sptr[j + 1]; ++e) wt[scells[e]] = pval[e];
            for (int e = sptr[j]; e < sptr[j + 1]; ++e) {
                int i = scells[e];
                double ap = 0.0;
                for (int p = rowptr[i]; p < rowptr[i + 1]; ++p) ap += val[p] * wt[col[p]];
                pn[e] = pval[e] - omega * ap / dg[i];
            }
            for (int e = sptr[j]; e < sptr[j + 1]; ++e) wt[scells[e]] = 0.0;
        }
        OR_PAR_FOR
        for (int i = 0; i < n; ++i) {
            double acc = 0.0;
            for (int k = cp[i]; k < cp[i + 1]; ++k) acc += pn[ce[k]];
            rs[i] = acc;
        }
        double inc = 0.0;
        OR_PAR_MAX(inc)
        for (int e = 0; e < nnzp; ++e) {
            double v = pn[e] / rs[scells[e]];
            double d = fabs(v - pval[e]);
            if (d > inc) inc = d;
            pval[e] = v;
        }
        if (inc_hist) inc_hist[it] = inc;
        ++it;
        if (inc < tol) break;
    }
    free(dg); free(w); free(pn); free(rs); free(cp); free(ce);
    *iters_out = it;
    return OR_OK;
}

/* Constant (indicator) basis: P_ij = 1 on block j (dynamic partitions,
 * Sec. 5.1). */
void or_constant_basis(int M, const int *sptr, double *pval) {
    for (int e = 0; e < sptr[M]; ++e) pval[e] = 1.0;
}

/* ------------------------------------------------------------------------ */
/* Galerkin coarse operator A_c = R A P with R = P^T (Eq. (10); Sec. 5,     */
/* Galerkin restriction).  Dense row-major M x M output.                    */
/* ------------------------------------------------------------------------ */
int or_galerkin(int n, const int *rowptr, const int *col, const double *val,
                int M, const int *sptr, const int *scells, const double *pval, double *Ac) {
    /* row view of P: cell -> (block, value) */
    int *cp = (int *)xcalloc((size_t)n + 1, sizeof(int));
    for (int e = 0; e < sptr[M]; ++e) cp[scells[e] + 1]++;
    for (int i = 0; i < n; ++i) cp[i + 1] += cp[i];
    int *cb = (int *)xmalloc((size_t)sptr[M] * sizeof(int));
    double *cv = (double *)xmalloc((size_t)sptr[M] * sizeof(double));
    int *f = (int *)xmalloc((size_t)n * sizeof(int));
    for (int i = 0; i < n; ++i) f[i] = cp[i];
    for (int j = 0; j < M; ++j)
        for (int e = sptr[j]; e < sptr[j + 1]; ++e) { int i = scells[e]; cb[f[i]] = j; cv[f[i]++] = pval[e]; }
    free(f);
    memset(Ac, 0, (size_t)M * M * sizeof(double));
    const int nt = OR_THREADS();                          /* work arrays per thread */
    double *w0 = (double *)xcalloc((size_t)n * nt, sizeof(double));
    int *mark0 = (int *)xmalloc((size_t)n * nt * sizeof(int));
    for (size_t i = 0; i < (size_t)n * nt; ++i) mark0[i] = -1;
    int *lst0 = (int *)xmalloc((size_t)n * nt * sizeof(int));
    OR_PAR_FOR_DYN
    for (int l = 0; l < M; ++l) {                         /* column l of A_c */
        double *w = w0 + (size_t)n * OR_TID();
        int *mark = mark0 + (size_t)n * OR_TID();
        int *lst = lst0 + (size_t)n * OR_TID();
        int nl = 0;
        for (int e = sptr[l]; e < sptr[l + 1]; ++e) w[scells[e]] = pval[e];
        /* cells where (A P_l) may be nonzero: the support and its neighbours */
        for (int e = sptr[l]; e < sptr[l + 1]; ++e) {
            int i = scells[e];
            for (int p = rowptr[i]; p < rowptr[i + 1]; ++p) {
                int k = col[p];
                if (mark[k] != l) { mark[k] = l; lst[nl++] = k; }
            }
        }
        for (int t = 0; t < nl; ++t) {
            int i = lst[t];
            double u = 0.0;
            for (int p = rowptr[i]; p < rowptr[i + 1]; ++p) u += val[p] * w[col[p]];
            for (int q = cp[i]; q < cp[i + 1]; ++q) Ac[(size_t)cb[q] * M + l] += cv[q] * u;
        }
        for (int e = sptr[l]; e < sptr[l + 1]; ++e) w[scells[e]] = 0.0;
    }
    free(cp); free(cb); free(cv); free(w0); free(mark0); free(lst0);
    return OR_OK;
}

/* Dense Cholesky A = L L^T (lower, row-major, in place; upper part zeroed). */
int or_cholesky(int M, double *L) {
    for (int k = 0; k < M; ++k) {
        double d = L[(size_t)k * M + k];
        for (int p = 0; p < k; ++p) d -= L[(size_t)k * M + p] * L[(size_t)k * M + p];
        if (!(d > 0.0)) return OR_ESINGULAR;
        d = sqrt(d);
        L[(size_t)k * M + k] = d;
        OR_PAR_FOR
        for (int i = k + 1; i < M; ++i) {
            double s = L[(size_t)i * M + k];
            for (int p = 0; p < k; ++p) s -= L[(size_t)i * M + p] * L[(size_t)k * M + p];
            L[(size_t)i * M + k] = s / d;
        }
    }
    for (int i = 0; i < M; ++i)
        for (int j = i + 1; j < M; ++j) L[(size_t)i * M + j] = 0.0;
    return OR_OK;
}

/* x = (L L^T)^{-1} b */
void or_cholesky_solve(int M, const double *L, const double *b, double *x) {
    for (int i = 0; i < M; ++i) {
        double s = b[i];
        for (int p = 0; p < i; ++p) s -= L[(size_t)i * M + p] * x[p];
        x[i] = s / L[(size_t)i * M + i];
    }
    for (int i = M - 1; i >= 0; --i) {
        double s = x[i];
        for (int p = i + 1; p < M; ++p) s -= L[(size_t)p * M + i] * x[p];
        x[i] = s / L[(size_t)i * M + i];
    }
}

/* ------------------------------------------------------------------------ */
/* Finite-volume coarse operator (Sec. 5, choice of the restriction: R sums  */
/* the fine cells of each block, R_ji = 1 for i in block j, 0 otherwise;     */
/* Sec. 6.4 b = 1): A_c = R A P, dense row-major M x M, in general not       */
/* symmetric.  part[i] is the block of cell i.                               */
/* ------------------------------------------------------------------------ */
int or_galerkin_fv(int n, const int *rowptr, const int *col, const double *val,
                   int M, const int *sptr, const int *scells, const double *pval, const int *part, double *Ac) {
    memset(Ac, 0, (size_t)M * M * sizeof(double));
    double *w = (double *)xcalloc((size_t)n, sizeof(double));
    int *mark = (int *)xmalloc((size_t)n * sizeof(int));
    for (int i = 0; i < n; ++i) mark[i] = -1;
    int *lst = (int *)xmalloc((size_t)n * sizeof(int));
    for (int l = 0; l < M; ++l) {
        int nl = 0;
        for (int e = sptr[l]; e < sptr[l + 1]; ++e) w[scells[e]] = pval[e];
        for (int e = sptr[l]; e < sptr[l + 1]; ++e) {
            int i = scells[e];
            for (int p = rowptr[i]; p < rowptr[i + 1]; ++p) {
                int k = col[p];
                if (mark[k] != l) { mark[k] = l; lst[nl++] = k; }
            }
        }
        for (int t = 0; t < nl; ++t) {      /* (A P_l)_i lands in row part[i] */
            int i = lst[t];
            double u = 0.0;
            for (int p = rowptr[i]; p < rowptr[i + 1]; ++p) u += val[p] * w[col[p]];
            Ac[(size_t)part[i] * M + l] += u;
        }
        for (int e = sptr[l]; e < sptr[l + 1]; ++e) w[scells[e]] = 0.0;
    }
    free(w); free(mark); free(lst);
    return OR_OK;
}

/* Dense LU with partial pivoting, P A = L U (Gaussian elimination, row     */
/* interchanges choosing the largest |entry| of the column, first such row  */
/* on ties).  In place: U on and above the diagonal, the multipliers of L   */
/* below it; piv[k] = the row exchanged with row k at step k.               */
int or_lu(int M, double *A, int *piv) {
    for (int k = 0; k < M; ++k) {
        int p = k;
        double best = fabs(A[(size_t)k * M + k]);
        for (int i = k + 1; i < M; ++i) {
            double v = fabs(A[(size_t)i * M + k]);
            if (v > best) { best = v; p = i; }
        }
        piv[k] = p;
        if (!(best > 0.0)) return OR_ESINGULAR;
        if (p != k)
            for (int j = 0; j < M; ++j) {
                double t = A[(size_t)k * M + j];
                A[(size_t)k * M + j] = A[(size_t)p * M + j];
                A[(size_t)p * M + j] = t;
            }
        for (int i = k + 1; i < M; ++i) {
            double l = A[(size_t)i * M + k] / A[(size_t)k * M + k];
            A[(size_t)i * M + k] = l;
            for (int j = k + 1; j < M; ++j) A[(size_t)i * M + j] -= l * A[(size_t)k * M + j];
        }
    }
    return OR_OK;
}

/* x = A^{-1} b from or_lu's factors: apply the interchanges to b, then     */
/* L y = P b (unit lower) and U x = y.                                        */
void or_lu_solve(int M, const double *LU, const int *piv, const double *b, double *x) {
    for (int i = 0; i < M; ++i) x[i] = b[i];
    for (int k = 0; k < M; ++k)
        if (piv[k] != k) { double t = x[k]; x[k] = x[piv[k]]; x[piv[k]] = t; }
    for (int i = 0; i < M; ++i) {
        double s = x[i];
        for (int p = 0; p < i; ++p) s -= LU[(size_t)i * M + p] * x[p];
        x[i] = s;
    }
    for (int i = M - 1; i >= 0; --i) {
        double s = x[i];
        for (int p = i + 1; p < M; ++p) s -= LU[(size_t)i * M + p] * x[p];
        x[i] = s / LU[(size_t)i * M + i];
    }
}

/* Well partition (Sec. 6.2, well bases): the perforated cells of well w form */
/* block w, every other cell the one remaining block (index n_wells), which   */
/* keeps the partition of unity.  Returns OR_EINVAL when a cell is listed    */
/* twice or is out of range.                                                 */
int or_partition_wells(int n, int n_wells, const int *wptr, const int *wcells, int *part, int *M_out) {
    for (int i = 0; i < n; ++i) part[i] = -1;
    for (int w = 0; w < n_wells; ++w)
        for (int e = wptr[w]; e < wptr[w + 1]; ++e) {
            int i = wcells[e];
            if (i < 0 || i >= n || part[i] != -1) return OR_EINVAL;
            part[i] = w;
        }
    for (int i = 0; i < n; ++i) if (part[i] == -1) part[i] = n_wells;
    *M_out = n_wells + 1;
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* ILU(0) smoother (Sec. 5.1 smoother S; Sec. 6.4 "Smooth").  Incomplete LU */
/* with zero fill-in on A's pattern, natural row order, IKJ form:           */
/* for each row i, for each k < i in row i: a_ik /= a_kk, then              */
/* a_ij -= a_ik a_kj for every j > k present in both rows.  lu holds L      */
/* (strict lower, unit diagonal implied) and U (upper incl. diagonal).      */
/* ------------------------------------------------------------------------ */
static int find_col(const int *ci, int s, int e, int c) {
    int lo = s, hi = e - 1;
    while (lo <= hi) {
        int m = (lo + hi) >> 1;
        if (ci[m] == c) return m;
        if (ci[m] < c) lo = m + 1; else hi = m - 1;
    }
    return -1;
}

int or_ilu0(int n, const int *rowptr, const int *col, const double *val, double *lu) {
    memcpy(lu, val, (size_t)rowptr[n] * sizeof(double));
    for (int i = 0; i < n; ++i) {
        for (int p = rowptr[i]; p < rowptr[i + 1] && col[p] < i; ++p) {
            int k = col[p];
            int dk = find_col(col, rowptr[k], rowptr[k + 1], k);
            if (dk < 0 || lu[dk] == 0.0) return OR_ESINGULAR;
            lu[p] /= lu[dk];
            for (int q = p + 1; q < rowptr[i + 1]; ++q) {
                int kj = find_col(col, rowptr[k], rowptr[k + 1], col[q]);
                if (kj >= 0) lu[q] -= lu[p] * lu[kj];
            }
        }
        int di = find_col(col, rowptr[i], rowptr[i + 1], i);
        if (di < 0 || lu[di] == 0.0) return OR_ESINGULAR;
    }
    return OR_OK;
}

/* z = (LU)^{-1} r: forward L y = r, then backward U z = y. */
void or_ilu0_apply(int n, const int *rowptr, const int *col, const double *lu, const double *r, double *z) {
    for (int i = 0; i < n; ++i) {
        double s = r[i];
        for (int p = rowptr[i]; p < rowptr[i + 1] && col[p] < i; ++p) s -= lu[p] * z[col[p]];
        z[i] = s;
    }
    for (int i = n - 1; i >= 0; --i) {
        double s = z[i], d = 0.0;
        for (int p = rowptr[i]; p < rowptr[i + 1]; ++p) {
            if (col[p] > i) s -= lu[p] * z[col[p]];
            else if (col[p] == i) d = lu[p];
        }
        z[i] = s / d;
    }
}

/* ------------------------------------------------------------------------ */
/* Iterative multiscale multibasis solver (Eq. (11)) inside a Richardson     */
/* outer loop (Sec. 5.2).  Per cycle, for each stage l in order:             */
/*     x <- x + S(q - A x)                 (one smoother application)        */
/*     x <- x + P^l (A_c^l)^{-1} P^l^T (q - A x)                             */
/* After the cycle, converged when ||q - A x||_2 <= tol ||q||_2.            */
/* Smoother 0 = ILU(0), 1 = Jacobi x += w D^{-1} r.                          */
/* Optional dynamic stage (Sec. 5.1 update schedule): after the cycles in   */
/* the schedule, dp = x^k - x^{k-1} defines a new dynamic partition with a  */
/* constant basis (or an MsRSB basis on hop supports when smoothed) that   */
/* replaces the dynamic stage, which runs after the fixed stages.           */
/* ------------------------------------------------------------------------ */
typedef struct {
    int M;
    const int *sptr;
    const int *scells;
    const double *pval;
    const double *L;     /* Cholesky factor of A_c, or or_lu factors when piv is set (M x M row-major) */
    const int *part;     /* finite volume: block of each cell (restriction R = block indicator); NULL: R = P^T */
    const int *piv;      /* or_lu interchanges (finite volume, or a non-symmetric Galerkin A_c); NULL: Cholesky */
} or_stage;

typedef struct {
    int schedule;        /* 0: none; 1: after every cycle; 2: after cycles 1 and 2 */
    int n_bins;
    double eps;
    int smoothed;        /* 0: constant basis; 1: MsRSB on hop supports */
    double omega;
    double tol;
    int max_iter;
    const double *val_unpinned;   /* for smoothing */
    const int *cells;    /* grid index of each active cell (for hop centres) */
    int nx, ny, nz;
    int *part_out;       /* n: last dynamic partition (or NULL) */
    int *md_hist;        /* max_iter entries: M of the dynamic stage used in each cycle (0 = none) */
} or_adapt;

typedef struct {
    int M;
    int *sptr, *scells;
    double *pval, *L;
} dyn_stage;

static void dyn_free(dyn_stage *d) {
    free(d->sptr); free(d->scells); free(d->pval); free(d->L);
    memset(d, 0, sizeof(*d));
}

static int dyn_build(int n, const int *rp, const int *ci, const double *val, const double *dp,
                     const or_adapt *ad, dyn_stage *d) {
    int *part = (int *)xmalloc((size_t)n * sizeof(int));
    int M, st;
    st = or_partition_dynamic(n, rp, ci, dp, ad->n_bins, ad->eps, part, &M);
    if (st) { free(part); return st; }
    if (ad->part_out) memcpy(ad->part_out, part, (size_t)n * sizeof(int));
    int *sp, *sc;
    if (ad->smoothed) st = or_support_hop(ad->nx, ad->ny, ad->nz, n, ad->cells, rp, ci, part, M, &sp, &sc);
    else st = or_support_block(n, part, M, &sp, &sc);
    if (st) { free(part); return st; }
    double *pv = (double *)xmalloc((size_t)sp[M] * sizeof(double));
    if (ad->smoothed) {
        int its;
        st = or_msrsb_basis(n, rp, ci, ad->val_unpinned, part, M, sp, sc, ad->omega, ad->tol, ad->max_iter, pv, &its, NULL);
    } else {
        or_constant_basis(M, sp, pv);
    }
    free(part);
    if (st) { free(sp); free(sc); free(pv); return st; }
    double *L = (double *)xmalloc((size_t)M * M * sizeof(double));
    or_galerkin(n, rp, ci, val, M, sp, sc, pv, L);
    st = or_cholesky(M, L);
    if (st) { free(sp); free(sc); free(pv); free(L); return st; }
    dyn_free(d);
    d->M = M; d->sptr = sp; d->scells = sc; d->pval = pv; d->L = L;
    return OR_OK;
}

static double nrm2(int n, const double *v) {
    double s = 0.0;
    OR_PAR_SUM(s)
    for (int i = 0; i < n; ++i) s += v[i] * v[i];
    return sqrt(s);
}

static void residual(int n, const int *rp, const int *ci, const double *v, const double *q, const double *x, double *r) {
    csr_mv(n, rp, ci, v, x, r);
    OR_PAR_FOR
    for (int i = 0; i < n; ++i) r[i] = q[i] - r[i];
}

static void coarse_correction(int n, const int *rp, const int *ci, const double *v, const double *q,
                              int M, const int *sptr, const int *scells, const double *pval, const double *L,
                              const int *part, const int *piv, double *x, double *r, double *d, double *xc) {
    residual(n, rp, ci, v, q, x, r);
    if (part) {                                          /* d = R r, R sums each block's cells */
        for (int j = 0; j < M; ++j) d[j] = 0.0;
        for (int i = 0; i < n; ++i) d[part[i]] += r[i];
        or_lu_solve(M, L, piv, d, xc);
    } else {
        OR_PAR_FOR
        for (int j = 0; j < M; ++j) {                   /* d = P^T r */
            double s = 0.0;
            for (int e = sptr[j]; e < sptr[j + 1]; ++e) s += pval[e] * r[scells[e]];
            d[j] = s;
        }
        if (piv) or_lu_solve(M, L, piv, d, xc);        /* non-symmetric A (Galerkin, LU factors) */
        else or_cholesky_solve(M, L, d, xc);
    }
    for (int j = 0; j < M; ++j)                          /* x += P xc */
        for (int e = sptr[j]; e < sptr[j + 1]; ++e) x[scells[e]] += pval[e] * xc[j];
}

int or_ms_solve(int n, const int *rowptr, const int *col, const double *val,
                int n_stages, const or_stage *stages,
                int smoother, const double *lu, double jac_omega,
                const double *q, double *x, double tol, int max_iter,
                or_adapt *adapt, int *iters_out, double *hist) {
    int Mmax = 1;
    for (int s = 0; s < n_stages; ++s) if (stages[s].M > Mmax) Mmax = stages[s].M;
    double *r = (double *)xmalloc((size_t)n * sizeof(double));
    double *z = (double *)xmalloc((size_t)n * sizeof(double));
    double *xprev = (double *)xmalloc((size_t)n * sizeof(double));
    double *dg = (double *)xmalloc((size_t)n * sizeof(double));
    for (int i = 0; i < n; ++i) { int p = diag_pos(rowptr, col, i); dg[i] = p >= 0 ? val[p] : 0.0; }
    dyn_stage dyn;
    memset(&dyn, 0, sizeof(dyn));
    int st = OR_OK;
    double nq = nrm2(n, q);
    residual(n, rowptr, col, val, q, x, r);
    double res = nq > 0 ? nrm2(n, r) / nq : 0.0;
    if (hist) hist[0] = res;
    int it = 0;
    if (nq == 0.0) { for (int i = 0; i < n; ++i) x[i] = 0.0; res = 0.0; }
    double *d = NULL, *xc = NULL;
    while (res > tol && it < max_iter) {
        int Mcur = Mmax > dyn.M ? Mmax : dyn.M;
        free(d); free(xc);
        d = (double *)xmalloc((size_t)Mcur * sizeof(double));
        xc = (double *)xmalloc((size_t)Mcur * sizeof(double));
        memcpy(xprev, x, (size_t)n * sizeof(double));
        int total = n_stages + (dyn.M > 0 ? 1 : 0);
        for (int s = 0; s < total; ++s) {
            residual(n, rowptr, col, val, q, x, r);
            if (smoother == 0) or_ilu0_apply(n, rowptr, col, lu, r, z);
            else for (int i = 0; i < n; ++i) z[i] = jac_omega * r[i] / dg[i];
            OR_PAR_FOR
            for (int i = 0; i < n; ++i) x[i] += z[i];
            if (s < n_stages)
                coarse_correction(n, rowptr, col, val, q, stages[s].M, stages[s].sptr, stages[s].scells,
                                  stages[s].pval, stages[s].L, stages[s].part, stages[s].piv, x, r, d, xc);
            else
                coarse_correction(n, rowptr, col, val, q, dyn.M, dyn.sptr, dyn.scells, dyn.pval, dyn.L,
                                  NULL, NULL, x, r, d, xc);
        }
        if (adapt && adapt->md_hist) adapt->md_hist[it] = dyn.M;
        ++it;
        residual(n, rowptr, col, val, q, x, r);
        res = nrm2(n, r) / nq;
        if (hist) hist[it] = res;
        if (adapt && adapt->schedule && res > tol &&
            (adapt->schedule == 1 || (adapt->schedule == 2 && it <= 2))) {
            for (int i = 0; i < n; ++i) z[i] = x[i] - xprev[i];
            st = dyn_build(n, rowptr, col, val, z, adapt, &dyn);
            if (st) break;
        }
    }
    free(d); free(xc); free(r); free(z); free(xprev); free(dg);
    dyn_free(&dyn);
    *iters_out = it;
    if (st) return st;
    return (res <= tol) ? OR_OK : OR_ENOTCONV;
}

/* Preconditioner of the outer Krylov solve (Sec. 5.2, "Richardson or GMRES"):
 * one multistage cycle applied to v from a zero initial guess, z = M^{-1} v. */
static void ms_cycle_from_zero(int n, const int *rp, const int *ci, const double *val, int n_stages,
                               const or_stage *stages, int smoother, const double *lu, double jac_omega,
                               const double *dg, const double *v, double *z, double *r, double *t, double *d,
                               double *xc) {
    for (int i = 0; i < n; ++i) z[i] = 0.0;
    for (int s = 0; s < n_stages; ++s) {
        residual(n, rp, ci, val, v, z, r);
        if (smoother == 0) or_ilu0_apply(n, rp, ci, lu, r, t);
        else for (int i = 0; i < n; ++i) t[i] = jac_omega * r[i] / dg[i];
        OR_PAR_FOR
        for (int i = 0; i < n; ++i) z[i] += t[i];
        coarse_correction(n, rp, ci, val, v, stages[s].M, stages[s].sptr, stages[s].scells, stages[s].pval,
                          stages[s].L, stages[s].part, stages[s].piv, z, r, d, xc);
    }
}

/* Restarted GMRES(m), right-preconditioned with the multistage cycle and
 * flexible (the preconditioned directions z_j are kept), as in Saad's
 * "Iterative Methods for Sparse Linear Systems", Alg. 9.6.  Arnoldi with
 * classical Gram-Schmidt applied twice; Givens rotations on the Hessenberg
 * columns; the rotated right-hand side gives ||q - A x|| after every step,
 * which is compared with tol ||q|| (hist[k] = that estimate / ||q|| after
 * step k).  At convergence or after m steps, x += Z y and the true residual
 * restarts the cycle.  max_iter bounds the Arnoldi steps (one preconditioner
 * application each). */
int or_ms_gmres(int n, const int *rowptr, const int *col, const double *val,
                int n_stages, const or_stage *stages,
                int smoother, const double *lu, double jac_omega,
                const double *q, double *x, double tol, int max_iter, int m,
                int *iters_out, double *hist) {
    if (m < 1) m = 1;
    int Mmax = 1;
    for (int s = 0; s < n_stages; ++s) if (stages[s].M > Mmax) Mmax = stages[s].M;
    double *V = (double *)xcalloc((size_t)(m + 1) * n, sizeof(double));
    double *Z = (double *)xcalloc((size_t)m * n, sizeof(double));
    double *H = (double *)xcalloc((size_t)(m + 1) * m, sizeof(double));   /* H[i*m + j] */
    double *cs = (double *)xcalloc((size_t)m, sizeof(double));
    double *sn = (double *)xcalloc((size_t)m, sizeof(double));
    double *g = (double *)xcalloc((size_t)m + 1, sizeof(double));
    double *y = (double *)xcalloc((size_t)m, sizeof(double));
    double *h2 = (double *)xcalloc((size_t)m + 1, sizeof(double));
    double *w = (double *)xmalloc((size_t)n * sizeof(double));
    double *r = (double *)xmalloc((size_t)n * sizeof(double));
    double *t = (double *)xmalloc((size_t)n * sizeof(double));
    double *dg = (double *)xmalloc((size_t)n * sizeof(double));
    double *d = (double *)xmalloc((size_t)Mmax * sizeof(double));
    double *xc = (double *)xmalloc((size_t)Mmax * sizeof(double));
    for (int i = 0; i < n; ++i) { int p = diag_pos(rowptr, col, i); dg[i] = p >= 0 ? val[p] : 0.0; }
    const double nq = nrm2(n, q);
    residual(n, rowptr, col, val, q, x, r);
    double res = nq > 0 ? nrm2(n, r) / nq : 0.0;
    if (hist) hist[0] = res;
    if (nq == 0.0) { for (int i = 0; i < n; ++i) x[i] = 0.0; res = 0.0; }
    int it = 0;
    while (res > tol && it < max_iter) {
        const double beta = nrm2(n, r);
        OR_PAR_FOR
        for (int i = 0; i < n; ++i) V[i] = r[i] / beta;
        for (int i = 0; i <= m; ++i) g[i] = 0.0;
        g[0] = beta;
        int k = 0;   /* Arnoldi steps in this restart */
        while (k < m && it < max_iter) {
            const double *vk = V + (size_t)k * n;
            double *zk = Z + (size_t)k * n;
            ms_cycle_from_zero(n, rowptr, col, val, n_stages, stages, smoother, lu, jac_omega, dg, vk, zk, r, t, d, xc);
            csr_mv(n, rowptr, col, val, zk, w);
            for (int i = 0; i <= k; ++i) H[i * m + k] = 0.0;
            for (int pass = 0; pass < 2; ++pass) {       /* h = V^T w; w -= V h (twice) */
                for (int i = 0; i <= k; ++i) {
                    const double *vi = V + (size_t)i * n;
                    double sdot = 0.0;
                    OR_PAR_SUM(sdot)
                    for (int l = 0; l < n; ++l) sdot += vi[l] * w[l];
                    h2[i] = sdot;
                }
                for (int i = 0; i <= k; ++i) {
                    const double *vi = V + (size_t)i * n;
                    OR_PAR_FOR
                    for (int l = 0; l < n; ++l) w[l] -= h2[i] * vi[l];
                    H[i * m + k] += h2[i];
                }
            }
            const double hn = nrm2(n, w);
            H[(k + 1) * m + k] = hn;
            if (hn > 0.0) {
                double *vn = V + (size_t)(k + 1) * n;
                OR_PAR_FOR
                for (int l = 0; l < n; ++l) vn[l] = w[l] / hn;
            }
            for (int i = 0; i < k; ++i) {                 /* previous rotations on column k */
                const double a = H[i * m + k], b = H[(i + 1) * m + k];
                H[i * m + k] = cs[i] * a + sn[i] * b;
                H[(i + 1) * m + k] = -sn[i] * a + cs[i] * b;
            }
            const double a = H[k * m + k], b = H[(k + 1) * m + k];
            const double rho = sqrt(a * a + b * b);
            cs[k] = rho > 0 ? a / rho : 1.0;
            sn[k] = rho > 0 ? b / rho : 0.0;
            H[k * m + k] = rho;
            H[(k + 1) * m + k] = 0.0;
            g[k + 1] = -sn[k] * g[k];
            g[k] = cs[k] * g[k];
            ++k;
            ++it;
            res = fabs(g[k]) / nq;
            if (hist) hist[it] = res;
            if (res <= tol || hn == 0.0) break;
        }
        for (int i = k - 1; i >= 0; --i) {              /* H(0:k,0:k) y = g(0:k) */
            double sacc = g[i];
            for (int l = i + 1; l < k; ++l) sacc -= H[i * m + l] * y[l];
            y[i] = sacc / H[i * m + i];
        }
        for (int i = 0; i < k; ++i) {
            const double *zi = Z + (size_t)i * n;
            OR_PAR_FOR
            for (int l = 0; l < n; ++l) x[l] += y[i] * zi[l];
        }
        residual(n, rowptr, col, val, q, x, r);
        res = nrm2(n, r) / nq;
        if (hist) hist[it] = res;
    }
    free(V); free(Z); free(H); free(cs); free(sn); free(g); free(y); free(h2);
    free(w); free(r); free(t); free(dg); free(d); free(xc);
    *iters_out = it;
    return (res <= tol) ? OR_OK : OR_ENOTCONV;
}

/* ------------------------------------------------------------ two-phase
 * Water / oil with Corey relative permeabilities (Sec. 2 two-phase model):
 * fl = (mu_w, mu_o, n_w, n_o, s_wc, s_or); Se = (S - s_wc)/(1 - s_wc - s_or)
 * clipped to [0, 1], krw = Se^n_w, kro = (1 - Se)^n_o. */
static void mobilities(const double *fl, double S, double *lw, double *lo) {
    double se = (S - fl[4]) / (1.0 - fl[4] - fl[5]);
    if (se < 0.0) se = 0.0;
    if (se > 1.0) se = 1.0;
    *lw = pow(se, fl[2]) / fl[0];
    *lo = pow(1.0 - se, fl[3]) / fl[1];
}

static double fw_of(const double *fl, double S) {
    double lw, lo;
    mobilities(fl, S, &lw, &lo);
    return (lw + lo) > 0.0 ? lw / (lw + lo) : 0.0;
}

void or_total_mobility(int n, const double *S, const double *fl, double *lam) {
    for (int i = 0; i < n; ++i) {
        double lw, lo;
        mobilities(fl, S[i], &lw, &lo);
        lam[i] = lw + lo;
    }
}

/* Largest slope of f_w: central differences on 2000 equal intervals of [0, 1]. */
double or_fw_max_slope(const double *fl) {
    double m = 0.0;
    for (int k = 1; k < 2000; ++k) {
        const double s0 = (double)(k - 1) / 2000.0, s1 = (double)(k + 1) / 2000.0;
        const double d = (fw_of(fl, s1) - fw_of(fl, s0)) / (s1 - s0);
        if (d > m) m = d;
    }
    return m;
}

/* Explicit single-point upstream transport over dt.  The connection
 * transmissibilities (with their face mobilities) are the negated
 * off-diagonals of the unpinned pressure matrix A; u_ij = T_ij (p_i - p_j)
 * leaves cell i.  Per substep of length h:
 *   S_i += h / (phi V) [ q_w,i - sum_j u_ij f_w(S_upstream(i,j)) ],
 * q_w,i = q_i (injection, q_i > 0) or q_i f_w(S_i) (production).  h = dt / k
 * with k the smallest count such that h <= cfl * min_i (phi V / outflow_i) /
 * max f_w', outflow_i = max(-q_i, 0) + sum of positive u_ij. */
int or_transport_step(int n, const int *rowptr, const int *col, const double *val, const double *p,
                      const double *q, double *S, const double *fl, double porosity, double volume, double cfl,
                      double dt, int *nsub_out) {
    const double pv = porosity * volume;
    double tmin = INFINITY;
    for (int i = 0; i < n; ++i) {
        double out = q[i] < 0.0 ? -q[i] : 0.0;
        for (int e = rowptr[i]; e < rowptr[i + 1]; ++e) {
            const int j = col[e];
            if (j == i) continue;
            const double u = -val[e] * (p[i] - p[j]);
            if (u > 0.0) out += u;
        }
        if (out > 0.0 && pv / out < tmin) tmin = pv / out;
    }
    const double slope = or_fw_max_slope(fl);
    const double hmax = slope > 0.0 ? cfl * tmin / slope : INFINITY;
    int k = 1;
    if (dt > 0.0 && isfinite(hmax)) {
        const double c = ceil(dt / hmax);
        if (c >= 1e7) return OR_EINVAL;
        k = c < 1.0 ? 1 : (int)c;
    }
    const double h = dt / k;
    double *Sn = (double *)xmalloc((size_t)n * sizeof(double));
    for (int step = 0; step < k; ++step) {
        for (int i = 0; i < n; ++i) {
            double acc = q[i] > 0.0 ? q[i] : q[i] * fw_of(fl, S[i]);
            for (int e = rowptr[i]; e < rowptr[i + 1]; ++e) {
                const int j = col[e];
                if (j == i) continue;
                const double u = -val[e] * (p[i] - p[j]);
                acc -= u * fw_of(fl, u >= 0.0 ? S[i] : S[j]);
            }
            Sn[i] = S[i] + h / pv * acc;
        }
        memcpy(S, Sn, (size_t)n * sizeof(double));
    }
    free(Sn);
    *nsub_out = k;
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* CPR pressure stage (Sec. 4, quasi-IMPES decoupling; Fig. 3 predictor)    */
/* for a compressible two-phase (water / oil) system, one fully implicit     */
/* time step with primary variables p (Pa) and s = s_w per cell.  Readings:  */
/*   rho_a(p) = rho_a0 exp(c_a (p - p_ref)), phi(p) = phi0 exp(c_r (p - p_ref)); */
/*   lambda_a = kr_a(s) / mu_a with the Corey curves above;                   */
/*   R_a,i = V/dt [phi rho_a s_a - (phi rho_a s_a)^0] + sum_j F_a,ij - q_a,i,  */
/*   F_a,ij = T_ij (lambda_a rho_a)(up) (p_i - p_j), up = the cell with the   */
/*   higher pressure (the lower index on a tie); q_a fixed mass rates.        */
/* cp = (mu_w, mu_o, n_w, n_o, s_wc, s_or, phi0, rho_w0, rho_o0, c_w, c_o,    */
/*       c_r, p_ref).                                                         */
/* ------------------------------------------------------------------------ */
static void cpr_mob(const double *cp, double s, double *lw, double *lo, double *dlw, double *dlo) {
    const double d = 1.0 - cp[4] - cp[5];
    const double x = (s - cp[4]) / d;
    double se = x, dse = 1.0 / d;
    if (x < 0.0) { se = 0.0; dse = 0.0; }          /* clipped: constant mobility */
    else if (x > 1.0) { se = 1.0; dse = 0.0; }
    *lw = pow(se, cp[2]) / cp[0];
    *lo = pow(1.0 - se, cp[3]) / cp[1];
    *dlw = cp[2] * pow(se, cp[2] - 1.0) * dse / cp[0];
    *dlo = -cp[3] * pow(1.0 - se, cp[3] - 1.0) * dse / cp[1];
}

static int cpr_upstream(int a, int b, const double *p) {
    if (p[a] > p[b]) return a;
    if (p[b] > p[a]) return b;
    return a < b ? a : b;
}

/* Residuals R_w, R_o (mass per time). */
void or_cpr_residual(int n, int nf, const int *fa, const int *fb, const double *T, double vol, const double *cp,
                     const double *p, const double *s, const double *p0, const double *s0, const double *qw,
                     const double *qo, double dt, double *Rw, double *Ro) {
    const double phi0 = cp[6], rw0 = cp[7], ro0 = cp[8], cw = cp[9], co = cp[10], cr = cp[11], pr = cp[12];
    for (int i = 0; i < n; ++i) {
        const double ph = phi0 * exp(cr * (p[i] - pr)), ph0 = phi0 * exp(cr * (p0[i] - pr));
        const double rw = rw0 * exp(cw * (p[i] - pr)), rwo = rw0 * exp(cw * (p0[i] - pr));
        const double ro = ro0 * exp(co * (p[i] - pr)), roo = ro0 * exp(co * (p0[i] - pr));
        Rw[i] = vol / dt * (ph * rw * s[i] - ph0 * rwo * s0[i]) - qw[i];
        Ro[i] = vol / dt * (ph * ro * (1.0 - s[i]) - ph0 * roo * (1.0 - s0[i])) - qo[i];
    }
    for (int f = 0; f < nf; ++f) {
        const int a = fa[f], b = fb[f], u = cpr_upstream(a, b, p);
        double lw, lo, dlw, dlo;
        cpr_mob(cp, s[u], &lw, &lo, &dlw, &dlo);
        const double dp = p[a] - p[b];
        const double Fw = T[f] * lw * rw0 * exp(cw * (p[u] - pr)) * dp;
        const double Fo = T[f] * lo * ro0 * exp(co * (p[u] - pr)) * dp;
        Rw[a] += Fw; Rw[b] -= Fw;
        Ro[a] += Fo; Ro[b] -= Fo;
    }
}

/* Jacobian blocks on A's CSR pattern: Jwp = dR_w/dp, Jop = dR_o/dp (full),  */
/* Dws, Dos = the diagonals of dR_w/ds, dR_o/ds; quasi-IMPES weights          */
/* w_w D_ws + w_o D_os = 0, w_w + w_o = 1 per cell; pressure system          */
/* Jstar = W_w Jwp + W_o Jop and rstar = W_w R_w + W_o R_o.                   */
int or_cpr_pressure(int n, const int *rowptr, const int *col, int nf, const int *fa, const int *fb,
                    const double *T, double vol, const double *cp, const double *p, const double *s,
                    const double *p0, const double *s0, const double *qw, const double *qo, double dt,
                    double *Jwp, double *Jop, double *Dws, double *Dos, double *Rw, double *Ro, double *ww,
                    double *wo, double *Jstar, double *rstar) {
    const double phi0 = cp[6], rw0 = cp[7], ro0 = cp[8], cw = cp[9], co = cp[10], cr = cp[11], pr = cp[12];
    const int nnz = rowptr[n];
    for (int e = 0; e < nnz; ++e) { Jwp[e] = 0.0; Jop[e] = 0.0; }
    or_cpr_residual(n, nf, fa, fb, T, vol, cp, p, s, p0, s0, qw, qo, dt, Rw, Ro);
    for (int i = 0; i < n; ++i) {                       /* accumulation */
        const double ph = phi0 * exp(cr * (p[i] - pr));
        const double rw = rw0 * exp(cw * (p[i] - pr)), ro = ro0 * exp(co * (p[i] - pr));
        const int d = diag_pos(rowptr, col, i);
        if (d < 0) return OR_EINVAL;
        Jwp[d] += vol / dt * ph * rw * (cr + cw) * s[i];
        Jop[d] += vol / dt * ph * ro * (cr + co) * (1.0 - s[i]);
        Dws[i] = vol / dt * ph * rw;
        Dos[i] = -vol / dt * ph * ro;
    }
    for (int f = 0; f < nf; ++f) {                      /* fluxes: +F in row a, -F in row b */
        const int a = fa[f], b = fb[f], u = cpr_upstream(a, b, p);
        double lw, lo, dlw, dlo;
        cpr_mob(cp, s[u], &lw, &lo, &dlw, &dlo);
        const double dp = p[a] - p[b];
        const double rwu = rw0 * exp(cw * (p[u] - pr)), rou = ro0 * exp(co * (p[u] - pr));
        const double gw = T[f] * lw * rwu, go = T[f] * lo * rou;
        /* dF/dp_a, dF/dp_b (the density of the upstream cell moves with its pressure) */
        const double wa = gw + (u == a ? dp * T[f] * lw * cw * rwu : 0.0);
        const double wb = -gw + (u == b ? dp * T[f] * lw * cw * rwu : 0.0);
        const double oa = go + (u == a ? dp * T[f] * lo * co * rou : 0.0);
        const double ob = -go + (u == b ? dp * T[f] * lo * co * rou : 0.0);
        const int aa = find_col(col, rowptr[a], rowptr[a + 1], a), ab = find_col(col, rowptr[a], rowptr[a + 1], b);
        const int bb = find_col(col, rowptr[b], rowptr[b + 1], b), ba = find_col(col, rowptr[b], rowptr[b + 1], a);
        if (aa < 0 || ab < 0 || bb < 0 || ba < 0) return OR_EINVAL;
        Jwp[aa] += wa; Jwp[ab] += wb; Jwp[ba] -= wa; Jwp[bb] -= wb;
        Jop[aa] += oa; Jop[ab] += ob; Jop[ba] -= oa; Jop[bb] -= ob;
        /* dF/ds of the upstream cell, on its own row only */
        const double sw = dp * T[f] * dlw * rwu, so = dp * T[f] * dlo * rou;
        if (u == a) { Dws[a] += sw; Dos[a] += so; }
        else { Dws[b] -= sw; Dos[b] -= so; }
    }
    for (int i = 0; i < n; ++i) {
        const double den = Dos[i] - Dws[i];
        if (!(den != 0.0)) return OR_ESINGULAR;
        ww[i] = Dos[i] / den;
        wo[i] = -Dws[i] / den;
        for (int e = rowptr[i]; e < rowptr[i + 1]; ++e) Jstar[e] = ww[i] * Jwp[e] + wo[i] * Jop[e];
        rstar[i] = ww[i] * Rw[i] + wo[i] * Ro[i];
    }
    return OR_OK;
}

/* Operation count of one linear iteration with N_p partitions (Sec. 6.4,
 * Eq. (12)):  c = N [ N_p (4d + 2b + 4) + N_c (d + 1) + N_c (2 d N_c + 1) ]. */
double or_cost_model(double N, double Np, double d, double b, double Nc) {
    return N * (Np * (4.0 * d + 2.0 * b + 4.0) + Nc * (d + 1.0) + Nc * (2.0 * d * Nc + 1.0));
}
