// Dense coarse-system algebra: the coarse solve x_c = A_c^{-1} d of Eq. (11).
//
// A_c (M x M, SPD by Galerkin construction, Eq. (10)) is factored once per
// coarse refresh by a blocked right-looking Cholesky (32-wide panels:
// diagonal block in shared memory, panel triangular solve, trailing
// symmetric update), then inverted as A_c^{-1} = L^{-T} L^{-1} (blocked
// forward substitution on the identity, then a Gram product), so every
// cycle's coarse solve is one dense matrix-vector product.
//
// FP32 path (mixed precision): A_c is symmetrically equilibrated,
// s_i = 1/sqrt(A_ii), factored and inverted in FP32, and the inverse is
// scaled back; the solve refines x_c in FP64 against the FP64 A_c.
//
// Finite-volume stages (A_c = R A P with R the block indicator, not
// symmetric) are inverted by Gauss-Jordan elimination with partial pivoting
// in one cooperative launch (k_gauss_jordan).
#include <cmath>
#include <cstdint>
#include <type_traits>

#include "grid_sync.cuh"
#include "ms_internal.h"

namespace msgb {

namespace {

constexpr int NB = 32;

template <typename T>
__device__ __forceinline__ T dsqrt(T v);
template <>
__device__ __forceinline__ double dsqrt<double>(double v) { return sqrt(v); }
template <>
__device__ __forceinline__ float dsqrt<float>(float v) { return sqrtf(v); }

// Factor the diagonal block A[k0:k0+nb, k0:k0+nb] in place (lower).
// FP64 latency and throughput are scarce on this part: the kernels below
// divide once per pivot (its reciprocal, kept in shared memory) and multiply
// elsewhere.
template <typename T>
__global__ void k_potrf_diag(T *A, int M, int k0, int nb, int *err) {
    __shared__ T a[NB][NB + 1];
    __shared__ T rp;
    const int r = threadIdx.y, c = threadIdx.x;
    if (r < nb && c <= r) a[r][c] = A[(int64_t)(k0 + r) * M + k0 + c];
    for (int p = 0; p < nb; ++p) {
        __syncthreads();
        if (r == p && c == p) {
            T d = a[p][p];
            if (!(d > T(0))) {
                atomicOr(err, kErrSingular);
                d = T(1);
            }
            const T sd = dsqrt<T>(d);
            a[p][p] = sd;
            rp = T(1) / sd;
        }
        __syncthreads();
        if (c == p && r > p && r < nb) a[r][p] *= rp;
        __syncthreads();
        if (r > p && r < nb && c > p && c <= r) a[r][c] -= a[r][p] * a[c][p];
    }
    __syncthreads();
    if (r < nb && c <= r) A[(int64_t)(k0 + r) * M + k0 + c] = a[r][c];
}

// Rows below the diagonal block: L_rk = A_rk L_kk^{-T}, one thread per row by
// forward substitution (x_c = (a_c - sum_{p<c} x_p L_cp) / L_cc).
template <typename T>
__global__ void k_trsm_panel(T *A, int M, int k0, int nb) {
    __shared__ T L[NB][NB + 1];
    __shared__ T rd[NB];
    for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
        const int r = e / NB, c = e % NB;
        L[r][c] = (r < nb && c <= r) ? A[(int64_t)(k0 + r) * M + k0 + c] : T(0);
    }
    __syncthreads();
    if (threadIdx.x < NB) rd[threadIdx.x] = threadIdx.x < nb ? T(1) / L[threadIdx.x][threadIdx.x] : T(0);
    __syncthreads();
    const int row = k0 + nb + blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= M) return;
    T *a = A + (int64_t)row * M + k0;
    T x[NB];
#pragma unroll
    for (int c = 0; c < NB; ++c) x[c] = c < nb ? a[c] : T(0);
#pragma unroll
    for (int c = 0; c < NB; ++c) {
        if (c < nb) {
            T s = x[c];
#pragma unroll
            for (int p = 0; p < c; ++p) s -= x[p] * L[c][p];
            x[c] = s * rd[c];
        }
    }
#pragma unroll
    for (int c = 0; c < NB; ++c)
        if (c < nb) a[c] = x[c];
}

// Trailing update of the lower triangle: A_ij -= sum_p L_ip L_jp over the panel.
template <typename T>
__global__ void k_syrk(T *A, int M, int k0, int nb) {
    const int k1 = k0 + nb;
    const int t = (M - k1 + NB - 1) / NB;
    // lower-triangular tile index
    int idx = blockIdx.x, bi = 0;
    while (idx > bi) { idx -= bi + 1; ++bi; }
    const int bj = idx;
    (void)t;
    __shared__ T Li[NB][NB + 1], Lj[NB][NB + 1];
    const int r = threadIdx.y, c = threadIdx.x;
    const int gi = k1 + bi * NB + r, gj = k1 + bj * NB + r;
    Li[r][c] = (gi < M && c < nb) ? A[(int64_t)gi * M + k0 + c] : T(0);
    Lj[r][c] = (gj < M && c < nb) ? A[(int64_t)gj * M + k0 + c] : T(0);
    __syncthreads();
    const int row = k1 + bi * NB + r, colj = k1 + bj * NB + c;
    if (row < M && colj < M && colj <= row) {
        T s = 0;
#pragma unroll 8
        for (int p = 0; p < NB; ++p) s += Li[r][p] * Lj[c][p];
        A[(int64_t)row * M + colj] -= s;
    }
}

// Y = L^{-1}: right-looking forward substitution on the identity.
// Step 1: rows k0..k0+nb of Y: X = L_kk^{-1} Y_k for columns c < k0+nb.
template <typename T>
__global__ void k_trsm_rows(const T *L, T *Y, int M, int k0, int nb) {
    __shared__ T Lk[NB][NB + 1];
    __shared__ T rd[NB];
    for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
        const int r = e / NB, c = e % NB;
        Lk[r][c] = (r < nb && c <= r) ? L[(int64_t)(k0 + r) * M + k0 + c] : T(0);
    }
    __syncthreads();
    if (threadIdx.x < NB) rd[threadIdx.x] = threadIdx.x < nb ? T(1) / Lk[threadIdx.x][threadIdx.x] : T(0);
    __syncthreads();
    const int cidx = blockIdx.x * blockDim.x + threadIdx.x;
    if (cidx >= k0 + nb) return;
    T x[NB];
#pragma unroll
    for (int r = 0; r < NB; ++r) x[r] = r < nb ? Y[(int64_t)(k0 + r) * M + cidx] : T(0);
#pragma unroll
    for (int r = 0; r < NB; ++r) {
        if (r < nb) {
            T s = x[r];
#pragma unroll
            for (int p = 0; p < r; ++p) s -= Lk[r][p] * x[p];
            x[r] = s * rd[r];
        }
    }
#pragma unroll
    for (int r = 0; r < NB; ++r)
        if (r < nb) Y[(int64_t)(k0 + r) * M + cidx] = x[r];
}

// Step 2: Y[i][c] -= sum_p L[i][k0+p] Y[k0+p][c] for i >= k0+nb, c < k0+nb.
template <typename T>
__global__ void k_trsm_update(const T *L, T *Y, int M, int k0, int nb) {
    const int k1 = k0 + nb;
    __shared__ T Ls[NB][NB + 1], Ys[NB][NB + 1];
    const int r = threadIdx.y, c = threadIdx.x;
    const int gi = k1 + blockIdx.y * NB + r;
    const int gc = blockIdx.x * NB + c;
    Ls[r][c] = (gi < M && c < nb) ? L[(int64_t)gi * M + k0 + c] : T(0);
    Ys[r][c] = (r < nb && gc < k1) ? Y[(int64_t)(k0 + r) * M + gc] : T(0);
    __syncthreads();
    if (gi < M && gc < k1) {
        T s = 0;
#pragma unroll 8
        for (int p = 0; p < NB; ++p) s += Ls[r][p] * Ys[p][c];
        Y[(int64_t)gi * M + gc] -= s;
    }
}

// X = Y^T Y restricted to k >= max(a, b) (Y lower triangular).
template <typename T>
__global__ void k_gram(const T *Y, T *X, int M) {
    __shared__ T Ya[NB][NB + 1], Yb[NB][NB + 1];
    const int r = threadIdx.y, c = threadIdx.x;
    const int a0 = blockIdx.y * NB, b0 = blockIdx.x * NB;
    const int ka = max(a0, b0);
    T s = 0;
    for (int k0 = (ka / NB) * NB; k0 < M; k0 += NB) {
        const int gk = k0 + r;
        Ya[r][c] = (gk < M && a0 + c < M) ? Y[(int64_t)gk * M + a0 + c] : T(0);
        Yb[r][c] = (gk < M && b0 + c < M) ? Y[(int64_t)gk * M + b0 + c] : T(0);
        __syncthreads();
#pragma unroll 8
        for (int p = 0; p < NB; ++p) s += Ya[p][r] * Yb[p][c];
        __syncthreads();
    }
    if (a0 + r < M && b0 + c < M) X[(int64_t)(a0 + r) * M + b0 + c] = s;
}

template <typename T>
__global__ void k_identity(T *Y, int M) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < (int64_t)M * M) Y[e] = (e / M == e % M) ? T(1) : T(0);
}

// FP32 equilibrated copy: S_ij = s_i A_ij s_j with s_i = 1/sqrt(A_ii).
__global__ void k_equilibrate(const double *A, float *S, double *scale, int M) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)M * M) return;
    const int r = (int)(e / M), c = (int)(e % M);
    const double sr = 1.0 / sqrt(A[(int64_t)r * M + r]), sc = 1.0 / sqrt(A[(int64_t)c * M + c]);
    S[e] = (float)(sr * A[e] * sc);
    if (c == 0) scale[r] = sr;
}

__global__ void k_unscale(float *X, const double *scale, int M) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)M * M) return;
    const int r = (int)(e / M), c = (int)(e % M);
    X[e] = (float)((double)X[e] * scale[r] * scale[c]);
}

__global__ void k_check_diag(const double *A, int M, int *err) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < M && !(A[(int64_t)r * M + r] > 0.0)) atomicOr(err, kErrSingular);
}

// y = A x, one warp per row.
// y = A x, one warp per row: 16-byte loads of the row (after the one to three
// elements that bring it to a 16-byte boundary) with kGemvU loads in flight per
// lane, so the row streams instead of waiting on one load at a time.
constexpr int kGemvU = 4;
// MODE 0: y = A x; 1: acc = (double)(A x); 2: acc += (double)(A x).
template <typename T, int MODE>
__global__ void __launch_bounds__(128) k_gemv(const T *__restrict__ A, int M, const T *__restrict__ x,
                                              T *__restrict__ y, double *__restrict__ acc) {
    using V = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
    constexpr int VW = 16 / sizeof(T);
    const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (row >= M) return;
    const T *a = A + (int64_t)row * M;
    int pre = (int)(((16 - ((uintptr_t)a & 15)) & 15) / sizeof(T));
    if (pre > M) pre = M;
    T s[4] = {T(0), T(0), T(0), T(0)};
    if (lane < pre) s[0] = a[lane] * x[lane];
    const int nv = (M - pre) / VW;
    const V *av = (const V *)(a + pre);
    const T *xp = x + pre;
    for (int v0 = lane; v0 < nv; v0 += 32 * kGemvU) {
        V q[kGemvU];
#pragma unroll
        for (int u = 0; u < kGemvU; ++u)
            if (v0 + 32 * u < nv) q[u] = __ldg(av + v0 + 32 * u);
#pragma unroll
        for (int u = 0; u < kGemvU; ++u) {
            const int v = v0 + 32 * u;
            if (v < nv) {
                const T *xv = xp + (int64_t)v * VW;
                if constexpr (VW == 4) s[u & 3] += q[u].x * xv[0] + q[u].y * xv[1] + q[u].z * xv[2] + q[u].w * xv[3];
                else s[u & 3] += q[u].x * xv[0] + q[u].y * xv[1];
            }
        }
    }
    for (int c = pre + nv * VW + lane; c < M; c += 32) s[0] += a[c] * x[c];
    T t = (s[0] + s[1]) + (s[2] + s[3]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    if (lane == 0) {
        if constexpr (MODE == 0) y[row] = t;
        else if constexpr (MODE == 1) acc[row] = (double)t;
        else acc[row] += (double)t;
    }
}

inline int gemv_blocks(int M) { return (M + 3) / 4; }

// Row `row` of A x for one warp, A read-only and x read through L2 (another
// block of the same launch wrote it); the sum is valid in lane 0.
__device__ __forceinline__ float gemv_row_cg(const float *__restrict__ A, int M, int row, const float *x, int lane) {
    const float *a = A + (int64_t)row * M;
    int pre = (int)(((16 - ((uintptr_t)a & 15)) & 15) / sizeof(float));
    if (pre > M) pre = M;
    float s[4] = {0.f, 0.f, 0.f, 0.f};
    if (lane < pre) s[0] = a[lane] * __ldcg(&x[lane]);
    const int nv = (M - pre) / 4;
    const float4 *av = (const float4 *)(a + pre);
    const float *xp = x + pre;
    for (int v0 = lane; v0 < nv; v0 += 32 * kGemvU) {
        float4 q[kGemvU];
#pragma unroll
        for (int u = 0; u < kGemvU; ++u)
            if (v0 + 32 * u < nv) q[u] = __ldg(av + v0 + 32 * u);
#pragma unroll
        for (int u = 0; u < kGemvU; ++u) {
            const int v = v0 + 32 * u;
            if (v < nv) {
                const float *xs = xp + (int64_t)v * 4;
                s[u & 3] += q[u].x * __ldcg(&xs[0]) + q[u].y * __ldcg(&xs[1]) + q[u].z * __ldcg(&xs[2]) + q[u].w * __ldcg(&xs[3]);
            }
        }
    }
    for (int c = pre + nv * 4 + lane; c < M; c += 32) s[0] += a[c] * __ldcg(&x[c]);
    float t = (s[0] + s[1]) + (s[2] + s[3]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    return t;
}

// rc = d - A x (FP64), and its FP32 copy.
__global__ void k_dense_residual(const double *__restrict__ A, int M, const double *__restrict__ d,
                                 const double *__restrict__ x, double *__restrict__ rc, float *__restrict__ rc32) {
    const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (row >= M) return;
    double s = 0;
    const double *a = A + (int64_t)row * M;
    for (int c = lane; c < M; c += 32) s += a[c] * x[c];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) {
        const double r = d[row] - s;
        rc[row] = r;
        rc32[row] = (float)r;
    }
}

// Nonzeros of each row of A_c (one warp per row): the largest count goes to *wmax.
__global__ void k_row_nnz(const double *__restrict__ A, int M, int *__restrict__ wmax) {
    const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (row >= M) return;
    int cnt = 0;
    const double *a = A + (int64_t)row * M;
    for (int c = lane; c < M; c += 32) cnt += a[c] != 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_down_sync(0xffffffffu, cnt, o);
    if (lane == 0) atomicMax(wmax, cnt);
}

// ELL copy of A_c: slot w of row r at [w M + r], columns ascending, padding
// column r with value 0 (one warp per row, compaction by ballot).
__global__ void k_ell_fill(const double *__restrict__ A, int M, int Wc, int *__restrict__ col,
                           double *__restrict__ val) {
    const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (row >= M) return;
    const double *a = A + (int64_t)row * M;
    int base = 0;
    for (int c0 = 0; c0 < M; c0 += 32) {
        const int c = c0 + lane;
        const double v = c < M ? a[c] : 0.0;
        const unsigned b = __ballot_sync(0xffffffffu, v != 0.0);
        const int pos = base + __popc(b & ((1u << lane) - 1u));
        if (v != 0.0 && pos < Wc) {
            col[(int64_t)pos * M + row] = c;
            val[(int64_t)pos * M + row] = v;
        }
        base += __popc(b);
    }
    for (int w = base + lane; w < Wc; w += 32) {
        col[(int64_t)w * M + row] = row;
        val[(int64_t)w * M + row] = 0.0;
    }
}

// rc = d - A x with the ELL copy (FP64), and its FP32 copy.
__global__ void k_ell_residual(const int *__restrict__ col, const double *__restrict__ val, int M, int Wc,
                               const double *__restrict__ d, const double *__restrict__ x, double *__restrict__ rc,
                               float *__restrict__ rc32) {
    const int row = blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= M) return;
    double s = 0.0;
    for (int w = 0; w < Wc; ++w) s += val[(int64_t)w * M + row] * x[col[(int64_t)w * M + row]];
    const double r = d[row] - s;
    rc[row] = r;
    rc32[row] = (float)r;
}

__global__ void k_axpy_f32(int M, const float *t, double *x, int assign) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < M) x[i] = (assign ? 0.0 : x[i]) + (double)t[i];
}

// Test vector v_i = 1 + 0.5 sin(i) for the FP32 inverse quality check.
// test vector with components along every eigenvector: uniform in [-1, 1)
// from a 32-bit integer hash of the index (a mix of odd-constant multiplies
// and xor-shifts)
__global__ void k_test_vector(int M, double *v) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= M) return;
    unsigned h = (unsigned)i * 0x9E3779B1u + 0x7F4A7C15u;
    h ^= h >> 16;
    h *= 0x85EBCA6Bu;
    h ^= h >> 13;
    h *= 0xC2B2AE35u;
    h ^= h >> 16;
    v[i] = (double)h * (2.0 / 4294967296.0) - 1.0;
}

// out[0] = ||x - v||^2, out[1] = ||v||^2 (one CTA, fixed order)
__global__ void k_err_norms(int M, const float *x, const double *v, double *out) {
    __shared__ double a[256], b[256];
    double e = 0.0, w = 0.0;
    for (int i = threadIdx.x; i < M; i += blockDim.x) {
        const double d = (double)x[i] - v[i];
        e += d * d;
        w += v[i] * v[i];
    }
    a[threadIdx.x] = e;
    b[threadIdx.x] = w;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) { a[threadIdx.x] += a[threadIdx.x + o]; b[threadIdx.x] += b[threadIdx.x + o]; }
        __syncthreads();
    }
    if (threadIdx.x == 0) { out[0] = a[0]; out[1] = b[0]; }
}

__global__ void k_d2f(int M, const double *a, float *b) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < M) b[i] = (float)a[i];
}

// ------------------------------------------------- Gauss-Jordan inversion
// Gauss-Jordan elimination with row interchanges (partial pivoting), one
// cooperative launch, the matrix double-buffered: step k reads `cur` and
// writes `nxt`, so no block overwrites what another still reads and one grid
// barrier per step suffices.  Step k, every block:
//   - reduces the per-block candidates of column k to the pivot row p (largest
//     |a_ik| over i >= k, lowest index on ties);
//   - for each of its rows i (block-cyclic), with src = the row that moves to
//     i (rows k and p exchanged): the pivot row scaled by 1 / a_pk into row k;
//     a_src,j - a_src,k a_pj / a_pk elsewhere; column k replaced by the
//     inverse's column (1 / a_pk at row k, -a_src,k / a_pk elsewhere);
//   - gathers its candidates of column k + 1 (double-buffered by parity).
// Every read of data another block wrote goes through L2 (ld.global.cg).
// The interchanges are undone on the columns afterwards (k_gj_order,
// k_gj_gather).  A zero pivot column records kErrSingular and continues
// with a zero reciprocal, so every block passes the same barriers.
constexpr int kGJThreads = 512;
constexpr int kGJRows = 8;     // rows of a block updated together (loads first)
constexpr int kGJCols = 2;     // columns per thread and row in one pass

// Pivot candidates compare |a_ik| through integer keys: the bit pattern of a
// non-negative double (or float) orders like its value, so the search keeps
// off the FP64 pipe, which is narrow on this part.  NaN counts as zero.
__device__ __forceinline__ unsigned long long gj_key(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull;
    return b > 0x7ff0000000000000ull ? 0ull : b;
}
__device__ __forceinline__ unsigned long long gj_key(float x) {
    const unsigned b = __float_as_uint(x) & 0x7fffffffu;
    return b > 0x7f800000u ? 0ull : (unsigned long long)b;
}

__device__ __forceinline__ void gj_better(unsigned long long &bv, int &bi, unsigned long long v, int i) {
    if (v > bv || (v == bv && i < bi)) { bv = v; bi = i; }
}

// Block-wide best candidate; every thread returns it.
__device__ __forceinline__ void gj_block_best(unsigned long long &bv, int &bi) {
    __shared__ unsigned long long s_v[kGJThreads / 32];
    __shared__ int s_i[kGJThreads / 32];
    __shared__ unsigned long long s_bv;
    __shared__ int s_bi;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long v = __shfl_down_sync(0xffffffffu, bv, o);
        const int i = __shfl_down_sync(0xffffffffu, bi, o);
        gj_better(bv, bi, v, i);
    }
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) { s_v[w] = bv; s_i[w] = bi; }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long v = s_v[0];
        int i = s_i[0];
        for (int q = 1; q < (int)(blockDim.x >> 5); ++q) gj_better(v, i, s_v[q], s_i[q]);
        s_bv = v;
        s_bi = i;
    }
    __syncthreads();
    bv = s_bv;
    bi = s_bi;
    __syncthreads();
}

template <typename T>
__global__ void __launch_bounds__(kGJThreads, 1) k_gauss_jordan(int M, T *A0, T *A1, unsigned long long *cand_v, int *cand_i,
                                                                int *piv, unsigned long long *bar, int *err) {
    const int G = gridDim.x;
    GridSync gs;
    gs.begin(bar, err);
    // candidates of column 0 (parity 0)
    {
        unsigned long long bv = 0ull;
        int bi = M;
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < M; i += G * blockDim.x)
            gj_better(bv, bi, gj_key(__ldcg(&A0[(int64_t)i * M])), i);
        gj_block_best(bv, bi);
        if (threadIdx.x == 0) { cand_v[blockIdx.x] = bv; cand_i[blockIdx.x] = bi; }
    }
    if (!gs.sync(M)) return;
    T *cur = A0, *nxt = A1;
    for (int k = 0; k < M; ++k) {
        const int par = k & 1;
        unsigned long long bv = 0ull;
        int bi = M;
        for (int t = threadIdx.x; t < G; t += blockDim.x)
            gj_better(bv, bi, __ldcg(&cand_v[par * G + t]), __ldcg(&cand_i[par * G + t]));
        gj_block_best(bv, bi);
        const bool ok = bv > 0ull && bi < M;
        const int p = ok ? bi : k;
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            piv[k] = p;
            if (!ok) atomicOr(err, kErrSingular);
        }
        const T *prow = cur + (int64_t)p * M;
        const T inv = ok ? T(1) / __ldcg(&prow[k]) : T(0);
        bv = 0ull;
        bi = M;
        for (int i0 = blockIdx.x; i0 < M; i0 += kGJRows * G) {
            int src[kGJRows];
            T f[kGJRows];
#pragma unroll
            for (int r = 0; r < kGJRows; ++r) {
                const int i = i0 + r * G;
                src[r] = i < M ? (i == k ? p : (i == p ? k : i)) : -1;
                f[r] = src[r] >= 0 ? __ldcg(&cur[(int64_t)src[r] * M + k]) : T(0);
            }
            for (int j0 = threadIdx.x; j0 < M; j0 += kGJCols * blockDim.x) {
                T pr[kGJCols];
                T v[kGJRows][kGJCols];
#pragma unroll
                for (int c = 0; c < kGJCols; ++c) {
                    const int j = j0 + c * blockDim.x;
                    pr[c] = j < M ? __ldcg(&prow[j]) : T(0);
#pragma unroll
                    for (int r = 0; r < kGJRows; ++r)
                        v[r][c] = (j < M && src[r] >= 0) ? __ldcg(&cur[(int64_t)src[r] * M + j]) : T(0);
                }
#pragma unroll
                for (int c = 0; c < kGJCols; ++c) {
                    const int j = j0 + c * blockDim.x;
                    if (j >= M) continue;
                    const T sc = pr[c] * inv;           // the scaled pivot row, once per column
#pragma unroll
                    for (int r = 0; r < kGJRows; ++r) {
                        if (src[r] < 0) continue;
                        const int i = i0 + r * G;
                        T x = i == k ? sc : v[r][c] - f[r] * sc;
                        if (j == k) x = i == k ? inv : -f[r] * inv;   // the inverse's column k (one thread)
                        nxt[(int64_t)i * M + j] = x;
                        if (j == k + 1 && i > k) gj_better(bv, bi, gj_key(x), i);
                    }
                }
            }
        }
        if (k + 1 == M) break;
        gj_block_best(bv, bi);
        if (threadIdx.x == 0) {
            cand_v[(par ^ 1) * G + blockIdx.x] = bv;
            cand_i[(par ^ 1) * G + blockIdx.x] = bi;
        }
        if (!gs.sync(M)) return;
        T *t = cur;
        cur = nxt;
        nxt = t;
    }
}

// Column order after the interchanges: undoing them in reverse order on the
// columns of the in-place result gives the inverse.
__global__ void k_gj_order(int M, const int *piv, int *idx) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    for (int j = 0; j < M; ++j) idx[j] = j;
    for (int k = M - 1; k >= 0; --k) {
        const int p = piv[k];
        const int t = idx[k];
        idx[k] = idx[p];
        idx[p] = t;
    }
}

template <typename T>
__global__ void k_gj_gather(int M, const T *__restrict__ A, const int *__restrict__ idx, T *__restrict__ X) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)M * M) return;
    const int r = (int)(e / M), c = (int)(e % M);
    X[e] = A[(int64_t)r * M + idx[c]];
}

// X = A^{-1}; A0 holds A on entry and A1 is scratch of the same size (both
// overwritten).
template <typename T>
void gauss_jordan_inverse(ms_coarse &c, T *A0, T *A1, T *X, int *err, cudaStream_t st) {
    const int M = c.M;
    auto kern = k_gauss_jordan<T>;
    int per_sm = 0, sms = 0, dev = 0;
    MS_CUDA(cudaGetDevice(&dev));
    MS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    MS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kGJThreads, 0));
    MS_REQUIRE(per_sm >= 1, MS_ERR_CUDA, "Gauss-Jordan kernel cannot be resident");
    const int G = std::max(1, std::min(sms, M));
    c.gj_cand_v.alloc(2 * G);
    c.gj_cand_i.alloc(2 * G);
    c.gj_piv.alloc(M);
    c.gj_idx.alloc(M);
    if (c.gj_bar.n == 0) {
        c.gj_bar.alloc(2);
        c.gj_bar.zero(st);
    }
    KernelScope ks_(st, sizeof(T) == 8 ? "coarse_gauss_jordan" : "coarse_gauss_jordan32", 0.0);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(G);
    cfg.blockDim = dim3(kGJThreads);
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;   // the grid barrier needs every block resident
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    MS_CUDA(cudaLaunchKernelEx(&cfg, kern, M, A0, A1, c.gj_cand_v.p, c.gj_cand_i.p, c.gj_piv.p, c.gj_bar.p, err));
    k_gj_order<<<1, 32, 0, st>>>(M, c.gj_piv.p, c.gj_idx.p);
    const int64_t MM = (int64_t)M * M;
    // step k writes A1 when k is even: the last step (k = M - 1) wrote A1 for odd M
    k_gj_gather<T><<<(int)((MM + 255) / 256), 256, 0, st>>>(M, (M & 1) ? A1 : A0, c.gj_idx.p, X);
    MS_CHECK_LAUNCH();
}

template <typename T>
void factor_inverse(T *A, T *Y, T *X, int M, int *err, cudaStream_t st) {
    KernelScope ks_(st, sizeof(T) == 8 ? "coarse_factor_inverse" : "coarse_factor_inverse32", 0.0);
    const dim3 tile(NB, NB);
    for (int k0 = 0; k0 < M; k0 += NB) {
        const int nb = std::min(NB, M - k0);
        k_potrf_diag<T><<<1, tile, 0, st>>>(A, M, k0, nb, err);
        const int rest = M - k0 - nb;
        if (rest > 0) {
            k_trsm_panel<T><<<(rest + 127) / 128, 128, 0, st>>>(A, M, k0, nb);
            const int t = (rest + NB - 1) / NB;
            k_syrk<T><<<t * (t + 1) / 2, tile, 0, st>>>(A, M, k0, nb);
        }
    }
    MS_CHECK_LAUNCH();
    const int64_t MM = (int64_t)M * M;
    k_identity<T><<<(int)((MM + 255) / 256), 256, 0, st>>>(Y, M);
    for (int k0 = 0; k0 < M; k0 += NB) {
        const int nb = std::min(NB, M - k0);
        const int k1 = k0 + nb;
        k_trsm_rows<T><<<(k1 + 127) / 128, 128, 0, st>>>(A, Y, M, k0, nb);
        if (M - k1 > 0) {
            dim3 g((k1 + NB - 1) / NB, (M - k1 + NB - 1) / NB);
            k_trsm_update<T><<<g, tile, 0, st>>>(A, Y, M, k0, nb);
        }
    }
    dim3 g((M + NB - 1) / NB, (M + NB - 1) / NB);
    k_gram<T><<<g, tile, 0, st>>>(Y, X, M);
    MS_CHECK_LAUNCH();
}

}  // namespace

// FP64: work64 holds [L | Y] (2 M^2), inv64 the inverse.
void dense_factor_inverse64(ms_coarse &c, int *err, cudaStream_t st) {
    const int M = c.M;
    const int64_t MM = (int64_t)M * M;
    c.work64.alloc(2 * MM);
    c.inv64.alloc(MM);
    k_check_diag<<<(M + 255) / 256, 256, 0, st>>>(c.Ac.p, M, err);
    MS_CUDA(cudaMemcpyAsync(c.work64.p, c.Ac.p, MM * sizeof(double), cudaMemcpyDeviceToDevice, st));
    factor_inverse<double>(c.work64.p, c.work64.p + MM, c.inv64.p, M, err, st);
}

// FP32: equilibrate, factor and invert in FP32, scale back.
void dense_factor_inverse32(ms_coarse &c, int *err, cudaStream_t st) {
    const int M = c.M;
    const int64_t MM = (int64_t)M * M;
    c.work32.alloc(2 * MM);
    c.inv32.alloc(MM);
    c.work64.alloc(M);   // scale vector
    k_check_diag<<<(M + 255) / 256, 256, 0, st>>>(c.Ac.p, M, err);
    k_equilibrate<<<(int)((MM + 255) / 256), 256, 0, st>>>(c.Ac.p, c.work32.p, c.work64.p, M);
    MS_CHECK_LAUNCH();
    factor_inverse<float>(c.work32.p, c.work32.p + MM, c.inv32.p, M, err, st);
    k_unscale<<<(int)((MM + 255) / 256), 256, 0, st>>>(c.inv32.p, c.work64.p, M);
    MS_CHECK_LAUNCH();
}

// Finite-volume stages: Gauss-Jordan with partial pivoting.  FP64: work64
// holds the two buffers of the matrix being reduced.
void dense_gj_inverse64(ms_coarse &c, int *err, cudaStream_t st) {
    const int M = c.M;
    const int64_t MM = (int64_t)M * M;
    c.work64.alloc(2 * MM);
    c.inv64.alloc(MM);
    MS_CUDA(cudaMemcpyAsync(c.work64.p, c.Ac.p, MM * sizeof(double), cudaMemcpyDeviceToDevice, st));
    gauss_jordan_inverse<double>(c, c.work64.p, c.work64.p + MM, c.inv64.p, err, st);
}

// FP32: equilibrated as the Cholesky path (positive diagonal required; the
// caller checks it first), reduced in FP32, scaled back.
void dense_gj_inverse32(ms_coarse &c, int *err, cudaStream_t st) {
    const int M = c.M;
    const int64_t MM = (int64_t)M * M;
    c.work32.alloc(2 * MM);
    c.inv32.alloc(MM);
    c.work64.alloc(M);   // scale vector
    k_equilibrate<<<(int)((MM + 255) / 256), 256, 0, st>>>(c.Ac.p, c.work32.p, c.work64.p, M);
    MS_CHECK_LAUNCH();
    gauss_jordan_inverse<float>(c, c.work32.p, c.work32.p + MM, c.inv32.p, err, st);
    k_unscale<<<(int)((MM + 255) / 256), 256, 0, st>>>(c.inv32.p, c.work64.p, M);
    MS_CHECK_LAUNCH();
}

void launch_check_diag(const ms_coarse &c, int *err, cudaStream_t st) {
    k_check_diag<<<(c.M + 255) / 256, 256, 0, st>>>(c.Ac.p, c.M, err);
    MS_CHECK_LAUNCH();
}

// Relative error ||inv32 (A_c v) - v|| / ||v||: bounds the contraction of
// the FP64 refinement that uses the FP32 inverse.
double coarse_inverse_check32(const ms_coarse &c, double *host2, cudaStream_t st) {
    const int M = c.M;
    DBuf<double> v, d, out;
    DBuf<float> d32, x32;
    v.alloc(M); d.alloc(M); out.alloc(2); d32.alloc(M); x32.alloc(M);
    k_test_vector<<<(M + 255) / 256, 256, 0, st>>>(M, v.p);
    k_gemv<double, 0><<<gemv_blocks(M), 128, 0, st>>>(c.Ac.p, M, v.p, d.p, nullptr);
    k_d2f<<<(M + 255) / 256, 256, 0, st>>>(M, d.p, d32.p);
    k_gemv<float, 0><<<gemv_blocks(M), 128, 0, st>>>(c.inv32.p, M, d32.p, x32.p, nullptr);
    k_err_norms<<<1, 256, 0, st>>>(M, x32.p, v.p, out.p);
    MS_CHECK_LAUNCH();
    MS_CUDA(cudaMemcpyAsync(host2, out.p, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
    MS_CUDA(cudaStreamSynchronize(st));
    return host2[1] > 0 ? std::sqrt(host2[0] / host2[1]) : 0.0;
}

// The whole mixed-precision coarse solve in one cooperative launch:
//   t = fp32(d); x = inv32 t; then `steps` times: t = fp32(d - A_c x) (FP64,
//   ELL copy of A_c), x += inv32 t,
// phases separated by grid barriers (2 + 2 steps), rows spread over the
// blocks (one warp per row for the products, one thread per row for the
// residuals).  Same arithmetic as the kernel chain of launch_coarse_refine.
__global__ void __launch_bounds__(128) k_refine_coop(const float *__restrict__ inv, int M, const int *__restrict__ ecol,
                                                     const double *__restrict__ eval, int Wc,
                                                     const double *__restrict__ d, double *xc, double *rc, float *t,
                                                     int steps, unsigned long long *bar, int *err) {
    GridSync gs;
    gs.begin(bar, err);
    const int total = 2 + 2 * steps;
    const int G = gridDim.x;
    const int lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
    const int gw = blockIdx.x * wpb + (threadIdx.x >> 5);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < M; i += G * blockDim.x) t[i] = (float)d[i];
    if (!gs.sync(total)) return;
    for (int row = gw; row < M; row += G * wpb) {
        const float v = gemv_row_cg(inv, M, row, t, lane);
        if (lane == 0) xc[row] = (double)v;
    }
    if (!gs.sync(total)) return;
    for (int st = 0; st < steps; ++st) {
        for (int row = blockIdx.x * blockDim.x + threadIdx.x; row < M; row += G * blockDim.x) {
            double sacc = 0.0;
            for (int w = 0; w < Wc; ++w) sacc += eval[(int64_t)w * M + row] * __ldcg(&xc[ecol[(int64_t)w * M + row]]);
            const double r = d[row] - sacc;
            rc[row] = r;
            t[row] = (float)r;
        }
        if (!gs.sync(total)) return;
        for (int row = gw; row < M; row += G * wpb) {
            const float v = gemv_row_cg(inv, M, row, t, lane);
            if (lane == 0) xc[row] += (double)v;
        }
        if (!gs.sync(total)) return;
    }
}

// ELL copy of A_c for the refinement residuals (kept only when A_c is sparse:
// at most M / 4 nonzeros per row).
void coarse_sparse_copy(ms_coarse &c, int *scratch, int *host, cudaStream_t st) {
    const int M = c.M;
    MS_CUDA(cudaMemsetAsync(scratch, 0, sizeof(int), st));
    k_row_nnz<<<(M + 7) / 8, 256, 0, st>>>(c.Ac.p, M, scratch);
    MS_CHECK_LAUNCH();
    MS_CUDA(cudaMemcpyAsync(host, scratch, sizeof(int), cudaMemcpyDeviceToHost, st));
    MS_CUDA(cudaStreamSynchronize(st));
    const int Wc = *host;
    if (Wc <= 0 || Wc > M / 4) {
        c.sp_w = 0;
        return;
    }
    c.sp_col.alloc((size_t)Wc * M);
    c.sp_val.alloc((size_t)Wc * M);
    k_ell_fill<<<(M + 7) / 8, 256, 0, st>>>(c.Ac.p, M, Wc, c.sp_col.p, c.sp_val.p);
    MS_CHECK_LAUNCH();
    c.sp_w = Wc;
    // blocks of the one-launch coarse solve (all resident: grid barriers)
    int dev = 0, sms = 0, per_sm = 0;
    MS_CUDA(cudaGetDevice(&dev));
    MS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    MS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_refine_coop, 128, 0));
    c.coop_blocks = per_sm >= 1 ? std::max(1, std::min(sms, (M + 3) / 4)) : 0;
    if (c.gj_bar.n == 0) {
        c.gj_bar.alloc(2);
        c.gj_bar.zero(st);
    }
    c.refine_err.alloc(1);
    c.refine_err.zero(st);
}

void launch_gemv64(const double *A, int M, const double *x, double *y, cudaStream_t st) {
    KernelScope ks_(st, "coarse_gemv", (double)M * M * 8 + (double)M * 16);
    k_gemv<double, 0><<<gemv_blocks(M), 128, 0, st>>>(A, M, x, y, nullptr);
    MS_CHECK_LAUNCH();
}

void launch_gemv32(const float *A, int M, const float *x, float *y, cudaStream_t st) {
    k_gemv<float, 0><<<gemv_blocks(M), 128, 0, st>>>(A, M, x, y, nullptr);
    MS_CHECK_LAUNCH();
}

// x_c = A_c^{-1} d with the FP32 inverse and `steps` FP64 refinement steps:
// x <- x + inv32 (d - A_c x).
void launch_coarse_refine(const ms_coarse &c, const double *d, double *xc, double *rc, float *t32a, float *t32b,
                          int steps, cudaStream_t st) {
    const int M = c.M;
    if (c.sp_w > 0 && c.coop_blocks > 0 && c.gj_bar.n) {
        KernelScope ks_(st, "coarse_refine", (double)M * M * 4 * (1 + steps) +
                                                 steps * ((double)c.sp_w * M * 12 + (double)M * 24));
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(c.coop_blocks);
        cfg.blockDim = dim3(128);
        cfg.stream = st;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeCooperative;   // grid barriers: every block resident
        at[0].val.cooperative = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        MS_CUDA(cudaLaunchKernelEx(&cfg, k_refine_coop, (const float *)c.inv32.p, M, (const int *)c.sp_col.p,
                                   (const double *)c.sp_val.p, c.sp_w, d, xc, rc, t32a, steps, c.gj_bar.p,
                                   c.refine_err.p));
        return;
    }
    const double resid = c.sp_w > 0 ? (double)c.sp_w * M * 12 + (double)M * 24 : (double)M * M * 8;
    KernelScope ks_(st, "coarse_refine", (double)M * M * 4 * (1 + steps) + steps * resid);
    k_d2f<<<(M + 255) / 256, 256, 0, st>>>(M, d, t32a);
    k_gemv<float, 1><<<gemv_blocks(M), 128, 0, st>>>(c.inv32.p, M, t32a, t32b, xc);
    for (int s = 0; s < steps; ++s) {
        if (c.sp_w > 0) k_ell_residual<<<(M + 127) / 128, 128, 0, st>>>(c.sp_col.p, c.sp_val.p, M, c.sp_w, d, xc, rc, t32a);
        else k_dense_residual<<<(M + 7) / 8, 256, 0, st>>>(c.Ac.p, M, d, xc, rc, t32a);
        k_gemv<float, 2><<<gemv_blocks(M), 128, 0, st>>>(c.inv32.p, M, t32a, t32b, xc);
    }
    MS_CHECK_LAUNCH();
}

}  // namespace msgb
