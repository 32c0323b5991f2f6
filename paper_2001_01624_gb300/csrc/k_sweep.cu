// Dense coarse inverse A_c^{-1} (the coarse solve of Eq. (11); its cost is
// the "solve for p_c" term of Sec. 6.4) by a blocked symmetric sweep in one
// cooperative launch, with the trailing updates on the tensor cores (FP32)
// or the CUDA cores (FP64).
//
// Sweeping an SPD matrix on pivot block K (32 rows and columns) with
// P = A_KK^{-1} replaces
//     A_KK -> -P,   A_iK -> A_iK P,   A_Kj -> P A_Kj,   A_ij -> A_ij - A_iK P A_Kj
// for i, j outside K; the result stays symmetric, and after every block has
// been swept the matrix holds -A^{-1}.  With G the Cholesky factor of A_KK
// and U the column panel of block K with its pivot rows replaced by -I, the
// whole step is one rank-32 update
//     A <- mask_K(A) - W W^T,   W = U G^{-T}   (mask_K zeroes rows and columns of K),
// which is the trailing update of a blocked Cholesky factorisation applied to
// the whole matrix.  Each step of the launch:
//   1. every block factors the 32 x 32 pivot block and inverts its factor
//      (one warp; identical results in every block);
//   2. the blocks form W for disjoint row ranges and publish it (grid barrier);
//   3. every block updates its lower tiles: FP32 -- 128 x 128 tiles, W_I W_J^T
//      on tcgen05 (kind::tf32, operands split into TF32 high and low parts,
//      hi*hi + hi*lo + lo*hi accumulated in FP32 in tensor memory), read back
//      with tcgen05.ld for the masked subtraction; FP64 -- 32 x 32 tiles on
//      the CUDA cores (grid barrier).
// Only tiles on or below the diagonal are updated (the matrix is symmetric);
// an element above the diagonal tiles is read from its mirror.  The padding
// beyond M is the identity, which the sweep leaves decoupled.  A pivot block
// that is not positive definite records kErrSingular; every grid barrier and
// tensor-core wait is bounded and records kErrTimeout.
#include <cmath>

#include "grid_sync.cuh"
#include "ms_internal.h"

namespace msgb {

namespace {

constexpr int kSwNB = 32;        // pivot block: rows and columns eliminated per step
constexpr int kSwThreads = 128;  // four warps (the four TMEM lane quarters)
constexpr int kTcTile = 128;     // FP32 tiles (tensor cores)
constexpr int k64Tile = 32;      // FP64 tiles (CUDA cores)
constexpr int kTcOpBytes = kTcTile * kSwNB * 4;   // one 128 x 32 TF32 operand in shared memory

__device__ __forceinline__ unsigned long long sw_now() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ uint32_t sw_smem(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Symmetric storage: tiles on or below the diagonal are current, so (r, c)
// in a tile above it is read from (c, r).
template <typename T>
__device__ __forceinline__ T sw_get(const T *X, int64_t ld, int tile, int r, int c) {
    return (r / tile >= c / tile) ? __ldcg(&X[(int64_t)r * ld + c]) : __ldcg(&X[(int64_t)c * ld + r]);
}

// Lower tile t (row-major enumeration of tiles with I >= J).
__device__ __forceinline__ void sw_tile(int t, int &I, int &J) {
    int i = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
    while ((i + 1) * (i + 2) / 2 <= t) ++i;
    while (i * (i + 1) / 2 > t) --i;
    I = i;
    J = t - i * (i + 1) / 2;
}

template <typename T>
__device__ __forceinline__ T sw_sqrt(T v);
template <>
__device__ __forceinline__ double sw_sqrt<double>(double v) { return sqrt(v); }
template <>
__device__ __forceinline__ float sw_sqrt<float>(float v) { return sqrtf(v); }

template <typename T>
__device__ __forceinline__ T sw_rsqrt(T v);
template <>
__device__ __forceinline__ double sw_rsqrt<double>(double v) { return rsqrt(v); }
template <>
__device__ __forceinline__ float sw_rsqrt<float>(float v) { return rsqrtf(v); }

// Step 1 (every thread of the block): G = chol(A_KK) in g (lower), the
// reciprocals of its diagonal in rd.  The trailing update of each column is
// spread element by element over the block (no lane idles in a warp
// instruction, which matters for FP64: a warp's FP64 instruction takes the
// pipe for all its lanes); one reciprocal square root per column.
template <typename T>
__device__ void sw_chol(const T *X, int64_t ld, int k0, T (*g)[kSwNB + 1], T *rd, int *err) {
    for (int e = threadIdx.x; e < kSwNB * kSwNB; e += blockDim.x) {
        const int r = e / kSwNB, c = e % kSwNB;
        g[r][c] = c <= r ? __ldcg(&X[(int64_t)(k0 + r) * ld + k0 + c]) : T(0);
    }
    __syncthreads();
    for (int p = 0; p < kSwNB; ++p) {
        // every thread reads the pivot; the column is scaled by its 1/sqrt
        T d = g[p][p];
        const bool bad = !(d > T(0));
        if (bad) d = T(1);
        const T rs = sw_rsqrt<T>(d);
        __syncthreads();
        if (threadIdx.x == 0) {
            g[p][p] = d * rs;
            rd[p] = rs;
            if (bad && blockIdx.x == 0) atomicOr(err, kErrSingular);
        } else if (threadIdx.x > p && threadIdx.x < kSwNB) {
            g[threadIdx.x][p] *= rs;
        }
        __syncthreads();
        // trailing rows/columns p+1..31: lower-triangle element e -> (p+1+rho, p+1+gam)
        const int m = kSwNB - 1 - p;
        for (int e = threadIdx.x; e < m * (m + 1) / 2; e += blockDim.x) {
            int rho = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
            while ((rho + 1) * (rho + 2) / 2 <= e) ++rho;
            while (rho * (rho + 1) / 2 > e) --rho;
            const int r = p + 1 + rho, c = p + 1 + e - rho * (rho + 1) / 2;
            g[r][c] -= g[r][p] * g[c][p];
        }
        __syncthreads();
    }
}

// Step 2: rows [r0, r1) of W = U G^{-T} (U the column panel of block K, its
// pivot rows -I) by forward substitution, one warp per row, lane j holding
// column j: W_j = (U_j - sum_{k<j} G_jk W_k) / G_jj.  Panel values are read
// from the stored (lower) tiles; `put` receives each W_ij.
template <typename T, int TILE, typename Put>
__device__ void sw_w_rows(const T *X, int64_t ld, int k0, int r0, int r1, T (*g)[kSwNB + 1], const T *rd, Put put) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int i = r0 + warp; i < r1; i += nw) {
        T u;
        if (i >= k0 && i < k0 + kSwNB) u = (i - k0 == lane) ? T(-1) : T(0);
        else if (i / TILE >= k0 / TILE) u = __ldcg(&X[(int64_t)i * ld + k0 + lane]);
        else u = __ldcg(&X[(int64_t)(k0 + lane) * ld + i]);   // above the diagonal tiles: the mirror
        T w = T(0);
#pragma unroll
        for (int j = 0; j < kSwNB; ++j) {
            const T wj = __shfl_sync(0xffffffffu, u, j) * rd[j];
            if (lane == j) w = wj;
            if (lane > j) u -= g[lane][j] * wj;
        }
        put(i, lane, w);
    }
}

// -------------------------------------------------------------- tcgen05
__device__ __forceinline__ uint64_t sw_sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;   // descriptor version; no swizzle, base offset 0
    return d;
}

// kind::tf32 instruction descriptor: D F32, A and B TF32, both K-major, M x N.
__host__ __device__ constexpr uint32_t sw_idesc_tf32(int M, int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ float sw_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

__device__ __forceinline__ void sw_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                 " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
                 "l"(a), "l"(b), "r"(idesc), "r"(acc)
                 : "memory");
}

__device__ __forceinline__ void sw_ld32(uint32_t taddr, uint32_t (&v)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,"
        "%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
          "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]),
          "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
          "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Bounded wait for phase `parity` of an mbarrier (1 s); false on timeout.
__device__ __forceinline__ bool sw_mbar_wait(uint64_t *bar, uint32_t parity) {
    unsigned long long t0 = 0;
    for (int spins = 0;; ++spins) {
        uint32_t ok;
        asm volatile("{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
                     : "=r"(ok)
                     : "r"(sw_smem(bar)), "r"(parity)
                     : "memory");
        if (ok) return true;
        if ((spins & 15) == 15) {
            const unsigned long long now = sw_now();
            if (t0 == 0) t0 = now;
            else if (now - t0 > 1000000000ull) return false;
        }
    }
}

// Offset (in floats) of element (r, k) of a 128 x 32 K-major operand in the
// no-swizzle core-matrix layout: 8 x 4 cores of 8 rows x 16 bytes, cores
// adjacent along K 128 B apart (LBO), along M 1024 B apart (SBO).
__host__ __device__ __forceinline__ int sw_core_off(int r, int k) {
    return (r >> 3) * 256 + (k >> 2) * 32 + (r & 7) * 4 + (k & 3);
}

// X: Mp x Mp FP32 (equilibrated A_c, identity padding), swept in place.
// whi / wlo: W as TF32 high / low parts, per 128-row tile in the operand
// layout (nT x 4096 floats each).  inv: M x M output, -X scaled by s_r s_c.
__global__ void __launch_bounds__(kSwThreads, 1)
    k_sweep_tc(int M, int Mp, float *X, float *whi, float *wlo, const double *scale, float *inv,
               unsigned long long *bar, int *err) {
    extern __shared__ __align__(1024) unsigned char sw_dyn[];
    float *op = (float *)sw_dyn;                         // A hi | A lo | B hi | B lo
    float (*g)[kSwNB + 1] = (float (*)[kSwNB + 1])(sw_dyn + 4 * kTcOpBytes);
    float *rd = (float *)(g + kSwNB);
    __shared__ uint32_t s_taddr;
    __shared__ __align__(8) uint64_t s_mbar;
    __shared__ int s_fail;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int G = gridDim.x;
    const int nT = Mp / kTcTile;
    const int nlow = nT * (nT + 1) / 2;
    const int steps = Mp / kSwNB;
    const int per = (Mp + G - 1) / G;
    const int r0 = min(Mp, blockIdx.x * per), r1 = min(Mp, r0 + per);
    const int64_t ld = Mp;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(sw_smem(&s_taddr)),
                     "r"(128u)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        s_fail = 0;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(sw_smem(&s_mbar)), "r"(1u) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t taddr = s_taddr;
    const uint32_t idesc = sw_idesc_tf32(kTcTile, kTcTile);
    uint32_t phase = 0;
    GridSync gs;
    gs.begin(bar, err);
    const int total = 2 * steps;
    bool ok = true;
    for (int st = 0; st < steps && ok; ++st) {
        const int k0 = st * kSwNB;
        sw_chol<float>(X, ld, k0, g, rd, err);
        sw_w_rows<float, kTcTile>(X, ld, k0, r0, r1, g, rd, [&](int i, int j, float w) {
            const int64_t o = (int64_t)(i / kTcTile) * (kTcTile * kSwNB) + sw_core_off(i % kTcTile, j);
            const float h = sw_tf32(w);
            whi[o] = h;
            wlo[o] = sw_tf32(w - h);
        });
        if (!gs.sync(total)) break;
        for (int t = blockIdx.x; t < nlow; t += G) {
            int I, J;
            sw_tile(t, I, J);
            // stage W_I (A) and W_J (B), high and low parts: 4 x 16 KB
            {
                const float4 *src[4] = {(const float4 *)(whi + (int64_t)I * 4096), (const float4 *)(wlo + (int64_t)I * 4096),
                                        (const float4 *)(whi + (int64_t)J * 4096), (const float4 *)(wlo + (int64_t)J * 4096)};
                float4 *dst = (float4 *)op;
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    for (int e = tid; e < 1024; e += kSwThreads) dst[q * 1024 + e] = __ldcg(&src[q][e]);
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncthreads();
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            if (tid == 0) {
                const uint32_t ah = sw_smem(op), al = ah + kTcOpBytes, bh = al + kTcOpBytes, bl = bh + kTcOpBytes;
#pragma unroll
                for (int s = 0; s < kSwNB / 8; ++s)
                    sw_mma(taddr, sw_sdesc(ah + 256 * s, 128, 1024), sw_sdesc(bh + 256 * s, 128, 1024), idesc, s > 0);
#pragma unroll
                for (int s = 0; s < kSwNB / 8; ++s)
                    sw_mma(taddr, sw_sdesc(ah + 256 * s, 128, 1024), sw_sdesc(bl + 256 * s, 128, 1024), idesc, 1);
#pragma unroll
                for (int s = 0; s < kSwNB / 8; ++s)
                    sw_mma(taddr, sw_sdesc(al + 256 * s, 128, 1024), sw_sdesc(bh + 256 * s, 128, 1024), idesc, 1);
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                 sw_smem(&s_mbar))
                             : "memory");
            }
            if (!sw_mbar_wait(&s_mbar, phase)) {
                // the products never completed in a second: record it, give
                // them one more bounded wait before tensor memory is released
                atomicOr(err, kErrTimeout);
                sw_mbar_wait(&s_mbar, phase);
                s_fail = 1;
            }
            phase ^= 1u;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            // masked subtraction: rows of warp `warp`, 32 columns at a time
            const int i = I * kTcTile + warp * 32 + lane;
            const bool rowK = i >= k0 && i < k0 + kSwNB;
            for (int c = 0; c < kTcTile; c += 32) {
                uint32_t v[32];
                sw_ld32(taddr + ((uint32_t)(warp * 32) << 16) + (uint32_t)c, v);
                const int j0 = J * kTcTile + c;
                const bool colK = j0 == k0;   // pivot blocks are 32-aligned: the chunk is all or nothing
                float4 *row = (float4 *)(X + (int64_t)i * ld + j0);
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    float4 x = __ldcg(&row[q]);
                    if (rowK || colK) x = make_float4(0.f, 0.f, 0.f, 0.f);
                    x.x -= __uint_as_float(v[4 * q]);
                    x.y -= __uint_as_float(v[4 * q + 1]);
                    x.z -= __uint_as_float(v[4 * q + 2]);
                    x.w -= __uint_as_float(v[4 * q + 3]);
                    __stcg(&row[q], x);
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncthreads();
            if (s_fail) break;
        }
        if (s_fail) break;
        ok = gs.sync(total);
    }
    // -A^{-1} is in X: unscale into the M x M output
    if (ok && !s_fail) {
        for (int64_t e = (int64_t)blockIdx.x * kSwThreads + tid; e < (int64_t)M * M; e += (int64_t)G * kSwThreads) {
            const int r = (int)(e / M), c = (int)(e % M);
            inv[e] = (float)(-(double)sw_get<float>(X, ld, kTcTile, r, c) * scale[r] * scale[c]);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(128u) : "memory");
}

// FP64: X Mp x Mp (A_c, identity padding), W (Mp x 32 row-major), inv M x M.
__global__ void __launch_bounds__(kSwThreads)
    k_sweep64(int M, int Mp, double *X, double *W, double *inv, unsigned long long *bar, int *err) {
    extern __shared__ __align__(16) unsigned char sw_dyn64[];
    double (*g)[kSwNB + 1] = (double (*)[kSwNB + 1])sw_dyn64;
    double *rd = (double *)(g + kSwNB);
    double (*wi)[kSwNB + 1] = g + kSwNB + 1;
    double (*wj)[kSwNB + 1] = wi + kSwNB;
    const int tid = threadIdx.x;
    const int G = gridDim.x;
    const int nT = Mp / k64Tile;
    const int nlow = nT * (nT + 1) / 2;
    const int steps = Mp / kSwNB;
    const int per = (Mp + G - 1) / G;
    const int r0 = min(Mp, blockIdx.x * per), r1 = min(Mp, r0 + per);
    const int64_t ld = Mp;
    GridSync gs;
    gs.begin(bar, err);
    const int total = 2 * steps;
    bool ok = true;
    // thread -> (row, 8 columns) of a 32 x 32 tile
    const int tr = tid >> 2, tc = (tid & 3) * 8;
    for (int st = 0; st < steps && ok; ++st) {
        const int k0 = st * kSwNB;
        sw_chol<double>(X, ld, k0, g, rd, err);
        sw_w_rows<double, k64Tile>(X, ld, k0, r0, r1, g, rd, [&](int i, int j, double w) { W[(int64_t)i * kSwNB + j] = w; });
        if (!gs.sync(total)) break;
        for (int t = blockIdx.x; t < nlow; t += G) {
            int I, J;
            sw_tile(t, I, J);
            for (int e = tid; e < kSwNB * kSwNB; e += kSwThreads) {
                const int r = e / kSwNB, k = e % kSwNB;
                wi[r][k] = __ldcg(&W[(int64_t)(I * k64Tile + r) * kSwNB + k]);
                wj[r][k] = __ldcg(&W[(int64_t)(J * k64Tile + r) * kSwNB + k]);
            }
            __syncthreads();
            double acc[8];
#pragma unroll
            for (int c = 0; c < 8; ++c) acc[c] = 0.0;
#pragma unroll 4
            for (int k = 0; k < kSwNB; ++k) {
                const double a = wi[tr][k];
#pragma unroll
                for (int c = 0; c < 8; ++c) acc[c] = fma(a, wj[tc + c][k], acc[c]);
            }
            const int i = I * k64Tile + tr, j0 = J * k64Tile + tc;
            const bool mask = (i >= k0 && i < k0 + kSwNB) || (J * k64Tile == k0);
            double2 *row = (double2 *)(X + (int64_t)i * ld + j0);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                double2 x = __ldcg(&row[q]);
                if (mask) x = make_double2(0.0, 0.0);
                x.x -= acc[2 * q];
                x.y -= acc[2 * q + 1];
                __stcg(&row[q], x);
            }
            __syncthreads();
        }
        ok = gs.sync(total);
    }
    if (ok) {
        for (int64_t e = (int64_t)blockIdx.x * kSwThreads + tid; e < (int64_t)M * M; e += (int64_t)G * kSwThreads) {
            const int r = (int)(e / M), c = (int)(e % M);
            inv[e] = -sw_get<double>(X, ld, k64Tile, r, c);
        }
    }
}

__global__ void k_sw_pad64(const double *A, int M, int Mp, double *X) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)Mp * Mp) return;
    const int r = (int)(e / Mp), c = (int)(e % Mp);
    X[e] = (r < M && c < M) ? A[(int64_t)r * M + c] : (r == c ? 1.0 : 0.0);
}

// Equilibrated FP32 copy s_r a_rc s_c (s = 1/sqrt(a_rr)) with identity padding.
__global__ void k_sw_pad32(const double *A, int M, int Mp, const double *scale, float *X) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)Mp * Mp) return;
    const int r = (int)(e / Mp), c = (int)(e % Mp);
    X[e] = (r < M && c < M) ? (float)(A[(int64_t)r * M + c] * scale[r] * scale[c]) : (r == c ? 1.f : 0.f);
}

__global__ void k_sw_scale(const double *A, int M, double *scale) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < M) {
        const double d = A[(int64_t)i * M + i];
        scale[i] = d > 0.0 ? 1.0 / sqrt(d) : 1.0;
    }
}

// Blocks of a sweep launch: one per SM at most, at least 8 (the W rows are
// split over them); every block must be resident (grid barriers).
int sw_blocks(int work) {
    int dev = 0, sms = 0;
    MS_CUDA(cudaGetDevice(&dev));
    MS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    return std::max(1, std::min(sms, std::max(work, 8)));
}

template <typename K>
void sw_check_resident(K kern, size_t smem, int G) {
    int dev = 0, sms = 0, per_sm = 0;
    MS_CUDA(cudaGetDevice(&dev));
    MS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    MS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kSwThreads, smem));
    MS_REQUIRE(per_sm >= 1 && G <= per_sm * sms, MS_ERR_CUDA, "coarse sweep kernel cannot be resident");
}

template <typename K, typename... Args>
void sw_launch(K kern, int G, size_t smem, cudaStream_t st, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(G);
    cfg.blockDim = dim3(kSwThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;   // grid barriers: every block resident
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    MS_CUDA(cudaLaunchKernelEx(&cfg, kern, args...));
}

void sw_bar(ms_coarse &c, cudaStream_t st) {
    if (c.gj_bar.n == 0) {
        c.gj_bar.alloc(2);
        c.gj_bar.zero(st);
    }
}

}  // namespace

// FP64 A_c^{-1} into c.inv64 (work64: the padded matrix and W).
void dense_sweep_inverse64(ms_coarse &c, int *err, cudaStream_t st) {
    const int M = c.M;
    const int Mp = (M + k64Tile - 1) / k64Tile * k64Tile;
    const int64_t PP = (int64_t)Mp * Mp;
    c.work64.alloc(PP + (int64_t)Mp * kSwNB);
    c.inv64.alloc((int64_t)M * M);
    sw_bar(c, st);
    const int nT = Mp / k64Tile;
    const int G = sw_blocks(nT * (nT + 1) / 2);
    const size_t smem = (size_t)(3 * kSwNB + 1) * (kSwNB + 1) * sizeof(double);
    static size_t cur = 0;
    MS_CUDA(raise_smem_limit(k_sweep64, smem, cur));
    sw_check_resident(k_sweep64, smem, G);
    KernelScope ks_(st, "coarse_sweep64", 0.0);
    k_sw_pad64<<<(int)((PP + 255) / 256), 256, 0, st>>>(c.Ac.p, M, Mp, c.work64.p);
    MS_CHECK_LAUNCH();
    sw_launch(k_sweep64, G, smem, st, M, Mp, c.work64.p, c.work64.p + PP, c.inv64.p, c.gj_bar.p, err);
}

// FP32 inverse of the equilibrated A_c on the tensor cores, scaled back into
// c.inv32 (work32: the padded matrix and W's TF32 parts; work64: the scale).
void dense_sweep_inverse32(ms_coarse &c, int *err, cudaStream_t st) {
    const int M = c.M;
    const int Mp = (M + kTcTile - 1) / kTcTile * kTcTile;
    const int64_t PP = (int64_t)Mp * Mp;
    const int nT = Mp / kTcTile;
    c.work32.alloc(PP + 2 * (int64_t)nT * 4096);
    c.work64.alloc(M);
    c.inv32.alloc((int64_t)M * M);
    sw_bar(c, st);
    const int G = sw_blocks(1 << 30);   // one block per SM: the W rows of a step spread over all of them
    const size_t smem = 4 * (size_t)kTcOpBytes + (size_t)(kSwNB + 1) * (kSwNB + 1) * sizeof(float);
    static size_t cur = 0;
    MS_CUDA(raise_smem_limit(k_sweep_tc, smem, cur));
    sw_check_resident(k_sweep_tc, smem, G);
    KernelScope ks_(st, "coarse_sweep_tc", 0.0);
    k_sw_scale<<<(M + 255) / 256, 256, 0, st>>>(c.Ac.p, M, c.work64.p);
    k_sw_pad32<<<(int)((PP + 255) / 256), 256, 0, st>>>(c.Ac.p, M, Mp, c.work64.p, c.work32.p);
    MS_CHECK_LAUNCH();
    sw_launch(k_sweep_tc, G, smem, st, M, Mp, c.work32.p, c.work32.p + PP, c.work32.p + PP + (int64_t)nT * 4096,
              (const double *)c.work64.p, c.inv32.p, c.gj_bar.p, err);
}

}  // namespace msgb
