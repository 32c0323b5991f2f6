// ILU(0) smoother (Sec. 5.1 smoother S; Sec. 6.4 "Smooth": two triangular
// solves).  Incomplete LU with zero fill-in on A's pattern in natural row
// order, IKJ form:  for each row i and each k < i in row i (ascending):
// a_ik /= u_kk, then a_ij -= a_ik u_kj for every j > k in both rows.
//
// Three sweep schemes for grids without the structured line sweeps: segment
// dataflow sweeps (the default; chained row runs, one warp scan each),
// level-synchronous sweeps (one cooperative launch, a grid barrier per
// level), and the flag-ordered sweeps below, which also factorise.
//
// Flag-ordered scheme: rows are visited in wavefront-level order (levels padded to
// whole warps so a warp never holds two levels).  Each thread owns one row,
// waits for the rows it depends on through per-row completion flags
// (acquire/release), computes, and publishes its own flag.  CTAs take their
// work in ticket order, so a CTA only ever waits on rows owned by CTAs that
// started before it: the sweep cannot deadlock.  Every wait is bounded; a
// wait that runs out raises an error bit and the sweep drains without
// further waiting.  Flags hold a sweep counter, so no reset pass is needed.
#include "grid_sync.cuh"
#include "ms_internal.h"

namespace msgb {

namespace {

constexpr int kSweepThreads = 128;
constexpr long long kSpinLimit = 1ll << 23;   // x up to 1 us back-off: several seconds at most

__device__ __forceinline__ int ld_acquire(const int *p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(int *p, int v) {
    asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Returns the sweep target value; *vb receives this CTA's ticket.
__device__ __forceinline__ int sweep_begin(int *sync, int *vb) {
    __shared__ int s_vb, s_tgt;
    if (threadIdx.x == 0) {
        s_vb = atomicAdd(&sync[1], 1);
        s_tgt = *((volatile int *)&sync[0]) + 1;
    }
    __syncthreads();
    *vb = s_vb;
    return s_tgt;
}

__device__ __forceinline__ void sweep_end(int *sync) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        int prev = atomicAdd(&sync[2], 1);
        if (prev == (int)gridDim.x - 1) {
            sync[1] = 0;
            sync[2] = 0;
            __threadfence();
            atomicAdd(&sync[0], 1);
        }
    }
}

// Bounded wait for flags[k] == tgt.  Gives up (and stops all later waits)
// once the error word is set.
// Polls back off exponentially (32 ns .. 1 us) so that rows waiting far
// ahead of the wavefront do not saturate L2 with flag reads.
__device__ __forceinline__ int ld_relaxed(const int *p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Relaxed polls with one acquire fence once the flag is seen (an acquire on
// every poll would keep invalidating the SM's L1).
__device__ __forceinline__ bool wait_row(const int *flags, int k, int tgt, int *sync) {
    if (ld_acquire(&flags[k]) == tgt) return true;
    long long spins = 0;
    unsigned ns = 32;
    while (ld_relaxed(&flags[k]) != tgt) {
        ++spins;
        if (spins > 4) {
            __nanosleep(ns);
            ns = ns < 1024 ? 2 * ns : 1024;
        }
        if ((spins & 63) == 0) {
            if (*((volatile int *)&sync[3]) != 0) return false;
            if (spins > kSpinLimit) {
                atomicOr(&sync[3], kErrTimeout);
                return false;
            }
        }
    }
    asm volatile("fence.acq_rel.gpu;" ::: "memory");
    return true;
}

// IKJ ILU(0) of the pinned A (values in FP64).  lu gets L (lower slots) and
// U (upper slots); udiag the U diagonal, dinv its reciprocal.
__global__ void __launch_bounds__(kSweepThreads) k_ilu_factor(int n, int W, int ntot, const int *__restrict__ lperm,
                                                              const int *__restrict__ col,
                                                              const double *__restrict__ off,
                                                              const double *__restrict__ diag, double *lu,
                                                              double *udiag, double *dinv, int *flags, int *sync) {
    int vb;
    const int tgt = sweep_begin(sync, &vb);
    const int t = vb * blockDim.x + threadIdx.x;
    const int i = t < ntot ? lperm[t] : -1;
    if (i >= 0) {
        for (int w = 0; w < W; ++w) lu[(int64_t)w * n + i] = off[(int64_t)w * n + i];
        double d = diag[i];
        bool ok = true;
        for (int w = 0; w < W && ok; ++w) {
            const int k = col[(int64_t)w * n + i];
            if (k >= i) break;     // lower slots come first (ascending); then upper slots / padding
            ok = wait_row(flags, k, tgt, sync);
            if (!ok) break;
            const double ukk = __ldcg(&udiag[k]);
            const double lik = lu[(int64_t)w * n + i] / ukk;
            lu[(int64_t)w * n + i] = lik;
            if (lik == 0.0) continue;
            // a_ij -= l_ik u_kj for j > k present in row k (upper part of row k)
            for (int v = 0; v < W; ++v) {
                const int j = __ldcg(&col[(int64_t)v * n + k]);
                if (j <= k) continue;
                const double ukj = __ldcg(&lu[(int64_t)v * n + k]);
                if (j == i) {
                    d -= lik * ukj;
                } else {
                    for (int w2 = w + 1; w2 < W; ++w2)
                        if (col[(int64_t)w2 * n + i] == j) { lu[(int64_t)w2 * n + i] -= lik * ukj; break; }
                }
            }
        }
        if (!(d != 0.0) || !(d == d)) atomicOr(&sync[3], kErrSingular);
        udiag[i] = d;
        dinv[i] = 1.0 / d;
        st_release(&flags[i], tgt);
    }
    sweep_end(sync);
}

// Forward sweep L y = r (unit lower triangular).
template <typename T, typename TR>
__global__ void __launch_bounds__(kSweepThreads) k_ilu_fwd(int n, int W, int ntot, const int *__restrict__ lperm,
                                                           const int *__restrict__ col, const T *__restrict__ lu,
                                                           const TR *__restrict__ r, T *y, int *flags, int *sync) {
    int vb;
    const int tgt = sweep_begin(sync, &vb);
    const int t = vb * blockDim.x + threadIdx.x;
    const int i = t < ntot ? lperm[t] : -1;
    if (i >= 0) {
        T s = (T)r[i];
        for (int w = 0; w < W; ++w) {
            const int k = col[(int64_t)w * n + i];
            if (k >= i) break;
            if (!wait_row(flags, k, tgt, sync)) break;
            s -= lu[(int64_t)w * n + i] * __ldcg(&y[k]);
        }
        y[i] = s;
        st_release(&flags[i], tgt);
    }
    sweep_end(sync);
}

// Backward sweep U z = y, rows in reverse level order.
template <typename T>
__global__ void __launch_bounds__(kSweepThreads) k_ilu_bwd(int n, int W, int ntot, const int *__restrict__ lperm,
                                                           const int *__restrict__ col, const T *__restrict__ lu,
                                                           const T *__restrict__ dinv, const T *__restrict__ y, T *z,
                                                           int *flags, int *sync) {
    int vb;
    const int tgt = sweep_begin(sync, &vb);
    const int t = vb * blockDim.x + threadIdx.x;
    const int i = t < ntot ? lperm[ntot - 1 - t] : -1;
    if (i >= 0) {
        T s = y[i];
        for (int w = 0; w < W; ++w) {
            const int k = col[(int64_t)w * n + i];
            if (k <= i) continue;
            if (!wait_row(flags, k, tgt, sync)) break;
            s -= lu[(int64_t)w * n + i] * __ldcg(&z[k]);
        }
        z[i] = s * dinv[i];
        st_release(&flags[i], tgt);
    }
    sweep_end(sync);
}

// Level-synchronous sweeps for any grid.  One cooperative launch walks the
// wavefront levels of the natural order (rows of one level are independent):
// the whole grid takes a level's rows, then meets at a grid barrier before the
// next level.  Forward L y = r, or backward (BWD) U z = y in reverse level order.
//
// Barrier: GridSync (bounded; a block that gives up records a timeout and the
// launch ends early).  A row's slots, right-hand side and pivot do not depend on the
// sweep's results, so each thread loads its next row before the barrier; after
// it only the neighbours' results are read.
constexpr int kLevelThreads = 512;
constexpr int kLevelSlots = 8;      // slots held in registers (wider rows take the flag-ordered sweeps)

template <typename T>
struct LevelRow {
    int i;
    int k[kLevelSlots];
    T v[kLevelSlots];
    T r, d;
};

// Row t of lperm (or none) with its slots of the triangle the sweep uses.
template <typename T, typename TR, bool BWD>
__device__ __forceinline__ void level_row_load(LevelRow<T> &row, int t, int e1, int n, int W,
                                               const int *__restrict__ lperm, const int *__restrict__ col,
                                               const T *__restrict__ lu, const T *__restrict__ dinv,
                                               const TR *__restrict__ rhs) {
    row.i = t < e1 ? lperm[t] : -1;
    if (row.i < 0) return;
    const int i = row.i;
    row.r = (T)rhs[i];
    row.d = BWD ? dinv[i] : T(1);
#pragma unroll
    for (int w = 0; w < kLevelSlots; ++w) {
        int k = i;
        T v = T(0);
        if (w < W) {
            k = col[(int64_t)w * n + i];
            v = lu[(int64_t)w * n + i];
        }
        const bool use = BWD ? k > i : k < i;
        row.k[w] = use ? k : -1;
        row.v[w] = v;
    }
}

template <typename T, typename TR, bool BWD>
__global__ void __launch_bounds__(kLevelThreads) k_level_sweep(int n, int W, int nlev, const int *__restrict__ lev_off,
                                                               const int *__restrict__ lperm,
                                                               const int *__restrict__ col, const T *__restrict__ lu,
                                                               const T *__restrict__ dinv,
                                                               const TR *__restrict__ rhs, T *out,
                                                               unsigned long long *bar, int *err) {
    const int G = gridDim.x;
    const int gsize = G * blockDim.x;
    const int j0 = threadIdx.x * G + blockIdx.x;     // rows of a level spread over all blocks first
    GridSync gs;
    gs.begin(bar, err, wait_limit_ns(err));   // err = sync word 3 of the system
    LevelRow<T> row;
    {
        const int L = BWD ? nlev - 1 : 0;
        level_row_load<T, TR, BWD>(row, lev_off[L] + j0, lev_off[L + 1], n, W, lperm, col, lu, dinv, rhs);
    }
    for (int li = 0; li < nlev; ++li) {
        const int L = BWD ? nlev - 1 - li : li;
        if (row.i >= 0) {
            T x[kLevelSlots];
#pragma unroll
            for (int w = 0; w < kLevelSlots; ++w) x[w] = row.k[w] >= 0 ? __ldcg(&out[row.k[w]]) : T(0);
            T s = row.r;
#pragma unroll
            for (int w = 0; w < kLevelSlots; ++w) s -= row.v[w] * x[w];
            out[row.i] = BWD ? s * row.d : s;
        }
        const int e0 = lev_off[L], e1 = lev_off[L + 1];
        for (int t = e0 + j0 + gsize; t < e1; t += gsize) {      // levels wider than the grid
            LevelRow<T> extra;
            level_row_load<T, TR, BWD>(extra, t, e1, n, W, lperm, col, lu, dinv, rhs);
            if (extra.i < 0) continue;
            T s = extra.r;
#pragma unroll
            for (int w = 0; w < kLevelSlots; ++w)
                if (extra.k[w] >= 0) s -= extra.v[w] * __ldcg(&out[extra.k[w]]);
            out[extra.i] = BWD ? s * extra.d : s;
        }
        if (li + 1 == nlev) break;
        const int Ln = BWD ? L - 1 : L + 1;
        level_row_load<T, TR, BWD>(row, lev_off[Ln] + j0, lev_off[Ln + 1], n, W, lperm, col, lu, dinv, rhs);
        if (!gs.sync(nlev - 1)) return;
    }
}

// Segment dataflow sweeps for any grid.  The rows are cut into segments: runs
// of consecutive rows whose only coupling inside the run is the chain (i-1, i)
// (the x-lines of the natural order, cut at inactive cells, at faults that
// couple rows of one line, and every kSegMax rows).  One warp solves one
// segment.  It forms B_i = r_i minus the couplings that leave the segment, then
// solves the chain y_i = B_i + a_i y_{i-1} (a_i = -l_{i,i-1}; backward
// z_i = d_i (y_i - sum_j u_ij z_j) + a_i z_{i+1}, a_i = -d_i u_{i,i+1}, d_i = 1/u_ii)
// by composing the affine maps of each lane's run of rows and scanning the
// compositions across the warp.  Warps take segments one ticket at a time in
// the order of their wavefront levels and stage what does not depend on the
// sweep (right-hand side, chain and coupling values) in shared memory.  Every
// result is also published as tagged 64-bit words (the sweep counter sync[0]
// in the high half, the value's bits in the low half: one word per FP32 value,
// two per FP64 value), so a warp polls the very values it gathers, without
// flags or fences.  A segment only gathers from segments handed out before
// it, so the sweep cannot deadlock and needs no grid-wide barrier; every wait
// is bounded.  Tickets come from sync[1]; sweep_end resets it and advances the
// sweep counter.
constexpr int kSegThreads = 64;          // two warps, one segment each at a time
constexpr int kSegPer = kSegMax / 32;    // rows per lane

__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_relaxed_u64(unsigned long long *p, unsigned long long v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Tagged words of row j (FP64: two words, low and high halves of the value).
template <typename T>
struct SegWord {
    unsigned long long lo, hi;
};

template <typename T>
__device__ __forceinline__ SegWord<T> seg_load(const unsigned long long *tw, int j) {
    SegWord<T> w;
    if constexpr (sizeof(T) == 8) {
        w.lo = ld_relaxed_u64(tw + 2 * (size_t)j);
        w.hi = ld_relaxed_u64(tw + 2 * (size_t)j + 1);
    } else {
        w.lo = ld_relaxed_u64(tw + j);
        w.hi = 0;
    }
    return w;
}

// True, with the value, once the words carry tag tg.
template <typename T>
__device__ __forceinline__ bool seg_check(const SegWord<T> &w, unsigned tg, T &x) {
    if constexpr (sizeof(T) == 8) {
        if ((unsigned)(w.lo >> 32) != tg || (unsigned)(w.hi >> 32) != tg) return false;
        x = __hiloint2double((int)(unsigned)w.hi, (int)(unsigned)w.lo);
    } else {
        if ((unsigned)(w.lo >> 32) != tg) return false;
        x = __uint_as_float((unsigned)w.lo);
    }
    return true;
}

template <typename T>
__device__ __forceinline__ void seg_publish(unsigned long long *tw, int i, unsigned tg, T v) {
    const unsigned long long hi = (unsigned long long)tg << 32;
    if constexpr (sizeof(T) == 8) {
        const unsigned long long b = (unsigned long long)__double_as_longlong(v);
        st_relaxed_u64(tw + 2 * (size_t)i, hi | (b & 0xffffffffull));
        st_relaxed_u64(tw + 2 * (size_t)i + 1, hi | (b >> 32));
    } else {
        st_relaxed_u64(tw + i, hi | __float_as_uint(v));
    }
}

template <typename T>
__device__ __forceinline__ T seg_fma(T a, T b, T c) {
    if constexpr (sizeof(T) == 4) return fmaf(a, b, c);
    else return fma(a, b, c);
}

// Shared memory of one warp: B, a, d, then KG coupling values and KG columns.
template <typename T, int KG>
__host__ __device__ constexpr size_t seg_smem_warp() {
    return (size_t)kSegMax * ((3 + KG) * sizeof(T) + KG * sizeof(int));
}

template <typename T, typename TR, bool BWD, int KG>
__global__ void __launch_bounds__(kSegThreads) k_seg_sweep(int n, int nseg, int kg, const int *__restrict__ seg_off,
                                                           const int *__restrict__ order, const T *__restrict__ ca,
                                                           const int *__restrict__ gcol,
                                                           const T *__restrict__ gval,
                                                           const T *__restrict__ dinv,
                                                           const TR *__restrict__ rhs, T *__restrict__ out,
                                                           unsigned long long *tw, int *sync) {
    extern __shared__ __align__(16) unsigned char seg_smem[];
    const int lane = threadIdx.x & 31;
    T *sb = (T *)(seg_smem + (threadIdx.x >> 5) * seg_smem_warp<T, KG>());
    T *sa = sb + kSegMax;
    T *sd = sa + kSegMax;
    T *sv = sd + kSegMax;                       // [KG][kSegMax]
    int *sc = (int *)(sv + KG * kSegMax);       // [KG][kSegMax]
    __shared__ int s_tgt;
    if (threadIdx.x == 0) s_tgt = *((volatile int *)&sync[0]) + 1;
    __syncthreads();
    const unsigned tg = (unsigned)s_tgt;
    bool failed = false;
    for (;;) {
        int t = 0;
        if (lane == 0) t = atomicAdd(&sync[1], 1);
        t = __shfl_sync(0xffffffffu, t, 0);
        if (t >= nseg) break;
        const int S = order[t];
        const int s0 = seg_off[S], len = seg_off[S + 1] - s0;
        // stage what does not depend on the sweep
#pragma unroll
        for (int c = 0; c < kSegPer; ++c) {
            const int p = c * 32 + lane;
            if (p < len) {
                const int i = s0 + p;
                sb[p] = (T)rhs[i];
                sa[p] = ca[i];
                if (BWD) sd[p] = dinv[i];
#pragma unroll
                for (int q = 0; q < KG; ++q)
                    if (q < kg) {
                        sc[q * kSegMax + p] = gcol[(int64_t)q * n + i];
                        sv[q * kSegMax + p] = gval[(int64_t)q * n + i];
                    }
            }
        }
        __syncwarp();
        // each lane's run of rows (contiguous); the products of the chain
        // coefficients the composition and the shuffle scan need depend only on
        // the factor, so they are formed here, before the couplings arrive:
        // the lane's product and the running product before each scan level
        const int C = (len + 31) >> 5;
        const int lo = lane * C, cnt = max(0, min(C, len - lo));
        T Am[5];
        {
            T A = T(1);   // in the order the rows are composed
            if (!BWD) {
                for (int c = 0; c < cnt; ++c) A *= sa[lo + c];
            } else {
                for (int c = cnt - 1; c >= 0; --c) A *= sa[lo + c];
            }
#pragma unroll
            for (int d = 1, lv = 0; d < 32; d <<= 1, ++lv) {
                Am[lv] = A;
                const T Ap = BWD ? __shfl_down_sync(0xffffffffu, A, d) : __shfl_up_sync(0xffffffffu, A, d);
                if (BWD ? lane + d < 32 : lane >= d) A *= Ap;
            }
        }
        // couplings leaving the segment, in slot order: poll the tagged words of
        // every coupling of the lane's rows in one round of loads until all
        // carry this sweep's tag, then subtract the products
        {
            static_assert(kSegPer * KG <= 32, "pending couplings fit one mask");
            T xv[kSegPer][KG];
            int jv[kSegPer][KG];
            unsigned pend = 0u;
            int qn = 0;   // couplings fill slots from 0: the largest count of the warp's rows
#pragma unroll
            for (int c = 0; c < kSegPer; ++c)
#pragma unroll
                for (int q = 0; q < KG; ++q) {
                    const int p = c * 32 + lane;
                    jv[c][q] = (q < kg && p < len) ? sc[q * kSegMax + p] : -1;
                    xv[c][q] = T(0);
                    if (jv[c][q] >= 0) {
                        pend |= 1u << (c * KG + q);
                        qn = max(qn, q + 1);
                    }
                }
            qn = (int)__reduce_max_sync(0xffffffffu, (unsigned)qn);
            unsigned long long t0 = 0;
            for (int spins = 0; pend && !failed; ++spins) {
                // all loads of the round first, then the tag checks
                SegWord<T> wv[kSegPer][KG];
#pragma unroll
                for (int c = 0; c < kSegPer; ++c)
#pragma unroll
                    for (int q = 0; q < KG; ++q)
                        if ((pend >> (c * KG + q)) & 1u) wv[c][q] = seg_load<T>(tw, jv[c][q]);
                const unsigned was = pend;
#pragma unroll
                for (int c = 0; c < kSegPer; ++c)
#pragma unroll
                    for (int q = 0; q < KG; ++q)
                        if ((was >> (c * KG + q)) & 1u)
                            if (seg_check<T>(wv[c][q], tg, xv[c][q])) pend &= ~(1u << (c * KG + q));
                if (!pend) break;
                if ((spins & 31) == 31) {
                    if (*((volatile int *)&sync[3]) != 0) failed = true;
                    const unsigned long long now = gs_now_ns();
                    if (t0 == 0) t0 = now;
                    else if (now - t0 > wait_limit_ns(sync + 3)) {
                        atomicOr(&sync[3], kErrTimeout);
                        failed = true;
                    }
                }
            }
            // only the slots some row of the warp uses (an FP64 instruction takes
            // the pipe for the whole warp, padding lanes included)
#pragma unroll
            for (int c = 0; c < kSegPer; ++c) {
                const int p = c * 32 + lane;
                if (p < len) {
                    T s = sb[p];
#pragma unroll
                    for (int q = 0; q < KG; ++q)
                        if (q < qn) s -= sv[q * kSegMax + p] * xv[c][q];
                    sb[p] = s;
                }
            }
        }
        if (BWD) {
#pragma unroll
            for (int c = 0; c < kSegPer; ++c) {
                const int p = c * 32 + lane;
                if (p < len) sb[p] *= sd[p];
            }
        }
        __syncwarp();
        // compose the lane's maps (offsets only), scan the compositions across
        // the warp with the products formed above, apply
        T Bc = T(0);
        T av[kSegPer], bv[kSegPer];
        if constexpr (sizeof(T) == 4) {   // rows held in registers
#pragma unroll
            for (int c = 0; c < kSegPer; ++c) {
                av[c] = c < cnt ? sa[lo + c] : T(0);
                bv[c] = c < cnt ? sb[lo + c] : T(0);
            }
#pragma unroll
            for (int k = 0; k < kSegPer; ++k) {
                const int c = BWD ? kSegPer - 1 - k : k;
                if (c < cnt) Bc = seg_fma(av[c], Bc, bv[c]);
            }
        } else {                          // rows read from shared memory
            if (!BWD) {
                for (int c = 0; c < cnt; ++c) Bc = seg_fma(sa[lo + c], Bc, sb[lo + c]);
            } else {
                for (int c = cnt - 1; c >= 0; --c) Bc = seg_fma(sa[lo + c], Bc, sb[lo + c]);
            }
        }
#pragma unroll
        for (int d = 1, lv = 0; d < 32; d <<= 1, ++lv) {
            const T Bp = BWD ? __shfl_down_sync(0xffffffffu, Bc, d) : __shfl_up_sync(0xffffffffu, Bc, d);
            if (BWD ? lane + d < 32 : lane >= d) Bc = seg_fma(Am[lv], Bp, Bc);
        }
        T x = BWD ? __shfl_down_sync(0xffffffffu, Bc, 1) : __shfl_up_sync(0xffffffffu, Bc, 1);
        if (BWD ? lane == 31 : lane == 0) x = T(0);
        if constexpr (sizeof(T) == 4) {
#pragma unroll
            for (int k = 0; k < kSegPer; ++k) {
                const int c = BWD ? kSegPer - 1 - k : k;
                if (c < cnt) {
                    x = seg_fma(av[c], x, bv[c]);
                    sb[lo + c] = x;
                }
            }
        } else {
            if (!BWD) {
                for (int c = 0; c < cnt; ++c) { x = seg_fma(sa[lo + c], x, sb[lo + c]); sb[lo + c] = x; }
            } else {
                for (int c = cnt - 1; c >= 0; --c) { x = seg_fma(sa[lo + c], x, sb[lo + c]); sb[lo + c] = x; }
            }
        }
        __syncwarp();
#pragma unroll
        for (int c = 0; c < kSegPer; ++c) {
            const int p = c * 32 + lane;
            if (p < len) {
                const T v = sb[p];
                out[s0 + p] = v;
                seg_publish<T>(tw, s0 + p, tg, v);
            }
        }
        __syncwarp();
    }
    sweep_end(sync);
}

// Chain coefficients and leaving couplings of every row, in the layout the
// segment sweeps read: v = [a fwd (n)][a bwd (n)][lower values (kgf n)]
// [upper values (kgb n)], gc = [lower columns (kgf n)][upper columns (kgb n)],
// couplings in slot order, padding column -1 with value 0.
template <typename T>
__global__ void k_seg_pack(int n, int W, int kgf, int kgb, const int *__restrict__ seg_id,
                           const int *__restrict__ seg_off, const int *__restrict__ col, const T *__restrict__ lu,
                           const T *__restrict__ dinv, int *__restrict__ gc, T *__restrict__ v) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int S = seg_id[i], s0 = seg_off[S], e0 = seg_off[S + 1];
    int *gcf = gc, *gcb = gc + (size_t)kgf * n;
    T *gvf = v + 2 * (size_t)n, *gvb = gvf + (size_t)kgf * n;
    T af = T(0), ab = T(0);
    int qf = 0, qb = 0;
    for (int w = 0; w < W; ++w) {
        const int k = col[(int64_t)w * n + i];
        if (k == i) continue;
        const T a = lu[(int64_t)w * n + i];
        if (k < i) {
            if (k == i - 1 && i > s0) af = -a;
            else if (qf < kgf) { gcf[(int64_t)qf * n + i] = k; gvf[(int64_t)qf * n + i] = a; ++qf; }
        } else {
            if (k == i + 1 && i + 1 < e0) ab = -dinv[i] * a;
            else if (qb < kgb) { gcb[(int64_t)qb * n + i] = k; gvb[(int64_t)qb * n + i] = a; ++qb; }
        }
    }
    for (; qf < kgf; ++qf) { gcf[(int64_t)qf * n + i] = -1; gvf[(int64_t)qf * n + i] = T(0); }
    for (; qb < kgb; ++qb) { gcb[(int64_t)qb * n + i] = -1; gvb[(int64_t)qb * n + i] = T(0); }
    v[i] = af;
    v[(size_t)n + i] = ab;
}

__global__ void k_copy_f32(const double *a, float *b, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (; i < n; i += (int64_t)gridDim.x * blockDim.x) b[i] = (float)a[i];
}

inline int sweep_blocks(const ms_system &s) { return (s.ntot + kSweepThreads - 1) / kSweepThreads; }

}  // namespace

void launch_ilu_factor(ms_system &s, bool fp32, cudaStream_t st) {
    const size_t en = std::max<size_t>((size_t)s.W * s.n, 1);
    s.lu64.alloc(en);
    s.dinv64.alloc(s.n);
    s.w_y.alloc(s.n);   // U diagonal scratch
    if (!s.ilu64_valid && !launch_ilu_factor_cluster(s, st)) {
        KernelScope ks_(st, "ilu_factor", (double)s.n * (8 + 8 + 8 + 4) + (double)s.W * s.n * (4 + 8 + 8));
        k_ilu_factor<<<sweep_blocks(s), kSweepThreads, 0, st>>>(s.n, s.W, s.ntot, s.lperm.p, s.col.p, s.off_p.p,
                                                                 s.diag.p, s.lu64.p, s.w_y.p, s.dinv64.p, s.flags.p,
                                                                 s.sync.p);
        MS_CHECK_LAUNCH();
    }
    if (fp32) {
        s.lu32.alloc(en);
        s.dinv32.alloc(s.n);
        k_copy_f32<<<1024, 256, 0, st>>>(s.lu64.p, s.lu32.p, (int64_t)en);
        k_copy_f32<<<256, 256, 0, st>>>(s.dinv64.p, s.dinv32.p, s.n);
        MS_CHECK_LAUNCH();
    }
}

void launch_ilu_apply64(ms_system &s, const double *r, double *y, double *z, cudaStream_t st) {
    const double nl = (double)s.nnz_lower;
    {
    KernelScope ks_(st, "ilu_fwd", nl * (4 + 8) + (double)s.n * (8 + 8));
    k_ilu_fwd<double, double><<<sweep_blocks(s), kSweepThreads, 0, st>>>(s.n, s.W, s.ntot, s.lperm.p, s.col.p,
                                                                          s.lu64.p, r, y, s.flags.p, s.sync.p);
    MS_CHECK_LAUNCH();
    }
    KernelScope ks_(st, "ilu_bwd", nl * (4 + 8) + (double)s.n * (8 + 8 + 8));
    k_ilu_bwd<double><<<sweep_blocks(s), kSweepThreads, 0, st>>>(s.n, s.W, s.ntot, s.lperm.p, s.col.p, s.lu64.p,
                                                                 s.dinv64.p, y, z, s.flags.p, s.sync.p);
    MS_CHECK_LAUNCH();
}

void launch_ilu_apply32(ms_system &s, const double *r, float *y, float *z, cudaStream_t st) {
    const double nl = (double)s.nnz_lower;
    {
    KernelScope ks_(st, "ilu_fwd32", nl * (4 + 4) + (double)s.n * (8 + 4));
    k_ilu_fwd<float, double><<<sweep_blocks(s), kSweepThreads, 0, st>>>(s.n, s.W, s.ntot, s.lperm.p, s.col.p,
                                                                         s.lu32.p, r, y, s.flags.p, s.sync.p);
    MS_CHECK_LAUNCH();
    }
    KernelScope ks_(st, "ilu_bwd32", nl * (4 + 4) + (double)s.n * (4 + 4 + 4));
    k_ilu_bwd<float><<<sweep_blocks(s), kSweepThreads, 0, st>>>(s.n, s.W, s.ntot, s.lperm.p, s.col.p, s.lu32.p,
                                                                s.dinv32.p, y, z, s.flags.p, s.sync.p);
    MS_CHECK_LAUNCH();
}

template <typename T, typename TR, bool BWD>
bool launch_level(ms_system &s, const T *lu, const T *dinv, const TR *rhs, T *out, cudaStream_t st) {
    if (s.W > kLevelSlots) return false;
    auto kern = k_level_sweep<T, TR, BWD>;
    static int per_sm = -1;
    if (per_sm < 0) {
        int b = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kern, kLevelThreads, 0) != cudaSuccess) {
            cudaGetLastError();
            b = 0;
        }
        per_sm = b;
    }
    if (per_sm < 1) return false;
    int sms = 0;
    MS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, s.device));
    // one block per SM (fewer arrivals per barrier); small systems fewer
    const int grid = std::max(1, std::min(sms, (s.ntot + kLevelThreads - 1) / kLevelThreads));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kLevelThreads);
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;   // all blocks co-resident (the grid barrier relies on it)
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    const cudaError_t e = cudaLaunchKernelEx(&cfg, kern, s.n, s.W, s.n_levels, (const int *)s.lev_off.p,
                                             (const int *)s.lperm.p, (const int *)s.col.p, lu, dinv, rhs, out,
                                             s.lev_bar.p, s.sync.p + 3);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return true;
}

template <typename T, typename TR>
bool level_apply(ms_system &s, const T *lu, const T *dinv, const TR *r, T *y, T *z, cudaStream_t st) {
    if (s.lev_off.n == 0 || s.W > kLevelSlots) return false;
    const double nl = (double)s.nnz_lower;
    {
        KernelScope ks_(st, sizeof(T) == 8 ? "ilu_level_fwd" : "ilu_level_fwd32", nl * (4 + sizeof(T)) + (double)s.n * (sizeof(TR) + sizeof(T)));
        if (!launch_level<T, TR, false>(s, lu, dinv, r, y, st)) return false;
    }
    KernelScope ks_(st, sizeof(T) == 8 ? "ilu_level_bwd" : "ilu_level_bwd32", nl * (4 + sizeof(T)) + (double)s.n * 3 * sizeof(T));
    return launch_level<T, T, true>(s, lu, dinv, y, z, st);
}

template <typename T, typename TR, bool BWD, int KG>
bool launch_seg_kg(ms_system &s, const T *vals, const T *dinv, const TR *rhs, T *out, cudaStream_t st) {
    auto kern = k_seg_sweep<T, TR, BWD, KG>;
    const size_t smem = (kSegThreads / 32) * seg_smem_warp<T, KG>();
    static size_t cur = 0;
    if (raise_smem_limit(kern, smem, cur) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    const int n = s.n, ns = s.n_seg, kgf = s.seg_kg[0];
    // enough warps for about three levels of segments in flight
    const int warps = std::max(1, std::min(ns, std::max(32, 3 * s.seg_width)));
    const int grid = (warps + kSegThreads / 32 - 1) / (kSegThreads / 32);
    const size_t goff = BWD ? (size_t)kgf * n : 0;
    kern<<<grid, kSegThreads, smem, st>>>(n, ns, s.seg_kg[BWD ? 1 : 0], s.seg_off.p, s.seg_ord.p + (BWD ? ns : 0),
                                          vals + (BWD ? (size_t)n : 0), s.seg_gc.p + goff,
                                          vals + 2 * (size_t)n + goff, dinv, rhs, out, s.seg_tag.p, s.sync.p);
    MS_CHECK_LAUNCH();
    return true;
}

template <typename T, typename TR, bool BWD>
bool launch_seg(ms_system &s, const T *vals, const T *dinv, const TR *rhs, T *out, cudaStream_t st) {
    const int kg = s.seg_kg[BWD ? 1 : 0];
    if (kg <= 2) return launch_seg_kg<T, TR, BWD, 2>(s, vals, dinv, rhs, out, st);
    if (kg <= 4) return launch_seg_kg<T, TR, BWD, 4>(s, vals, dinv, rhs, out, st);
    if (kg <= 8) return launch_seg_kg<T, TR, BWD, 8>(s, vals, dinv, rhs, out, st);
    return false;
}

template <typename T, typename TR>
bool seg_apply(ms_system &s, const T *vals, const T *dinv, const TR *r, T *y, T *z, cudaStream_t st) {
    if (s.n_seg == 0 || vals == nullptr) return false;
    const double nl = (double)s.nnz_lower;
    {
        KernelScope ks_(st, sizeof(T) == 8 ? "ilu_seg_fwd" : "ilu_seg_fwd32",
                        nl * (4 + sizeof(T)) + (double)s.n * (sizeof(TR) + sizeof(T)));
        if (!launch_seg<T, TR, false>(s, vals, dinv, r, y, st)) return false;
    }
    KernelScope ks_(st, sizeof(T) == 8 ? "ilu_seg_bwd" : "ilu_seg_bwd32", nl * (4 + sizeof(T)) + (double)s.n * 3 * sizeof(T));
    return launch_seg<T, T, true>(s, vals, dinv, y, z, st);
}

}  // namespace msgb

namespace msgb {

void launch_ilu_seg_pack(ms_system &s, bool fp32, cudaStream_t st) {
    if (s.n_seg == 0) return;
    const size_t kg = (size_t)s.seg_kg[0] + s.seg_kg[1];
    s.seg_gc.alloc(std::max<size_t>(kg * s.n, 1));
    const int g = (s.n + 255) / 256;
    KernelScope ks_(st, "ilu_seg_pack", (double)s.W * s.n * (4 + (fp32 ? 4 : 8)) + (double)kg * s.n * (4 + (fp32 ? 4 : 8)));
    if (fp32) {
        s.seg_v32.alloc((2 + kg) * s.n);
        k_seg_pack<float><<<g, 256, 0, st>>>(s.n, s.W, s.seg_kg[0], s.seg_kg[1], s.seg_id.p, s.seg_off.p, s.col.p,
                                             s.lu32.p, s.dinv32.p, s.seg_gc.p, s.seg_v32.p);
    } else {
        s.seg_v64.alloc((2 + kg) * s.n);
        k_seg_pack<double><<<g, 256, 0, st>>>(s.n, s.W, s.seg_kg[0], s.seg_kg[1], s.seg_id.p, s.seg_off.p, s.col.p,
                                              s.lu64.p, s.dinv64.p, s.seg_gc.p, s.seg_v64.p);
    }
    MS_CHECK_LAUNCH();
}

bool launch_ilu_seg64(ms_system &s, const double *r, double *y, double *z, cudaStream_t st) {
    return seg_apply<double, double>(s, s.seg_v64.p, s.dinv64.p, r, y, z, st);
}

bool launch_ilu_seg32(ms_system &s, const double *r, float *y, float *z, cudaStream_t st) {
    return seg_apply<float, double>(s, s.seg_v32.p, s.dinv32.p, r, y, z, st);
}

bool launch_ilu_level64(ms_system &s, const double *r, double *y, double *z, cudaStream_t st) {
    return level_apply<double, double>(s, s.lu64.p, s.dinv64.p, r, y, z, st);
}

bool launch_ilu_level32(ms_system &s, const double *r, float *y, float *z, cudaStream_t st) {
    return level_apply<float, double>(s, s.lu32.p, s.dinv32.p, r, y, z, st);
}

// Level-ordered FP64 sweeps with caller-provided scratch: the intermediate
// vector y (n doubles), per-row flags (n ints) and the sweep words (8 ints).
// No tracing scope here: the allocation-free entry point uses this launcher.
void launch_ilu_apply64_scratch(const ms_system &s, const double *r, double *y, double *z, int *flags, int *sync,
                                cudaStream_t st) {
    k_ilu_fwd<double, double><<<sweep_blocks(s), kSweepThreads, 0, st>>>(s.n, s.W, s.ntot, s.lperm.p, s.col.p,
                                                                          s.lu64.p, r, y, flags, sync);
    MS_CHECK_LAUNCH();
    k_ilu_bwd<double><<<sweep_blocks(s), kSweepThreads, 0, st>>>(s.n, s.W, s.ntot, s.lperm.p, s.col.p, s.lu64.p,
                                                                 s.dinv64.p, y, z, flags, sync);
    MS_CHECK_LAUNCH();
}

}  // namespace msgb
