// ILU(0) triangular sweeps on structured grids, line-scan form.
//
// Natural-order ILU(0) on the 7-point pattern: the forward sweep is
//     y(x,j,k) = r - Lx y(x-1,j,k) - Ly y(x,j-1,k) - Lz y(x,j,k-1),
// the backward sweep the mirror image with U and the reciprocal diagonal.
// Given the two neighbouring x-lines (j-1,k) and (j,k-1), the x-line (j,k)
// is a first-order linear recurrence  v(x) = A(x) v(x-1) + B(x)  in x, which a
// warp solves in parallel: each lane composes the affine maps of its E
// consecutive cells, a 5-round shuffle scan composes the lanes, and each lane
// re-expands its cells.  The result is the exact ILU(0) sweep up to the
// reassociation of these products.  x-lines are contiguous in memory, so
// every load and store is coalesced.
//
// The remaining dependencies form a wavefront over (j, k) lines.  A CTA owns a
// TJ x TK tile of lines; warp w walks the k-row tk = w along j, one line per
// step (line (tj, w) at step tj + w), keeping its previous line in registers
// and passing each finished line to warp w + 1 through double-buffered shared
// memory (one barrier per step).  Line inputs for step s + 1 are fetched with
// per-lane async copies during step s (barriers do not wait on them).  Tiles
// hand over their high j / k face lines as tagged words (payload + sweep
// counter, validated by the consumer) and pace each other with tagged
// per-tile progress hints; tickets follow a topological order of the tile
// grid, and every wait is bounded.
#include "ms_internal.h"

namespace msgb {

namespace {

constexpr long long kSpinLimit = 1ll << 24;
constexpr int EMAX = 8;   // cells per lane: lines up to 256 cells

__device__ __forceinline__ void st_tag(unsigned long long *p, unsigned payload, unsigned tag) {
    const unsigned long long w = ((unsigned long long)tag << 32) | payload;
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(w) : "memory");
}

__device__ __forceinline__ unsigned long long ld_tag(const unsigned long long *p) {
    unsigned long long w;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(w) : "l"(p) : "memory");
    return w;
}

template <int BYTES>
__device__ __forceinline__ void cp_async(void *smem_dst, const void *gsrc, bool valid) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    const int sb = valid ? BYTES : 0;
    if (BYTES == 16)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(gsrc), "r"(sb) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;" ::"r"(d), "l"(gsrc), "n"(BYTES), "r"(sb)
                     : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait0() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

template <typename T>
struct Tag;
template <>
struct Tag<float> {
    __device__ static void put(unsigned long long *p, float v, unsigned tag) { st_tag(p, __float_as_uint(v), tag); }
    __device__ static bool ok(const unsigned long long *w, unsigned tag) { return (unsigned)(w[0] >> 32) == tag; }
    __device__ static float value(const unsigned long long *w) { return __uint_as_float((unsigned)w[0]); }
};
template <>
struct Tag<double> {
    __device__ static void put(unsigned long long *p, double v, unsigned tag) {
        const unsigned long long b = (unsigned long long)__double_as_longlong(v);
        st_tag(p, (unsigned)b, tag);
        st_tag(p + 1, (unsigned)(b >> 32), tag);
    }
    __device__ static bool ok(const unsigned long long *w, unsigned tag) {
        return (unsigned)(w[0] >> 32) == tag && (unsigned)(w[1] >> 32) == tag;
    }
    __device__ static double value(const unsigned long long *w) {
        return __longlong_as_double((long long)(((w[1] & 0xffffffffull) << 32) | (w[0] & 0xffffffffull)));
    }
};

// Read a tagged value from global memory, waiting (bounded) for this sweep's tag.
template <typename T>
__device__ __forceinline__ T take_tagged(const unsigned long long *p, unsigned tag, int *sync) {
    unsigned long long w[2];
    long long spins = 0;
    while (true) {
        w[0] = ld_tag(p);
        w[1] = sizeof(T) == 8 ? ld_tag(p + 1) : 0ull;
        if (Tag<T>::ok(w, tag)) break;
        if ((++spins & 255) == 0) {
            if (*((volatile int *)&sync[3]) != 0) break;
            if (spins > kSpinLimit) {
                atomicOr(&sync[3], kErrTimeout);
                break;
            }
        }
    }
    return Tag<T>::value(w);
}

template <typename T>
__device__ __forceinline__ T shfl_up(T v, int d) {
    return __shfl_up_sync(0xffffffffu, v, d);
}

constexpr int RING = 4;   // line inputs are fetched RING - 1 steps ahead

template <typename T, typename TR, bool BWD>
__global__ void __launch_bounds__(256) k_line_sweep(int nx, int ny, int nz, int TJ, int TK, int NJ, int NK, int E,
                                                     const int *__restrict__ order, const T *__restrict__ c0,
                                                     const T *__restrict__ c1, const T *__restrict__ c2,
                                                     const T *__restrict__ dinv, const TR *__restrict__ rhs,
                                                     T *__restrict__ out, unsigned long long *jface,
                                                     unsigned long long *kface, unsigned long long *progress,
                                                     int *sync) {
    constexpr int NA = BWD ? 5 : 4;   // rhs, c0, c1, c2 (, dinv) ring arrays
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int LW = 32 * E;            // padded line length held by a warp
    // shared: exchange [2][TK][LW] T | input ring [RING][NA-1][TK][LW] T | rhs ring [RING][TK][LW] TR |
    //         k-face ring (warp 0) [RING][LW] x 16 B | progress ring [RING][2] x 16 B
    extern __shared__ __align__(16) unsigned char smraw[];
    T *xch = reinterpret_cast<T *>(smraw);
    size_t off = ((size_t)2 * TK * LW * sizeof(T) + 15) & ~(size_t)15;
    T *ring = reinterpret_cast<T *>(smraw + off);
    off += (size_t)RING * (NA - 1) * TK * LW * sizeof(T);
    off = (off + 15) & ~(size_t)15;
    TR *rring = reinterpret_cast<TR *>(smraw + off);
    off += (size_t)RING * TK * LW * sizeof(TR);
    off = (off + 15) & ~(size_t)15;
    unsigned long long *kring = reinterpret_cast<unsigned long long *>(smraw + off);   // [RING][LW][2]
    off += (size_t)RING * LW * 16;
    unsigned long long *pring = reinterpret_cast<unsigned long long *>(smraw + off);   // [RING][2][2]

    __shared__ int s_vb, s_tgt;
    if (tid == 0) {
        s_vb = atomicAdd(&sync[1], 1);
        s_tgt = *((volatile int *)&sync[0]) + 1;
    }
    __syncthreads();
    const int tile = order[s_vb];
    const unsigned tag = (unsigned)s_tgt;
    const int J = tile % NJ, K = tile / NJ;
    const int steps = TJ + TK - 1;
    const int km = K * TK + w;                       // mirrored k of this warp's row
    const bool rowlive = km < nz;
    const int kr = BWD ? nz - 1 - km : km;           // real k
    const long long plane = (long long)nx * ny;
    const int prodJ = J > 0 ? (J - 1) + NJ * K : -1;
    const int prodK = K > 0 ? J + NJ * (K - 1) : -1;
    const bool feedJ = J + 1 < NJ;
    const bool feedK = K + 1 < NK && w == TK - 1;

    // real x of this lane's cell e, and whether it exists
    auto xreal = [&](int e) { const int xm = lane * E + e; return BWD ? nx - 1 - xm : xm; };
    auto xok = [&](int e) { return lane * E + e < nx; };

    // line (tj, w) of this tile exists when the row is live and its j is inside the grid
    auto line_j = [&](int tj) { return J * TJ + tj; };   // mirrored j
    auto line_live = [&](int tj) { return rowlive && tj >= 0 && tj < TJ && line_j(tj) < ny; };
    auto row_base = [&](int tj) {                         // real index of x = 0 of line (tj, w)
        const int jm = line_j(tj);
        const int jr = BWD ? ny - 1 - jm : jm;
        return (long long)nx * jr + plane * kr;
    };

    // async fetch of the inputs of line tj into ring slot b (one commit group)
    auto fetch = [&](int b, int tj) {
        const bool live = line_live(tj);
        const long long base = live ? row_base(tj) : 0;
        for (int e = 0; e < E; ++e) {
            const bool v = live && xok(e);
            const long long c = v ? base + xreal(e) : 0;
            const int at = lane * E + e;
            cp_async<sizeof(TR)>(rring + ((size_t)b * TK + w) * LW + at, rhs + c, v);
            cp_async<sizeof(T)>(ring + (((size_t)b * (NA - 1) + 0) * TK + w) * LW + at, c0 + c, v);
            cp_async<sizeof(T)>(ring + (((size_t)b * (NA - 1) + 1) * TK + w) * LW + at, c1 + c, v);
            cp_async<sizeof(T)>(ring + (((size_t)b * (NA - 1) + 2) * TK + w) * LW + at, c2 + c, v);
            if (BWD) cp_async<sizeof(T)>(ring + (((size_t)b * (NA - 1) + 3) * TK + w) * LW + at, dinv + c, v);
        }
        // warp 0 also needs the k-face line (tj, TK-1) of tile (J, K-1)
        if (w == 0 && prodK >= 0 && live) {
            const unsigned long long *src = kface + (((long long)prodK * TJ + tj) * nx) * 2;
            for (int e = 0; e < E; ++e)
                cp_async<16>(kring + (((size_t)b * LW) + lane * E + e) * 2, src + (long long)(xok(e) ? lane * E + e : 0) * 2,
                             xok(e));
        }
        if (tid == 0 && prodK >= 0) cp_async<16>(pring + (size_t)b * 4 + 2, progress + 2 * prodK, true);
        cp_async_commit();
    };

    // pacing (thread 0): before the step-s barrier, producer (J, K-1) must have
    // completed the step that makes the k-face line fetched during step s;
    // j-face lines are taken (validated) when used, once per warp and tile
    unsigned seenK = 0;
    auto prog_of = [&](unsigned long long v) -> unsigned { return (unsigned)(v >> 32) == tag ? (unsigned)v : 0u; };
    auto pace = [&](int s, int b) {
        if (tid != 0 || prodK < 0) return;
        const int ahead = s + RING - 1;   // line tj = ahead of warp 0 is fetched during step s
        if (ahead >= TJ) return;
        const unsigned needK = (unsigned)min(ahead + TK, steps);   // produced at producer step ahead + TK - 1
        seenK = max(seenK, prog_of(pring[b * 4 + 2]));
        long long spins = 0;
        while (seenK < needK) {
            seenK = max(seenK, prog_of(ld_tag(progress + 2 * prodK)));
            if ((++spins & 255) == 0) {
                if (*((volatile int *)&sync[3]) != 0) break;
                if (spins > kSpinLimit) {
                    atomicOr(&sync[3], kErrTimeout);
                    break;
                }
            }
        }
    };

    T prevline[EMAX];
#pragma unroll
    for (int e = 0; e < EMAX; ++e) prevline[e] = T(0);

#pragma unroll
    for (int q = 0; q < RING - 1; ++q) fetch(q, q - w);   // inputs of steps 0 .. RING-2
    for (int s = 0; s < steps; ++s) {
        const int b = s % RING;
        cp_async_wait<RING - 2>();              // this thread's copies for step s have landed
        pace(s, b);
        __syncthreads();                        // lines of step s-1 visible; ring slot of step s-1 free
        if (tid == 0 && s > 0) st_tag(progress + 2 * tile, (unsigned)s, tag);   // steps 0..s-1 complete
        fetch((s + RING - 1) % RING, s + RING - 1 - w);   // prefetch while this step is solved
        const int tj = s - w;
        if (line_live(tj)) {
            const long long base = row_base(tj);
            const T *xin = xch + ((size_t)((s - 1) & 1) * TK + (w - 1)) * LW;   // warp w-1's line of step s-1
            T A[EMAX], B[EMAX];
            // neighbour lines: (tj-1) in registers (or the j-face of tile J-1), (w-1) in shared
            // memory (or the k-face of tile K-1 for warp 0)
            const bool jin = line_j(tj) > 0, kin = km > 0;
            const unsigned long long *jsrc =
                (tj == 0 && prodJ >= 0) ? jface + (((long long)prodJ * TK + w) * nx) * 2 : nullptr;
#pragma unroll
            for (int e = 0; e < EMAX; ++e) {
                A[e] = T(1);
                B[e] = T(0);
                if (e < E && xok(e)) {
                    const int at = lane * E + e;
                    T nj = T(0), nk = T(0);
                    if (jin) nj = jsrc ? take_tagged<T>(jsrc + (long long)at * 2, tag, sync) : prevline[e];
                    if (kin) {
                        if (w > 0) nk = xin[at];
                        else {
                            const unsigned long long *kw = kring + (((size_t)b * LW) + at) * 2;
                            nk = Tag<T>::ok(kw, tag) ? Tag<T>::value(kw)
                                                     : take_tagged<T>(kface + (((long long)prodK * TJ + tj) * nx + at) * 2,
                                                                      tag, sync);
                        }
                    }
                    const T r = (T)rring[((size_t)b * TK + w) * LW + at];
                    const T a0 = ring[(((size_t)b * (NA - 1) + 0) * TK + w) * LW + at];
                    const T a1 = ring[(((size_t)b * (NA - 1) + 1) * TK + w) * LW + at];
                    const T a2 = ring[(((size_t)b * (NA - 1) + 2) * TK + w) * LW + at];
                    T bb = r - a1 * nj - a2 * nk;
                    T aa = -a0;
                    if (BWD) {
                        const T d = ring[(((size_t)b * (NA - 1) + 3) * TK + w) * LW + at];
                        bb *= d;
                        aa *= d;
                    }
                    A[e] = aa;
                    B[e] = bb;
                }
            }
            // lane composition: (a, b) applied after (A, B): (a A, a B + b)
            T LA = T(1), LB = T(0);
#pragma unroll
            for (int e = 0; e < EMAX; ++e)
                if (e < E) {
                    LB = A[e] * LB + B[e];
                    LA = A[e] * LA;
                }
            // warp inclusive scan of the lane maps (Kogge-Stone)
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const T pa = shfl_up(LA, d), pb = shfl_up(LB, d);
                if (lane >= d) {
                    LB = LA * pb + LB;
                    LA = LA * pa;
                }
            }
            // value entering this lane: the prefix of lanes < lane applied to 0
            T v = shfl_up(LB, 1);
            if (lane == 0) v = T(0);
#pragma unroll
            for (int e = 0; e < EMAX; ++e)
                if (e < E) {
                    v = A[e] * v + B[e];
                    prevline[e] = v;
                }
            T *xo = xch + ((size_t)(s & 1) * TK + w) * LW;
#pragma unroll
            for (int e = 0; e < EMAX; ++e)
                if (e < E && xok(e)) {
                    const int at = lane * E + e;
                    out[base + xreal(e)] = prevline[e];
                    xo[at] = prevline[e];
                    if (feedJ && tj == TJ - 1) Tag<T>::put(jface + (((long long)tile * TK + w) * nx + at) * 2, prevline[e], tag);
                    if (feedK) Tag<T>::put(kface + (((long long)tile * TJ + tj) * nx + at) * 2, prevline[e], tag);
                }
        }
    }
    cp_async_wait0();
    __syncthreads();
    if (tid == 0) {
        st_tag(progress + 2 * tile, (unsigned)steps, tag);
        __threadfence();
        const int prev_done = atomicAdd(&sync[2], 1);
        if (prev_done == (int)gridDim.x - 1) {
            sync[1] = 0;
            sync[2] = 0;
            __threadfence();
            atomicAdd(&sync[0], 1);
        }
    }
}

template <typename T, typename TR, bool BWD>
size_t line_smem(int TK, int E) {
    constexpr int NA = BWD ? 5 : 4;
    const int LW = 32 * E;
    size_t off = ((size_t)2 * TK * LW * sizeof(T) + 15) & ~(size_t)15;
    off += (size_t)RING * (NA - 1) * TK * LW * sizeof(T);
    off = (off + 15) & ~(size_t)15;
    off += (size_t)RING * TK * LW * sizeof(TR);
    off = (off + 15) & ~(size_t)15;
    off += (size_t)RING * LW * 16;
    off += (size_t)RING * 32;
    return off;
}

template <typename T, typename TR, bool BWD>
void launch_lines(ms_system &s, const T *a0, const T *a1, const T *a2, const T *dinv, const TR *rhs, T *out,
                  cudaStream_t st) {
    const int E = (s.nx + 31) / 32;
    const int nT = s.LNJ * s.LNK;
    const size_t smem = line_smem<T, TR, BWD>(s.LTK, E);
    auto kern = k_line_sweep<T, TR, BWD>;
    static size_t smem_set = 48 * 1024;
    if (smem > smem_set) {
        MS_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        smem_set = smem;
    }
    kern<<<nT, 32 * s.LTK, smem, st>>>(s.nx, s.ny, s.nz, s.LTJ, s.LTK, s.LNJ, s.LNK, E, s.line_order.p, a0, a1, a2,
                                       dinv, rhs, out, s.lface_j.p, s.lface_k.p, s.line_progress.p, s.sync.p);
    MS_CHECK_LAUNCH();
}

template <typename T, typename TR>
void lines_apply(ms_system &s, const T *coef, const T *dinv, const TR *r, T *y, T *z, cudaStream_t st) {
    const int64_t n = s.n;
    const double nl = (double)s.nnz_lower;
    {
        KernelScope ks_(st, sizeof(T) == 8 ? "ilu_fwd" : "ilu_fwd32", nl * sizeof(T) + (double)n * (sizeof(TR) + sizeof(T)));
        launch_lines<T, TR, false>(s, coef, coef + n, coef + 2 * n, nullptr, r, y, st);
    }
    KernelScope ks_(st, sizeof(T) == 8 ? "ilu_bwd" : "ilu_bwd32", nl * sizeof(T) + (double)n * 3 * sizeof(T));
    launch_lines<T, T, true>(s, coef + 3 * n, coef + 4 * n, coef + 5 * n, dinv, y, z, st);
}

}  // namespace

bool lines_supported(const ms_system &s) { return s.structured && s.nx <= 32 * EMAX && s.LTK > 0; }

void launch_ilu_lines64(ms_system &s, const double *r, double *y, double *z, cudaStream_t st) {
    lines_apply<double, double>(s, s.dcoef64.p, s.dinv64.p, r, y, z, st);
}

void launch_ilu_lines32(ms_system &s, const double *r, float *y, float *z, cudaStream_t st) {
    lines_apply<float, double>(s, s.dcoef32.p, s.dinv32.p, r, y, z, st);
}

void launch_ilu_lines32f(ms_system &s, const float *r, float *y, float *z, cudaStream_t st) {
    lines_apply<float, float>(s, s.dcoef32.p, s.dinv32.p, r, y, z, st);
}

}  // namespace msgb
