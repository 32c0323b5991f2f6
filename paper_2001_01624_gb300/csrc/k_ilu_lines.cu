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
// memory (one barrier per step).  Lane 0 of each warp fetches the inputs of
// its line RING - 1 steps ahead with bulk copies (one per array and line, the
// line's span rounded out to 16 bytes) into a shared-memory ring, completing on
// one mbarrier per warp and slot.  Tiles hand over their high j / k face lines
// as tagged words (payload + sweep counter, validated by the consumer) and pace
// each other with tagged per-tile progress hints; tickets follow a topological
// order of the tile grid, and every wait is bounded.
//
// A step is short and its work is a chain of dependent instructions executed
// by one or two warps per SM sub-partition, so the step time is set by that
// chain's latency: the cell count per lane is a compile-time constant and all
// per-line addressing is hoisted out of the step loop.
#include "ms_internal.h"

namespace msgb {

namespace {

constexpr long long kSpinLimit = 1ll << 24;

__device__ __forceinline__ void st_tag(unsigned long long *p, unsigned payload, unsigned tag) {
    const unsigned long long w = ((unsigned long long)tag << 32) | payload;
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(w) : "memory");
}

__device__ __forceinline__ unsigned long long ld_tag(const unsigned long long *p) {
    unsigned long long w;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(w) : "l"(p) : "memory");
    return w;
}

// Bulk (TMA-class) copies global -> shared completing on an mbarrier.
__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"((unsigned)__cvta_generic_to_shared(bar)), "r"(count)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect(unsigned long long *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"((unsigned)__cvta_generic_to_shared(bar)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
        : "=r"(ok)
        : "r"((unsigned)__cvta_generic_to_shared(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ void bulk_g2s(void *smem_dst, const void *gsrc, unsigned bytes, unsigned long long *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            (unsigned)__cvta_generic_to_shared(smem_dst)),
        "l"(gsrc), "r"(bytes), "r"((unsigned)__cvta_generic_to_shared(bar))
        : "memory");
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

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

// Shared window per input array, warp and ring slot: the line plus up to 16
// bytes of alignment slack on each side, a multiple of 16 bytes long.
__host__ __device__ constexpr int win_elems(int nx, int esz) {
    return (nx + 3 * (16 / esz) + 16 / esz - 1) / (16 / esz) * (16 / esz);
}

// One sweep (forward, or backward when BWD) over the tiles of the line grid;
// E cells per lane (lines of up to 32 E cells).
template <typename T, typename TR, bool BWD, int E>
__global__ void __launch_bounds__(256, 1) k_line_sweep(int nx, int ny, int nz, int TJ, int TK, int NJ, int NK,
                                                    const int *__restrict__ order, const T *__restrict__ c0,
                                                    const T *__restrict__ c1, const T *__restrict__ c2,
                                                    const T *__restrict__ dinv, const TR *__restrict__ rhs,
                                                    T *__restrict__ out, unsigned long long *jface,
                                                    unsigned long long *kface, unsigned long long *progress,
                                                    int *sync) {
    constexpr int NC = BWD ? 4 : 3;   // coefficient windows: c0, c1, c2 (, dinv)
    constexpr int LW = 32 * E;
    constexpr int SG = BWD ? -1 : 1;  // direction of x inside a line (cell order along the sweep)
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int WT = win_elems(nx, sizeof(T));
    const int WR = win_elems(nx, sizeof(TR));
    // shared: exchange [2][TK][LW] T | coefficient windows [RING][NC][TK][WT] T |
    //         rhs windows [RING][TK][WR] TR | k-face windows (warp 0) [RING][nx] x 16 B | mbarriers [RING][TK]
    extern __shared__ __align__(16) unsigned char smraw[];
    T *xch = reinterpret_cast<T *>(smraw);
    size_t off = ((size_t)2 * TK * LW * sizeof(T) + 15) & ~(size_t)15;
    T *cwin = reinterpret_cast<T *>(smraw + off);
    off += (size_t)RING * NC * TK * WT * sizeof(T);
    TR *rwin = reinterpret_cast<TR *>(smraw + off);
    off += (size_t)RING * TK * WR * sizeof(TR);
    unsigned long long *kwin = reinterpret_cast<unsigned long long *>(smraw + off);
    off += (size_t)RING * nx * 16;
    unsigned long long *mbar = reinterpret_cast<unsigned long long *>(smraw + off);

    __shared__ int s_vb, s_tgt;
    if (tid == 0) {
        s_vb = atomicAdd(&sync[1], 1);
        s_tgt = *((volatile int *)&sync[0]) + 1;
    }
    if (lane == 0)
        for (int q = 0; q < RING; ++q) mbar_init(&mbar[q * TK + w], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    __syncthreads();
    const int tile = order[s_vb];
    const unsigned tag = (unsigned)s_tgt;
    const int J = tile % NJ, K = tile / NJ;
    const int steps = TJ + TK - 1;
    const int km = K * TK + w;                           // mirrored k of this warp's row
    const bool rowlive = km < nz;
    const int kr = BWD ? nz - 1 - km : km;               // real k
    const int nlive = min(TJ, ny - J * TJ);              // lines of this tile in j
    const int prodJ = J > 0 ? (J - 1) + NJ * K : -1;
    const int prodK = K > 0 ? J + NJ * (K - 1) : -1;
    const bool feedJ = J + 1 < NJ;
    const bool feedK = K + 1 < NK && w == TK - 1;
    // real index of x = 0 of line tj: base0 + dj * tj
    const long long plane = (long long)nx * ny;
    const long long base0 = (long long)nx * (BWD ? ny - 1 - J * TJ : J * TJ) + plane * kr;
    const long long dj = BWD ? -(long long)nx : (long long)nx;
    // per-warp shared offsets (elements)
    const int cw_w = w * WT, rw_w = w * WR;
    const int cslot = NC * TK * WT, carr = TK * WT, rslot = TK * WR;

    // span of a line in a global array, rounded out to 16-byte granules (never
    // leaving the granule of a valid address, so inside the mapped allocation)
    auto span_len = [&](unsigned long long b0, int esz) {
        return (unsigned)((((b0 + (unsigned long long)nx * esz) + 15ull) & ~15ull) - (b0 & ~15ull));
    };
    // lane 0 of each warp issues the bulk copies of line tj into ring slot q
    auto fetch = [&](int q, int tj) {
        if (lane != 0) return;
        unsigned long long *bar = &mbar[q * TK + w];
        if (!rowlive || tj < 0 || tj >= nlive) {
            mbar_arrive_expect(bar, 0);
            return;
        }
        const long long base = base0 + dj * tj;
        const unsigned long long ar = (unsigned long long)(size_t)(rhs + base),
                                 a0 = (unsigned long long)(size_t)(c0 + base),
                                 a1 = (unsigned long long)(size_t)(c1 + base),
                                 a2 = (unsigned long long)(size_t)(c2 + base),
                                 a3 = BWD ? (unsigned long long)(size_t)(dinv + base) : 0ull;
        const unsigned lr = span_len(ar, sizeof(TR)), l0 = span_len(a0, sizeof(T)), l1 = span_len(a1, sizeof(T)),
                       l2 = span_len(a2, sizeof(T)), l3 = BWD ? span_len(a3, sizeof(T)) : 0u;
        const bool kf = (w == 0 && prodK >= 0);
        mbar_arrive_expect(bar, lr + l0 + l1 + l2 + l3 + (kf ? (unsigned)nx * 16 : 0u));
        T *cq = cwin + q * cslot + cw_w;
        bulk_g2s(rwin + q * rslot + rw_w, (const void *)(size_t)(ar & ~15ull), lr, bar);
        bulk_g2s(cq, (const void *)(size_t)(a0 & ~15ull), l0, bar);
        bulk_g2s(cq + carr, (const void *)(size_t)(a1 & ~15ull), l1, bar);
        bulk_g2s(cq + 2 * carr, (const void *)(size_t)(a2 & ~15ull), l2, bar);
        if (BWD) bulk_g2s(cq + 3 * carr, (const void *)(size_t)(a3 & ~15ull), l3, bar);
        if (kf) bulk_g2s(kwin + (size_t)q * nx * 2, kface + (((long long)prodK * TJ + tj) * nx) * 2, (unsigned)nx * 16, bar);
    };
    // the copies read valid memory and always complete; the wait is still
    // bounded (2 s of device time unless the system sets another bound) and
    // reports a timeout instead of hanging
    auto wait_slot = [&](int q, unsigned parity) {
        unsigned long long t0 = 0;
        int spins = 0;
        while (!mbar_try_wait(&mbar[q * TK + w], parity)) {
            if ((++spins & 63) == 0) {
                const unsigned long long now = global_ns();
                if (t0 == 0) t0 = now;
                else if (now - t0 > wait_limit_ns(sync + 3)) {
                    atomicOr(&sync[3], kErrTimeout);
                    break;
                }
            }
        }
    };

    // pacing (thread 0): producer (J, K-1) must have completed the step that
    // makes the k-face line fetched during step s; j-face lines are taken
    // (validated) when used, once per warp and tile
    unsigned seenK = 0;
    auto pace = [&](int s) {
        if (tid != 0 || prodK < 0) return;
        const int ahead = s + RING - 1;
        if (ahead >= TJ) return;
        const unsigned needK = (unsigned)min(ahead + TK, steps);
        long long spins = 0;
        while (seenK < needK) {
            const unsigned long long v = ld_tag(progress + 2 * prodK);
            if ((unsigned)(v >> 32) == tag) seenK = max(seenK, (unsigned)v);
            if ((++spins & 255) == 0) {
                if (*((volatile int *)&sync[3]) != 0) break;
                if (spins > kSpinLimit) {
                    atomicOr(&sync[3], kErrTimeout);
                    break;
                }
            }
        }
    };

    T prevline[E];
#pragma unroll
    for (int e = 0; e < E; ++e) prevline[e] = T(0);

    for (int q = 0; q < RING - 1; ++q) {   // the first RING-1 fetches need the producer's progress too
        pace(q - (RING - 1));
        __syncwarp();
        fetch(q, q - w);
    }
    int q = 0;
    unsigned parity = 0;
    for (int s = 0; s < steps; ++s) {
        pace(s);
        __syncthreads();   // lines of step s-1 visible; slot of step s-1 free; pacing done
        if (tid == 0 && s > 0) st_tag(progress + 2 * tile, (unsigned)s, tag);   // steps 0..s-1 complete
        fetch(q == 0 ? RING - 1 : q - 1, s + RING - 1 - w);
        const int tj = s - w;
        wait_slot(q, parity);
        if (rowlive && tj >= 0 && tj < nlive) {
            const long long base = base0 + dj * tj;
            const unsigned bl = (unsigned)base;
            // element shift of the line's first cell inside each 16-byte aligned window
            const int shr = (int)((((unsigned)(size_t)rhs + bl * (unsigned)sizeof(TR)) & 15u) / sizeof(TR));
            const int sh0 = (int)((((unsigned)(size_t)c0 + bl * (unsigned)sizeof(T)) & 15u) / sizeof(T));
            const int sh1 = (int)((((unsigned)(size_t)c1 + bl * (unsigned)sizeof(T)) & 15u) / sizeof(T));
            const int sh2 = (int)((((unsigned)(size_t)c2 + bl * (unsigned)sizeof(T)) & 15u) / sizeof(T));
            const int sh3 = BWD ? (int)((((unsigned)(size_t)dinv + bl * (unsigned)sizeof(T)) & 15u) / sizeof(T)) : 0;
            const int x0 = BWD ? nx - 1 : 0;   // window position of the first cell along the sweep
            const TR *rl = rwin + q * rslot + rw_w + shr + x0;
            const T *cq = cwin + q * cslot + cw_w + x0;
            const T *cl0 = cq + sh0, *cl1 = cq + carr + sh1, *cl2 = cq + 2 * carr + sh2;
            const T *cl3 = cq + 3 * carr + sh3;
            T A[E], B[E];
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int at = lane * E + e;
                A[e] = T(1);
                B[e] = T(0);
                if (at < nx) {
                    T nj = T(0), nk = T(0);
                    if (tj > 0) nj = prevline[e];
                    else if (J > 0) nj = take_tagged<T>(jface + (((long long)prodJ * TK + w) * nx + at) * 2, tag, sync);
                    if (w > 0) nk = xch[(((s - 1) & 1) * TK + (w - 1)) * LW + at];
                    else if (K > 0) {
                        const unsigned long long *kw = kwin + ((size_t)q * nx + at) * 2;
                        nk = Tag<T>::ok(kw, tag)
                                 ? Tag<T>::value(kw)
                                 : take_tagged<T>(kface + (((long long)prodK * TJ + tj) * nx + at) * 2, tag, sync);
                    }
                    const int xi = SG * at;
                    T bb = (T)rl[xi] - cl1[xi] * nj - cl2[xi] * nk;
                    T aa = -cl0[xi];
                    if (BWD) {
                        const T d = cl3[xi];
                        bb *= d;
                        aa *= d;
                    }
                    A[e] = aa;
                    B[e] = bb;
                }
            }
            T LA = A[0], LB = B[0];
#pragma unroll
            for (int e = 1; e < E; ++e) {
                LB = A[e] * LB + B[e];
                LA = A[e] * LA;
            }
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const T pa = shfl_up(LA, d), pb = shfl_up(LB, d);
                if (lane >= d) {
                    LB = LA * pb + LB;
                    LA = LA * pa;
                }
            }
            T v = shfl_up(LB, 1);
            if (lane == 0) v = T(0);
#pragma unroll
            for (int e = 0; e < E; ++e) {
                v = A[e] * v + B[e];
                prevline[e] = v;
            }
            T *xo = xch + ((s & 1) * TK + w) * LW;
            T *ob = out + base + x0;
            const bool putJ = feedJ && tj == TJ - 1;
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int at = lane * E + e;
                if (at < nx) {
                    ob[SG * at] = prevline[e];
                    xo[at] = prevline[e];
                    if (putJ) Tag<T>::put(jface + (((long long)tile * TK + w) * nx + at) * 2, prevline[e], tag);
                    if (feedK) Tag<T>::put(kface + (((long long)tile * TJ + tj) * nx + at) * 2, prevline[e], tag);
                }
            }
        }
        if (++q == RING) {
            q = 0;
            parity ^= 1u;
        }
    }
    // drain: the last RING-1 fetches were issued for steps beyond the tile
    for (int s = steps; s < steps + RING - 1; ++s) {
        wait_slot(q, parity);
        if (++q == RING) {
            q = 0;
            parity ^= 1u;
        }
    }
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

// cells per lane: the smallest of 2, 4, 8 covering the line
inline int line_e(int nx) { return nx <= 64 ? 2 : nx <= 128 ? 4 : 8; }

template <typename T, typename TR, bool BWD>
size_t line_smem(int nx, int TK) {
    constexpr int NC = BWD ? 4 : 3;
    const int LW = 32 * line_e(nx);
    const int WT = win_elems(nx, sizeof(T)), WR = win_elems(nx, sizeof(TR));
    size_t off = ((size_t)2 * TK * LW * sizeof(T) + 15) & ~(size_t)15;
    off += (size_t)RING * NC * TK * WT * sizeof(T);
    off += (size_t)RING * TK * WR * sizeof(TR);
    off += (size_t)RING * nx * 16;
    off += (size_t)RING * TK * 8;
    return off;
}

template <typename T, typename TR, bool BWD, int E>
void launch_lines_e(ms_system &s, const T *a0, const T *a1, const T *a2, const T *dinv, const TR *rhs, T *out,
                    cudaStream_t st) {
    const int nT = s.LNJ * s.LNK;
    const size_t smem = line_smem<T, TR, BWD>(s.nx, s.LTK);
    auto kern = k_line_sweep<T, TR, BWD, E>;
    static size_t smem_set = 48 * 1024;
    MS_CUDA(raise_smem_limit(kern, smem, smem_set));
    kern<<<nT, 32 * s.LTK, smem, st>>>(s.nx, s.ny, s.nz, s.LTJ, s.LTK, s.LNJ, s.LNK, s.line_order.p, a0, a1, a2, dinv,
                                       rhs, out, s.lface_j.p, s.lface_k.p, s.line_progress.p, s.sync.p);
    MS_CHECK_LAUNCH();
}

template <typename T, typename TR, bool BWD>
void launch_lines(ms_system &s, const T *a0, const T *a1, const T *a2, const T *dinv, const TR *rhs, T *out,
                  cudaStream_t st) {
    switch (line_e(s.nx)) {
        case 2: launch_lines_e<T, TR, BWD, 2>(s, a0, a1, a2, dinv, rhs, out, st); break;
        case 4: launch_lines_e<T, TR, BWD, 4>(s, a0, a1, a2, dinv, rhs, out, st); break;
        default: launch_lines_e<T, TR, BWD, 8>(s, a0, a1, a2, dinv, rhs, out, st); break;
    }
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
