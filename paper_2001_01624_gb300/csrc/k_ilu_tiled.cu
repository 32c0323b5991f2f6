// ILU(0) triangular sweeps on structured Cartesian grids (natural order).
//
// With the 7-point (5-point in 2D) pattern, row i of the forward sweep
//     y_i = r_i - L_i,-x y_{i-1} - L_i,-y y_{i-nx} - L_i,-z y_{i-nx*ny}
// depends on the three lower neighbours only, and the backward sweep
//     z_i = (y_i - U_i,+x z_{i+1} - U_i,+y z_{i+nx} - U_i,+z z_{i+nx*ny}) / U_ii
// on the three upper ones: the dependency graph is the wavefront x + y + z,
// whatever the values (exact ILU(0) of the natural ordering, no reordering).
//
// Mapping: one thread owns one x-pencil (fixed j, k) and walks it from x = 0
// to nx - 1 (mirrored for the backward sweep), so the x-dependency stays in
// a register.  A CTA owns a TJ x TK tile of pencils and advances them in
// skewed lock-step: at step t, pencil (tj, tk) handles x = t - tj - tk, so its
// (j-1) and (k-1) neighbours produced their value one step earlier and pass
// it through shared memory (double-buffered by step parity).  Pencils on the
// low faces of the tile read the neighbouring tile's values from global
// memory after that tile has published enough progress (release/acquire on a
// per-tile counter tagged with the sweep counter).  Inputs for step t + D are
// loaded at step t (register ring) so no load latency sits on the wavefront.
// Tiles take tickets in an order where every tile follows its producers, so
// waiting never deadlocks; waits are bounded and raise an error bit.
#include "ms_internal.h"

namespace msgb {

namespace {

constexpr long long kSpinLimit = 1ll << 24;

// Tagged words: a 32-bit payload with the 32-bit sweep counter in the high
// half, written and read as single 64-bit accesses.  A consumer accepts a
// word only when its tag is the current sweep's, so no flag, fence or
// ordering between words is needed: each word validates itself.
__device__ __forceinline__ void st_tag(unsigned long long *p, unsigned payload, unsigned tag) {
    const unsigned long long w = ((unsigned long long)tag << 32) | payload;
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(w) : "memory");
}

__device__ __forceinline__ unsigned long long ld_tag(const unsigned long long *p) {
    unsigned long long w;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(w) : "l"(p) : "memory");
    return w;
}

__device__ __forceinline__ void prefetch_l2(const void *p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }

// Tagged face values: 16 bytes per value, one (float) or two (double)
// tagged 64-bit words, so a consumer can fetch a value with one 16-byte
// async copy and validate it in shared memory.
template <typename T>
struct Tagged;
template <>
struct Tagged<float> {
    __device__ static void put(unsigned long long *p, float v, unsigned tag) { st_tag(p, __float_as_uint(v), tag); }
    __device__ static bool ok(const unsigned long long *w, unsigned tag) { return (unsigned)(w[0] >> 32) == tag; }
    __device__ static float value(const unsigned long long *w) { return __uint_as_float((unsigned)w[0]); }
};
template <>
struct Tagged<double> {
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

// Asynchronous global -> shared copies (per thread).  src_bytes = 0 fills
// the destination with zeros without reading the source.
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
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Tile sweep.  Per step: one CTA barrier, two shared-memory neighbour reads,
// one fused multiply-add chain.  Inputs of step t + D are copied
// asynchronously into a per-thread shared-memory ring at step t (async
// copies are not waited for by the barrier).  Tiles exchange their high j
// and k faces through tagged face buffers: jface[tile][tk][x] feeds tile
// (J+1, K), kface[tile][tj][x] feeds tile (J, K+1); a consumer validates the
// prefetched face value when it uses it and re-reads it (bounded) while it
// still carries an older sweep's tag.
template <typename T, typename TR, bool BWD, int D>
__global__ void __launch_bounds__(512) k_tile_sweep(int nx, int ny, int nz, int TJ, int TK, int NJ, int NK,
                                                    const int *__restrict__ order, const T *__restrict__ c0,
                                                    const T *__restrict__ c1, const T *__restrict__ c2,
                                                    const T *__restrict__ dinv, const TR *__restrict__ rhs,
                                                    T *__restrict__ out, unsigned long long *jface,
                                                    unsigned long long *kface, unsigned long long *progress,
                                                    int *sync) {
    using TG = Tagged<T>;
    constexpr int NA = BWD ? 5 : 4;            // rhs, c0, c1, c2 (, dinv)
    extern __shared__ __align__(16) unsigned char smraw[];
    const int tid = threadIdx.x;
    const int nthr = blockDim.x;
    const int ncomp = TJ * TK;
    // shared layout: [2][ncomp] exchange | ring [D][NA-1][nthr] of T | rhs ring [D][nthr] of TR |
    // j-face ring [D][TK] and k-face ring [D][TJ] of 16-byte tagged values
    T *sm = reinterpret_cast<T *>(smraw);
    size_t off = (((size_t)2 * ncomp * sizeof(T)) + 15) & ~(size_t)15;
    TR *rrs = nullptr;   // rhs ring kept in its own type
    T *ring = reinterpret_cast<T *>(smraw + off);
    off += (size_t)D * (NA - 1) * nthr * sizeof(T);
    off = (off + 15) & ~(size_t)15;
    rrs = reinterpret_cast<TR *>(smraw + off);
    off += (size_t)D * nthr * sizeof(TR);
    off = (off + 15) & ~(size_t)15;
    unsigned long long *fringJ = reinterpret_cast<unsigned long long *>(smraw + off);
    unsigned long long *fringK = fringJ + (size_t)D * TK * 2;
    unsigned long long *pring = fringK + (size_t)D * TJ * 2;   // [D][2] producer progress words (x2 for 16 B)

    __shared__ int s_vb, s_tgt;
    const int steps = nx + TJ + TK - 2;
    if (tid == 0) {
        s_vb = atomicAdd(&sync[1], 1);
        s_tgt = *((volatile int *)&sync[0]) + 1;
    }
    __syncthreads();
    const int tile = order[s_vb];
    const unsigned tag = (unsigned)s_tgt;
    const int J = tile % NJ, K = tile / NJ;
    const int tj = tid % TJ, tk = tid / TJ;
    const int jm = J * TJ + tj, km = K * TK + tk;   // mirrored pencil coordinates
    const bool live = tid < ncomp && jm < ny && km < nz;
    const int j = BWD ? ny - 1 - jm : jm, k = BWD ? nz - 1 - km : km;
    const long long plane = (long long)nx * ny;
    const long long row0 = live ? (long long)nx * j + plane * k : 0;   // real index of x = 0
    const bool needJ = live && tj == 0 && J > 0;
    const bool needK = live && tk == 0 && K > 0;
    const bool feedJ = live && tj == TJ - 1 && J + 1 < NJ;
    const bool feedK = live && tk == TK - 1 && K + 1 < NK;
    const unsigned long long *inJ = jface + (needJ ? (((long long)((J - 1) + NJ * K) * TK + tk) * nx) * 2 : 0);
    const unsigned long long *inK = kface + (needK ? (((long long)(J + NJ * (K - 1)) * TJ + tj) * nx) * 2 : 0);
    unsigned long long *outJ = jface + (feedJ ? (((long long)tile * TK + tk) * nx) * 2 : 0);
    unsigned long long *outK = kface + (feedK ? (((long long)tile * TJ + tj) * nx) * 2 : 0);

    // stream this pencil's inputs into L2 now; the async ring then hits L2
    if (live) {
        for (int x = 0; x < nx; x += 128 / (int)sizeof(T)) {
            const long long c = row0 + x;
            prefetch_l2(c0 + c);
            prefetch_l2(c1 + c);
            prefetch_l2(c2 + c);
            if (BWD) prefetch_l2(dinv + c);
            prefetch_l2(rhs + c);
        }
    }

    auto slot = [&](int d, int a) -> T * { return ring + ((size_t)d * (NA - 1) + a) * nthr + tid; };
    auto fslotJ = [&](int d) -> unsigned long long * { return fringJ + ((size_t)d * TK + tk) * 2; };
    auto fslotK = [&](int d) -> unsigned long long * { return fringK + ((size_t)d * TJ + tj) * 2; };
    // issue the copies for mirrored x into ring slot d (one commit group per call)
    auto issue = [&](int d, int xm) {
        const bool v = live && xm >= 0 && xm < nx;
        const long long c = v ? row0 + (BWD ? nx - 1 - xm : xm) : 0;
        cp_async<sizeof(TR)>(rrs + (size_t)d * nthr + tid, rhs + c, v);
        cp_async<sizeof(T)>(slot(d, 0), c0 + c, v);
        cp_async<sizeof(T)>(slot(d, 1), c1 + c, v);
        cp_async<sizeof(T)>(slot(d, 2), c2 + c, v);
        if (BWD) cp_async<sizeof(T)>(slot(d, 3), dinv + c, v);
        if (needJ) cp_async<16>(fslotJ(d), inJ + (long long)(v ? xm : 0) * 2, v);
        if (needK) cp_async<16>(fslotK(d), inK + (long long)(v ? xm : 0) * 2, v);
        cp_async_commit();
    };
    // value of a face word in shared memory, re-read from global while stale
    auto accept = [&](unsigned long long *w, const unsigned long long *src) -> T {
        unsigned long long g[2] = {w[0], w[1]};
        long long spins = 0;
        while (!TG::ok(g, tag)) {
            if ((++spins & 255) == 0) {
                if (*((volatile int *)&sync[3]) != 0) break;
                if (spins > kSpinLimit) {
                    atomicOr(&sync[3], kErrTimeout);
                    break;
                }
            }
            g[0] = ld_tag(src);
            g[1] = ld_tag(src + 1);
        }
        return TG::value(g);
    };

    // Pacing: tile progress words are hints only (tags make the data safe).
    // Thread 0 fetches the producers' progress through the async ring and,
    // before the barrier of step t, waits until the producers have completed
    // the steps whose face values this CTA prefetches at step t.  A consumer
    // thus trails its producer far enough that face prefetches are fresh,
    // instead of re-polling stale values on every step.
    const int prodJ = J > 0 ? (J - 1) + NJ * K : -1;
    const int prodK = K > 0 ? J + NJ * (K - 1) : -1;
    const bool pacer = tid == 0 && (prodJ >= 0 || prodK >= 0);
    unsigned seenJ = 0, seenK = 0;   // producer steps known complete (this sweep)
    auto progress_of = [&](unsigned long long w) -> unsigned {
        return (unsigned)(w >> 32) == tag ? (unsigned)w : 0u;
    };
    auto pace = [&](int t, int u) {
        if (!pacer) return;
        const unsigned nJ = (unsigned)min(t + D + TJ, steps), nK = (unsigned)min(t + D + TK, steps);
        if (prodJ >= 0) seenJ = max(seenJ, progress_of(pring[u * 4 + 0]));
        if (prodK >= 0) seenK = max(seenK, progress_of(pring[u * 4 + 2]));
        long long spins = 0;
        while ((prodJ >= 0 && seenJ < nJ) || (prodK >= 0 && seenK < nK)) {
            if (prodJ >= 0 && seenJ < nJ) seenJ = max(seenJ, progress_of(ld_tag(progress + 2 * prodJ)));
            if (prodK >= 0 && seenK < nK) seenK = max(seenK, progress_of(ld_tag(progress + 2 * prodK)));
            if ((++spins & 255) == 0) {
                if (*((volatile int *)&sync[3]) != 0) break;
                if (spins > kSpinLimit) {
                    atomicOr(&sync[3], kErrTimeout);
                    break;
                }
            }
        }
    };
    auto issue_progress = [&](int u) {
        if (!pacer) return;
        if (prodJ >= 0) cp_async<16>(pring + u * 4 + 0, progress + 2 * prodJ, true);   // 16 B: via L2
        if (prodK >= 0) cp_async<16>(pring + u * 4 + 2, progress + 2 * prodK, true);
    };

    const int skew = tj + tk;
#pragma unroll
    for (int d = 0; d < D; ++d) {
        issue_progress(d);
        issue(d, d - skew);
    }
    T prev = T(0);
    for (int t0 = 0; t0 < steps; t0 += D) {
#pragma unroll
        for (int u = 0; u < D; ++u) {
            const int t = t0 + u;
            if (t < steps) {
                cp_async_wait<D - 1>();          // this thread's copies for step t have landed
                pace(t, u);
                if (t > 0) __syncthreads();      // step t-1 values in shared memory
                if (tid == 0 && t > 0) st_tag(progress + 2 * tile, (unsigned)t, tag);   // steps 0..t-1 done
                const int xm = t - skew;
                if (live && xm >= 0 && xm < nx) {
                    const T *smp = sm + ((t - 1) & 1) * ncomp;
                    const T nj = tj > 0 ? smp[tk * TJ + tj - 1]
                                        : (needJ ? accept(fslotJ(u), inJ + (long long)xm * 2) : T(0));
                    const T nk = tk > 0 ? smp[(tk - 1) * TJ + tj]
                                        : (needK ? accept(fslotK(u), inK + (long long)xm * 2) : T(0));
                    T s = (T)rrs[(size_t)u * nthr + tid] - *slot(u, 0) * prev - *slot(u, 1) * nj - *slot(u, 2) * nk;
                    if (BWD) s *= *slot(u, 3);
                    out[row0 + (BWD ? nx - 1 - xm : xm)] = s;
                    if (feedJ) TG::put(outJ + (long long)xm * 2, s, tag);
                    if (feedK) TG::put(outK + (long long)xm * 2, s, tag);
                    prev = s;
                    sm[(t & 1) * ncomp + tk * TJ + tj] = s;
                }
                issue_progress(u);
                issue(u, xm + D);
            }
        }
    }
    cp_async_wait<0>();
    __syncthreads();
    if (tid == 0) st_tag(progress + 2 * tile, (unsigned)steps, tag);
    if (tid == 0) {
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

template <typename T, typename TR, bool BWD, int D>
size_t tile_smem(int TJ, int TK) {
    constexpr int NA = BWD ? 5 : 4;
    const int nthr = TJ * TK;
    size_t off = (((size_t)2 * nthr * sizeof(T)) + 15) & ~(size_t)15;
    off += (size_t)D * (NA - 1) * nthr * sizeof(T);
    off = (off + 15) & ~(size_t)15;
    off += (size_t)D * nthr * sizeof(TR);
    off = (off + 15) & ~(size_t)15;
    off += (size_t)D * (TJ + TK) * 16;
    off += (size_t)D * 32;   // progress ring
    return off;
}

// Direction-major factor coefficients from the ELL factor.
template <typename T>
__global__ void k_extract_dirs(int n, const int8_t *__restrict__ dslot, const double *__restrict__ lu, T *coef) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
#pragma unroll
    for (int d = 0; d < 6; ++d) {
        const int w = dslot[(int64_t)d * n + i];
        coef[(int64_t)d * n + i] = w >= 0 ? (T)lu[(int64_t)w * n + i] : T(0);
    }
}

// register-ring depth: steps of load latency hidden (bounded by registers)
template <typename T> constexpr int ring_depth() { return 8; }

template <typename T, typename TR, bool BWD>
void launch_sweep(ms_system &s, const T *a0, const T *a1, const T *a2, const T *dinv, const TR *rhs, T *out,
                  cudaStream_t st) {
    constexpr int D = ring_depth<T>();
    const int nT = s.NJ * s.NK;
    const int threads = s.TJ * s.TK;
    const size_t smem = tile_smem<T, TR, BWD, D>(s.TJ, s.TK);
    auto kern = k_tile_sweep<T, TR, BWD, D>;
    static size_t smem_set = 48 * 1024;   // per instantiation
    MS_CUDA(raise_smem_limit(kern, smem, smem_set));
    kern<<<nT, threads, smem, st>>>(s.nx, s.ny, s.nz, s.TJ, s.TK, s.NJ, s.NK, s.tile_order.p, a0, a1, a2, dinv, rhs,
                                    out, s.face_j.p, s.face_k.p, s.tile_progress.p, s.sync.p);
    MS_CHECK_LAUNCH();
}

template <typename T, typename TR>
void tiled_apply(ms_system &s, const T *coef, const T *dinv, const TR *r, T *y, T *z, cudaStream_t st) {
    const int64_t n = s.n;
    const double nl = (double)s.nnz_lower;
    {
        KernelScope ks_(st, sizeof(T) == 8 ? "ilu_fwd" : "ilu_fwd32", nl * sizeof(T) + (double)n * (sizeof(TR) + sizeof(T)));
        launch_sweep<T, TR, false>(s, coef, coef + n, coef + 2 * n, nullptr, r, y, st);
    }
    KernelScope ks_(st, sizeof(T) == 8 ? "ilu_bwd" : "ilu_bwd32", nl * sizeof(T) + (double)n * 3 * sizeof(T));
    launch_sweep<T, T, true>(s, coef + 3 * n, coef + 4 * n, coef + 5 * n, dinv, y, z, st);
}

}  // namespace

void launch_ilu_extract_dirs(ms_system &s, bool fp32, cudaStream_t st) {
    const int g = (s.n + 255) / 256;
    if (fp32) {
        s.dcoef32.alloc((size_t)6 * s.n);
        k_extract_dirs<float><<<g, 256, 0, st>>>(s.n, s.dir_slot.p, s.lu64.p, s.dcoef32.p);
    } else {
        s.dcoef64.alloc((size_t)6 * s.n);
        k_extract_dirs<double><<<g, 256, 0, st>>>(s.n, s.dir_slot.p, s.lu64.p, s.dcoef64.p);
    }
    MS_CHECK_LAUNCH();
}

void launch_ilu_tiled64(ms_system &s, const double *r, double *y, double *z, cudaStream_t st) {
    tiled_apply<double, double>(s, s.dcoef64.p, s.dinv64.p, r, y, z, st);
}

void launch_ilu_tiled32(ms_system &s, const double *r, float *y, float *z, cudaStream_t st) {
    tiled_apply<float, double>(s, s.dcoef32.p, s.dinv32.p, r, y, z, st);
}

void launch_ilu_tiled32f(ms_system &s, const float *r, float *y, float *z, cudaStream_t st) {
    tiled_apply<float, float>(s, s.dcoef32.p, s.dinv32.p, r, y, z, st);
}

}  // namespace msgb
