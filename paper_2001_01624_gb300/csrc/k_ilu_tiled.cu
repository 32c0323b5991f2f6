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

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void fence_acq_rel_gpu() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }

__device__ __forceinline__ void st_release_u64(unsigned long long *p, unsigned long long v) {
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Bounded wait until *p >= need (thread 0 only).
__device__ __forceinline__ unsigned long long wait_progress(const unsigned long long *p, unsigned long long need,
                                                            int *sync) {
    unsigned long long v = ld_acquire_u64(p);
    long long spins = 0;
    while (v < need) {
        if ((++spins & 255) == 0) {
            if (*((volatile int *)&sync[3]) != 0) return need;
            if (spins > kSpinLimit) {
                atomicOr(&sync[3], kErrTimeout);
                return need;
            }
        }
        v = ld_acquire_u64(p);
    }
    return v;
}

__device__ __forceinline__ int ld_acquire_cta_s32(const volatile int *p) {
    int v;
    asm volatile("ld.acquire.cta.shared::cta.u32 %0, [%1];" : "=r"(v) : "r"((unsigned)__cvta_generic_to_shared((const void *)p)) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_cta_s32(volatile int *p, int v) {
    asm volatile("st.release.cta.shared::cta.u32 [%0], %1;" ::"r"((unsigned)__cvta_generic_to_shared((const void *)p)), "r"(v) : "memory");
}

__device__ __forceinline__ void compute_barrier(int nthreads) {
    asm volatile("bar.sync 1, %0;" ::"r"(nthreads) : "memory");
}

// Warp-specialised tile sweep.  Warps 0..W-1 compute (TJ x TK pencils, one
// named barrier per step among themselves); the last warp handles all
// cross-CTA traffic: it publishes this tile's completed step count (release)
// whenever the compute warps advance, and polls the producer tiles
// (acquire), handing their progress to the compute warps through shared
// memory.  Fence and poll latency thus delay the wavefront once per tile hop
// instead of once per step.
template <typename T, typename TR, bool BWD, int D>
__global__ void __launch_bounds__(544, 1) k_tile_sweep(int nx, int ny, int nz, int TJ, int TK, int NJ,
                                                    const int *__restrict__ order, const T *__restrict__ c0,
                                                    const T *__restrict__ c1, const T *__restrict__ c2,
                                                    const T *__restrict__ dinv, const TR *__restrict__ rhs,
                                                    T *__restrict__ out, unsigned long long *prog, int *sync) {
    extern __shared__ unsigned char smraw[];
    T *sm = reinterpret_cast<T *>(smraw);   // [2][TK][TJ]
    __shared__ int s_vb, s_tgt;
    __shared__ volatile int s_done, s_availJ, s_availK, s_abort;
    const int tid = threadIdx.x;
    const int ncomp = TJ * TK;
    const int ncw = (ncomp + 31) / 32;      // compute warps
    const int steps = nx + TJ + TK - 2;
    if (tid == 0) {
        s_vb = atomicAdd(&sync[1], 1);
        s_tgt = *((volatile int *)&sync[0]) + 1;
    }
    __syncthreads();
    const int tile = order[s_vb];
    const unsigned long long epoch = (unsigned long long)(unsigned)s_tgt << 32;
    const int J = tile % NJ, K = tile / NJ;
    const int prodJ = J > 0 ? (J - 1) + NJ * K : -1;
    const int prodK = K > 0 ? J + NJ * (K - 1) : -1;
    if (tid == 0) {
        s_done = 0;
        s_availJ = prodJ >= 0 ? 0 : steps;
        s_availK = prodK >= 0 ? 0 : steps;
        s_abort = 0;
    }
    __syncthreads();

    if (tid >= ncw * 32) {
        // ------------------------------------------------ communication warp
        if (tid == ncw * 32) {
            int published = 0, aJ = s_availJ, aK = s_availK;
            long long spins = 0;
            while (true) {
                const int d = ld_acquire_cta_s32(&s_done);
                if (d > published) {
                    st_release_u64(&prog[tile], epoch | (unsigned long long)d);
                    published = d;
                }
                // relaxed polls; one acquire fence only when a producer advanced
                int nJ = aJ, nK = aK;
                if (aJ < steps) {
                    const unsigned long long v = ld_relaxed_u64(&prog[prodJ]);
                    nJ = v >= epoch ? (int)(v - epoch) : 0;
                }
                if (aK < steps) {
                    const unsigned long long v = ld_relaxed_u64(&prog[prodK]);
                    nK = v >= epoch ? (int)(v - epoch) : 0;
                }
                if (nJ > aJ || nK > aK) {
                    fence_acq_rel_gpu();
                    if (nJ > aJ) { aJ = nJ; st_release_cta_s32(&s_availJ, aJ); }
                    if (nK > aK) { aK = nK; st_release_cta_s32(&s_availK, aK); }
                }
                if (published == steps && aJ >= steps && aK >= steps) break;
                if ((++spins & 1023) == 0) {
                    if (*((volatile int *)&sync[3]) != 0 || spins > kSpinLimit) {
                        if (spins > kSpinLimit) atomicOr(&sync[3], kErrTimeout);
                        s_abort = 1;
                        break;
                    }
                }
            }
        }
    } else {
        // ----------------------------------------------------- compute warps
        const int tj = tid % TJ, tk = tid / TJ;
        const int jm = J * TJ + tj, km = K * TK + tk;   // mirrored pencil coordinates
        const bool live = tid < ncomp && jm < ny && km < nz;
        const int j = BWD ? ny - 1 - jm : jm, k = BWD ? nz - 1 - km : km;
        const long long plane = (long long)nx * ny;
        const long long row0 = (long long)nx * j + plane * k;   // real index of x = 0
        const long long oy = BWD ? -(long long)nx : (long long)nx;
        const long long oz = BWD ? -plane : plane;
        const bool needJ = live && tj == 0 && jm > 0;
        const bool needK = live && tk == 0 && km > 0;
        const int nct = ncw * 32;

        T rr[D], a0[D], a1[D], a2[D], di[D], vj[D], vk[D];
        auto load = [&](int d, int xm) {
            rr[d] = T(0); a0[d] = T(0); a1[d] = T(0); a2[d] = T(0); di[d] = T(1); vj[d] = T(0); vk[d] = T(0);
            if (!live || xm < 0 || xm >= nx) return;
            const long long c = row0 + (BWD ? nx - 1 - xm : xm);
            rr[d] = (T)__ldg(&rhs[c]);
            a0[d] = __ldg(&c0[c]);
            a1[d] = __ldg(&c1[c]);
            a2[d] = __ldg(&c2[c]);
            if (BWD) di[d] = __ldg(&dinv[c]);
            if (needJ) vj[d] = __ldcg(&out[c - oy]);
            if (needK) vk[d] = __ldcg(&out[c - oz]);
        };
        // loads at step t need producers to have completed min(t + D + TJ|TK, steps) steps
        auto ready = [&](int t) {
            if (tid == 0) {
                const int nJ = min(t + D + TJ, steps), nK = min(t + D + TK, steps);
                long long spins = 0;
                while (s_availJ < nJ || s_availK < nK) {
                    if (s_abort) break;
                    if (++spins > (kSpinLimit << 4)) {
                        atomicOr(&sync[3], kErrTimeout);
                        s_abort = 1;
                        break;
                    }
                }
                __threadfence_block();
            }
        };

        ready(0);
        compute_barrier(nct);
        const int skew = tj + tk;
#pragma unroll
        for (int d = 0; d < D; ++d) load(d, d - skew);
        T prev = T(0);
        for (int t = 0; t < steps; ++t) {
            if (t > 0) {
                ready(t);
                compute_barrier(nct);   // step t-1 complete: values in shared memory, producers ready
                if (tid == 0) st_release_cta_s32(&s_done, t);
            }
            const int xm = t - skew;
            if (live && xm >= 0 && xm < nx) {
                const T *smp = sm + ((t - 1) & 1) * ncomp;
                const T nj = tj > 0 ? smp[tk * TJ + tj - 1] : vj[0];
                const T nk = tk > 0 ? smp[(tk - 1) * TJ + tj] : vk[0];
                T s = rr[0] - a0[0] * prev - a1[0] * nj - a2[0] * nk;
                if (BWD) s *= di[0];
                out[row0 + (BWD ? nx - 1 - xm : xm)] = s;
                prev = s;
                sm[(t & 1) * ncomp + tk * TJ + tj] = s;
            }
#pragma unroll
            for (int d = 0; d < D - 1; ++d) {
                rr[d] = rr[d + 1]; a0[d] = a0[d + 1]; a1[d] = a1[d + 1]; a2[d] = a2[d + 1];
                di[d] = di[d + 1]; vj[d] = vj[d + 1]; vk[d] = vk[d + 1];
            }
            load(D - 1, xm + D);
        }
        compute_barrier(nct);
        if (tid == 0) st_release_cta_s32(&s_done, steps);
    }
    __syncthreads();
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
template <typename T> constexpr int ring_depth() { return sizeof(T) == 8 ? 4 : 8; }

template <typename T, typename TR>
void tiled_apply(ms_system &s, const T *coef, const T *dinv, const TR *r, T *y, T *z, cudaStream_t st) {
    const int nT = s.NJ * s.NK;
    const int ncomp = s.TJ * s.TK;
    const int threads = 32 * ((ncomp + 31) / 32) + 32;   // compute warps + one communication warp
    const size_t smem = 2 * (size_t)ncomp * sizeof(T);
    const int64_t n = s.n;
    const double nl = (double)s.nnz_lower;
    {
        KernelScope ks_(st, sizeof(T) == 8 ? "ilu_fwd" : "ilu_fwd32", nl * sizeof(T) + (double)n * (sizeof(TR) + sizeof(T)));
        k_tile_sweep<T, TR, false, ring_depth<T>()><<<nT, threads, smem, st>>>(
            s.nx, s.ny, s.nz, s.TJ, s.TK, s.NJ, s.tile_order.p, coef, coef + n, coef + 2 * n, nullptr, r, y,
            s.tile_prog.p, s.sync.p);
        MS_CHECK_LAUNCH();
    }
    KernelScope ks_(st, sizeof(T) == 8 ? "ilu_bwd" : "ilu_bwd32", nl * sizeof(T) + (double)n * 3 * sizeof(T));
    k_tile_sweep<T, T, true, ring_depth<T>()><<<nT, threads, smem, st>>>(s.nx, s.ny, s.nz, s.TJ, s.TK, s.NJ,
                                                              s.tile_order.p, coef + 3 * n, coef + 4 * n,
                                                              coef + 5 * n, dinv, y, z, s.tile_prog.p, s.sync.p);
    MS_CHECK_LAUNCH();
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

}  // namespace msgb
