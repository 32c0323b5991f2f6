// Row-parallel kernels on the ELL storage of A: two-point flux assembly
// (Sec. 3), residuals / SpMV with deterministic norms, the Jacobi smoother,
// restriction d = P^T r and prolongation x += P x_c (Eq. (11)).
//
// Layout: slot w of row i lives at [w*n + i], so a warp reading slot w of 32
// consecutive rows issues one coalesced 128/256-byte access.  Every
// reduction uses a fixed tree and a fixed block order, so results do not
// depend on scheduling.
#include <cfloat>

#include <algorithm>

#include "ms_internal.h"

namespace msgb {

namespace {

constexpr int kThreads = 256;

inline int blocks_for(int64_t n, int t = kThreads) { return (int)((n + t - 1) / t); }
// grid of the kernels that end in a deterministic block reduction: few enough
// blocks that the last-block hand-off (one counter increment per block) stays
// short, enough to keep every SM busy (4 per SM)
inline int reduce_grid(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>(blocks_for(n), 4 * 152)); }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Sum of v over the CTA (result valid in thread 0); fixed order.
__device__ __forceinline__ double block_sum(double v) {
    __shared__ double part[32];
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) part[wid] = v;
    __syncthreads();
    double s = 0.0;
    if (wid == 0) {
        s = (lane < (int)(blockDim.x >> 5)) ? part[lane] : 0.0;
        s = warp_sum(s);
    }
    __syncthreads();
    return s;
}

// Deterministic two-level reduction: each CTA stores its partial; the last
// CTA to finish adds the partials in index order and writes sqrt(sum).
__device__ __forceinline__ void finish_norm(double blk, double *red, unsigned int *cnt, double *out) {
    __shared__ bool last;
    if (threadIdx.x == 0) {
        red[blockIdx.x] = blk;
        __threadfence();
        unsigned int prev = atomicAdd(cnt, 1u);
        last = (prev == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double s = 0.0;
#pragma unroll 8   // independent loads in flight; the sum order is unchanged
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) s += __ldcg(&red[b]);
    s = block_sum(s);
    if (threadIdx.x == 0) {
        out[0] = sqrt(s);
        *cnt = 0u;
    }
}

// ------------------------------------------------------------- assembly
__global__ void k_check_perm(const double *perm, int64_t count, int *flag) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (; i < count; i += (int64_t)gridDim.x * blockDim.x) {
        double k = perm[i];
        if (!(k >= 0.0) || isinf(k)) atomicOr(flag, 1);
    }
}

__global__ void k_face_trans(int nf, const int *__restrict__ ga, const int *__restrict__ gb,
                             const int8_t *__restrict__ axis, const double *__restrict__ mult,
                             const int *__restrict__ fa, const int *__restrict__ fb, const double *__restrict__ perm,
                             const double *__restrict__ mob, const double *__restrict__ pprev, double dx, double dy,
                             double dz, double *__restrict__ T) {
    int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nf) return;
    const int ax = axis[f];
    const double h = ax == 0 ? dx : (ax == 1 ? dy : dz);
    const double area = ax == 0 ? dy * dz : (ax == 1 ? dx * dz : dx * dy);
    const double ta = perm[3 * (int64_t)ga[f] + ax] * area / (0.5 * h);
    const double tb = perm[3 * (int64_t)gb[f] + ax] * area / (0.5 * h);
    const double m = mult[f];
    double t = (ta > 0.0 && tb > 0.0 && m > 0.0) ? m / (1.0 / ta + 1.0 / tb) : 0.0;
    if (mob) {
        const int a = fa[f], b = fb[f];
        double lf;
        if (pprev && pprev[a] != pprev[b]) lf = pprev[a] > pprev[b] ? mob[a] : mob[b];
        else lf = 0.5 * (mob[a] + mob[b]);
        t *= lf;
    }
    T[f] = t;
}

// A_ii = sum of incident T, A_ij = -T_ij (unpinned); pinned copy drops the
// off-diagonals of row ref and column ref.
__global__ void k_row_assemble(int n, int W, int ref, const int *__restrict__ rf_ptr, const int *__restrict__ rf_face,
                               const uint8_t *__restrict__ rf_slot, const double *__restrict__ T,
                               const int *__restrict__ col, double *__restrict__ off_u, double *__restrict__ off_p,
                               double *__restrict__ diag) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int w = 0; w < W; ++w) off_u[(int64_t)w * n + i] = 0.0;
    double d = 0.0;
    for (int p = rf_ptr[i]; p < rf_ptr[i + 1]; ++p) {
        const double t = T[rf_face[p]];
        d += t;
        off_u[(int64_t)rf_slot[p] * n + i] -= t;
    }
    diag[i] = d;
    for (int w = 0; w < W; ++w) {
        const int64_t at = (int64_t)w * n + i;
        const int c = col[at];
        off_p[at] = (c != i && (i == ref || c == ref)) ? 0.0 : off_u[at];
    }
}

// ------------------------------------------------------------- SpMV family
// Row i of A v in slot order (diagonal first).  WM > 0: at most WM
// connections, every column and coefficient loaded before the gathers, so a
// row's loads are in flight together (the sum keeps its order).
template <int WM>
__device__ __forceinline__ double row_av(int n, int W, int i, const int *__restrict__ col,
                                         const double *__restrict__ off, double d, const double *__restrict__ v) {
    double s = d * v[i];
    if constexpr (WM > 0) {
        int c[WM];
        double a[WM];
#pragma unroll
        for (int w = 0; w < WM; ++w) {
            const int64_t at = (int64_t)w * n + i;
            c[w] = w < W ? col[at] : i;
            a[w] = w < W ? off[at] : 0.0;
        }
#pragma unroll
        for (int w = 0; w < WM; ++w)
            if (w < W) s += a[w] * v[c[w]];
    } else {
        for (int w = 0; w < W; ++w) {
            const int64_t at = (int64_t)w * n + i;
            s += off[at] * v[col[at]];
        }
    }
    return s;
}

template <int WM>
__global__ void k_spmv(int n, int W, const int *__restrict__ col, const double *__restrict__ off,
                       const double *__restrict__ diag, const double *__restrict__ x, double *__restrict__ y) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    y[i] = row_av<WM>(n, W, i, col, off, diag[i], x);
}

// r = q - A x and ||r||_2
template <int WM>
__global__ void k_residual(int n, int W, const int *__restrict__ col, const double *__restrict__ off,
                           const double *__restrict__ diag, const double *__restrict__ q,
                           const double *__restrict__ x, double *__restrict__ r, float *__restrict__ r32,
                           double *red, unsigned int *cnt, double *norm_out) {
    double ss = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double s = row_av<WM>(n, W, i, col, off, diag[i], x);
        const double ri = q[i] - s;
        r[i] = ri;
        if (r32) r32[i] = (float)ri;
        ss += ri * ri;
    }
    if (norm_out) finish_norm(block_sum(ss), red, cnt, norm_out);
}

// r -= A z ; x += z   (after a smoother correction z)
template <int WM>
__global__ void k_residual_update(int n, int W, const int *__restrict__ col, const double *__restrict__ off,
                                  const double *__restrict__ diag, double *__restrict__ r, double *__restrict__ x,
                                  const double *__restrict__ z) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double zi = z[i];
    const double s = row_av<WM>(n, W, i, col, off, diag[i], z);
    r[i] -= s;
    x[i] += zi;
}

// mixed form: r32 = r - A32 z (single precision), x += z
__global__ void k_residual_update32(int n, int W, const int *__restrict__ col, const float *__restrict__ off,
                                    const float *__restrict__ diag, const double *__restrict__ r,
                                    float *__restrict__ r32, double *__restrict__ x, const float *__restrict__ z) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float zi = z[i];
    float s = diag[i] * zi;
    for (int w = 0; w < W; ++w) {
        const int64_t at = (int64_t)w * n + i;
        s = fmaf(off[at], z[col[at]], s);
    }
    r32[i] = (float)r[i] - s;
    x[i] += (double)zi;
}

__global__ void k_jacobi(int n, const double *__restrict__ r, const double *__restrict__ diag, double omega,
                         double *__restrict__ z) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) z[i] = omega * r[i] / diag[i];
}

__global__ void k_jacobi32(int n, const double *__restrict__ r, const float *__restrict__ diag, float omega,
                           float *__restrict__ z) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) z[i] = omega * (float)r[i] / diag[i];
}

__global__ void k_norm2(int n, const double *__restrict__ v, double *red, unsigned int *cnt, double *out) {
    double a = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double x = v[i];
        a += x * x;
    }
    finish_norm(block_sum(a), red, cnt, out);
}

__global__ void k_sub(int n, const double *a, const double *b, double *c) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) c[i] = a[i] - b[i];
}

__global__ void k_set_zero_at(double *v, int idx) {
    if (threadIdx.x == 0 && blockIdx.x == 0) v[idx] = 0.0;
}

__global__ void k_widen(const float *a, double *b, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (; i < n; i += (int64_t)gridDim.x * blockDim.x) b[i] = (double)a[i];
}

__global__ void k_to_float(const double *a, float *b, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (; i < n; i += (int64_t)gridDim.x * blockDim.x) b[i] = (float)a[i];
}

// ------------------------------------------------------ restrict / prolong
// d_j = sum over row j of R (the support of block j with weights P_ij, or the
// cells of block j with unit weights) of R_ji r_i, one warp per column
// chunk: chunk sums in a fixed lane order, then the last chunk of a column to
// finish adds the column's chunk sums in chunk order (deterministic; balanced
// however uneven the supports are).  ACC is the accumulation type.
template <typename TV, typename TR, typename TD, typename ACC>
__global__ void k_restrict_ch(int nch, const int *__restrict__ ch_beg, const int *__restrict__ ch_col,
                              const int *__restrict__ ch_ptr, const int *__restrict__ cptr,
                              const int *__restrict__ ccell, const TV *__restrict__ cval, const TR *__restrict__ r,
                              double *part, unsigned *cnt, TD *__restrict__ d) {
    const int c = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (c >= nch) return;
    const int j = ch_col[c];
    const int e0 = ch_beg[c], e1 = min(e0 + kColChunk, cptr[j + 1]);
    ACC s = ACC(0);
    if (cval)
        for (int e = e0 + lane; e < e1; e += 32) s += (ACC)cval[e] * (ACC)r[ccell[e]];
    else   // unit weights: the finite-volume restriction sums the block's cells
        for (int e = e0 + lane; e < e1; e += 32) s += (ACC)r[ccell[e]];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane != 0) return;
    const int q0 = ch_ptr[j], k = ch_ptr[j + 1] - q0;
    if (k == 1) {
        d[j] = (TD)s;
        return;
    }
    part[c] = (double)s;
    __threadfence();
    if (atomicAdd(&cnt[j], 1u) == (unsigned)(k - 1)) {   // last chunk of column j
        __threadfence();
        ACC t = ACC(0);
#pragma unroll 4
        for (int q = q0; q < q0 + k; ++q) t += (ACC)__ldcg(part + q);
        d[j] = (TD)t;
        cnt[j] = 0u;
    }
}

// x_i += sum_s P_{i,s} x_c[block(s)]; BM bounds the slots so that every
// slot's block id and value load before the gathers (padding slots come last)
template <typename TV, typename TC, int BM>
__global__ void k_prolong(int n, int B, const int *__restrict__ pid, const TV *__restrict__ pval,
                          const TC *__restrict__ xc, double *__restrict__ x) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    TC s = 0;
    if (BM > 0) {
        int j[BM > 0 ? BM : 1];
        TV pv[BM > 0 ? BM : 1];
#pragma unroll
        for (int t = 0; t < BM; ++t) {
            const int64_t at = (int64_t)t * n + i;
            j[t] = t < B ? pid[at] : kSlotPad;
            pv[t] = t < B ? pval[at] : TV(0);
        }
#pragma unroll
        for (int t = 0; t < BM; ++t)
            if (j[t] != kSlotPad) s += (TC)pv[t] * xc[j[t]];
    } else {
        for (int t = 0; t < B; ++t) {
            const int64_t at = (int64_t)t * n + i;
            const int jj = pid[at];
            if (jj == kSlotPad) break;
            s += (TC)pval[at] * xc[jj];
        }
    }
    x[i] += (double)s;
}

}  // namespace

// ---------------------------------------------------------------- launchers
void launch_check_perm(const double *perm, int64_t count, int *flag, cudaStream_t st) {
    int blocks = (int)std::min<int64_t>((count + kThreads - 1) / kThreads, 4096);
    k_check_perm<<<std::max(blocks, 1), kThreads, 0, st>>>(perm, count, flag);
    MS_CHECK_LAUNCH();
}

void launch_face_trans(ms_system &s, const double *perm, const double *mob, const double *pprev, cudaStream_t st) {
    if (s.nf == 0) return;
    KernelScope ks_(st, "face_trans", (double)s.nf * (4 + 4 + 1 + 8 + 16 + 8) + (mob ? (double)s.nf * 2 * (4 + 8 + (pprev ? 8 : 0)) : 0.0));
    k_face_trans<<<blocks_for(s.nf), kThreads, 0, st>>>(s.nf, s.f_ga.p, s.f_gb.p, s.f_axis.p, s.f_mult.p, s.f_a.p,
                                                         s.f_b.p, perm, mob, pprev, s.dx, s.dy, s.dz, s.f_T.p);
    MS_CHECK_LAUNCH();
}

void launch_row_assemble(ms_system &s, cudaStream_t st) {
    KernelScope ks_(st, "row_assemble", (double)s.n * (4 + 8) + (double)s.nf * 2 * (4 + 1 + 8) + (double)s.W * s.n * (4 + 3 * 8));
    k_row_assemble<<<blocks_for(s.n), kThreads, 0, st>>>(s.n, s.W, s.ref, s.rf_ptr.p, s.rf_face.p, s.rf_slot.p,
                                                          s.f_T.p, s.col.p, s.off_u.p, s.off_p.p, s.diag.p);
    MS_CHECK_LAUNCH();
}

void launch_spmv(const ms_system &s, const double *x, double *y, cudaStream_t st) {
    KernelScope ks_(st, "spmv", (double)s.n * (8 + 8 + 8) + (double)s.W * s.n * (4 + 8));
    if (s.W <= 6) k_spmv<6><<<blocks_for(s.n), kThreads, 0, st>>>(s.n, s.W, s.col.p, s.off_p.p, s.diag.p, x, y);
    else k_spmv<0><<<blocks_for(s.n), kThreads, 0, st>>>(s.n, s.W, s.col.p, s.off_p.p, s.diag.p, x, y);
    MS_CHECK_LAUNCH();
}

void launch_residual(const ms_system &s, const double *q, const double *x, double *r, double *red,
                     unsigned int *cnt, double *norm_out, cudaStream_t st, float *r32) {
    KernelScope ks_(st, "residual", (double)s.n * (8 + 8 + 8 + 8 + (r32 ? 4 : 0)) + (double)s.W * s.n * (4 + 8));
    if (s.W <= 6)
        k_residual<6><<<reduce_grid(s.n), kThreads, 0, st>>>(s.n, s.W, s.col.p, s.off_p.p, s.diag.p, q, x, r, r32, red,
                                                              cnt, norm_out);
    else
        k_residual<0><<<reduce_grid(s.n), kThreads, 0, st>>>(s.n, s.W, s.col.p, s.off_p.p, s.diag.p, q, x, r, r32, red,
                                                              cnt, norm_out);
    MS_CHECK_LAUNCH();
}

void launch_residual_update(const ms_system &s, double *r, double *x, const double *z, cudaStream_t st) {
    KernelScope ks_(st, "residual_update", (double)s.n * (8 + 8 + 16 + 16) + (double)s.W * s.n * (4 + 8));
    if (s.W <= 6) k_residual_update<6><<<blocks_for(s.n), kThreads, 0, st>>>(s.n, s.W, s.col.p, s.off_p.p, s.diag.p, r, x, z);
    else k_residual_update<0><<<blocks_for(s.n), kThreads, 0, st>>>(s.n, s.W, s.col.p, s.off_p.p, s.diag.p, r, x, z);
    MS_CHECK_LAUNCH();
}

void launch_residual_update32(const ms_system &s, const double *r, float *r32, double *x, const float *z,
                              cudaStream_t st) {
    KernelScope ks_(st, "residual_update32", (double)s.n * (4 + 4 + 8 + 4 + 16) + (double)s.W * s.n * (4 + 4));
    k_residual_update32<<<blocks_for(s.n), kThreads, 0, st>>>(s.n, s.W, s.col.p, s.off_p32.p, s.diag32.p, r, r32,
                                                               x, z);
    MS_CHECK_LAUNCH();
}

void launch_jacobi(const ms_system &s, const double *r, double *z, double omega, cudaStream_t st) {
    KernelScope ks_(st, "jacobi", (double)s.n * 24);
    k_jacobi<<<blocks_for(s.n), kThreads, 0, st>>>(s.n, r, s.diag.p, omega, z);
    MS_CHECK_LAUNCH();
}

void launch_jacobi32(const ms_system &s, const double *r, float *z, float omega, cudaStream_t st) {
    KernelScope ks_(st, "jacobi32", (double)s.n * 16);
    k_jacobi32<<<blocks_for(s.n), kThreads, 0, st>>>(s.n, r, s.diag32.p, omega, z);
    MS_CHECK_LAUNCH();
}

namespace {
// End of a Richardson cycle inside a graph: count the cycle, record the
// relative residual ||q - A x|| / ||q|| (norms[1] / norms[0]) and keep the
// loop going while it is above tol, finite, and under the cycle cap.
__global__ void k_cycle_control(const double *norms, double tol, int max_iter, int *ctl_it, double *ctl_res,
                                double *hist, cudaGraphConditionalHandle handle) {
    const int it = *ctl_it + 1;
    *ctl_it = it;
    const double res = norms[0] > 0.0 ? norms[1] / norms[0] : 0.0;
    *ctl_res = res;
    if (hist) hist[it] = res;
    cudaGraphSetConditional(handle, (res > tol && it < max_iter && res == res) ? 1u : 0u);
}
}  // namespace

void launch_cycle_control(const double *norms, double tol, int max_iter, int *ctl_it, double *ctl_res, double *hist,
                          cudaGraphConditionalHandle handle, cudaStream_t st) {
    KernelScope ks_(st, "cycle_control", 0.0);
    k_cycle_control<<<1, 1, 0, st>>>(norms, tol, max_iter, ctl_it, ctl_res, hist, handle);
    MS_CHECK_LAUNCH();
}

namespace {
// h[i] = sum_l V[i n + l] w[l] for i < k (Krylov basis against one vector):
// each block forms its partial sums of all k products over a grid-stride
// slice, then the last block to finish adds each product's partials in block
// order (deterministic).
__global__ void k_multidot(int n, int k, const double *__restrict__ V, const double *__restrict__ w, double *red,
                           unsigned int *cnt, double *h) {
    for (int i = 0; i < k; ++i) {
        double a = 0.0;
        const double *vi = V + (int64_t)i * n;
        for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < n; l += gridDim.x * blockDim.x) a += vi[l] * w[l];
        a = block_sum(a);
        if (threadIdx.x == 0) red[(int64_t)blockIdx.x * k + i] = a;
    }
    __shared__ bool last;
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(cnt, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int i = wid; i < k; i += (int)(blockDim.x >> 5)) {
        double t = 0.0;
#pragma unroll 8
        for (int b = lane; b < (int)gridDim.x; b += 32) t += __ldcg(&red[(int64_t)b * k + i]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
        if (lane == 0) h[i] = t;
    }
    if (threadIdx.x == 0) *cnt = 0u;
}

// The same products with the vectors taken 8 at a time (blockIdx.y = group of
// 8): each thread keeps 8 partial sums over a grid-stride slice, warp trees and
// the block's warps in order give the block partials, and the last block of
// each group adds its group's partials in block order (deterministic).
// Warp sums of eight accumulators with nine additions per lane instead of
// forty: halves of the set are exchanged at lane distances 16, 8 and 4 (a
// transposing butterfly), then the one accumulator left is summed over
// distances 2 and 1.  Lanes pair exactly as in a shuffle-down tree (the
// partner's value is added second on one side, first on the other, and a + b
// equals b + a), so every sum is the same bit for bit.  Accumulator i ends in
// lanes 4i .. 4i+3.
__device__ __forceinline__ double warp_sum8(const double (&acc)[8], int lane) {
    double a4[4], a2[2];
    const bool h16 = lane & 16, h8 = lane & 8, h4 = lane & 4;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const double keep = h16 ? acc[4 + j] : acc[j];
        const double send = h16 ? acc[j] : acc[4 + j];
        a4[j] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
    }
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        const double keep = h8 ? a4[2 + j] : a4[j];
        const double send = h8 ? a4[j] : a4[2 + j];
        a2[j] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
    }
    double a = (h4 ? a2[1] : a2[0]) + __shfl_xor_sync(0xffffffffu, h4 ? a2[0] : a2[1], 4);
    a += __shfl_xor_sync(0xffffffffu, a, 2);
    a += __shfl_xor_sync(0xffffffffu, a, 1);
    return a;
}

__global__ void __launch_bounds__(256) k_multidot8(int n, int k, const double *__restrict__ V,
                                                   const double *__restrict__ w, double *red, unsigned int *cnt,
                                                   double *h) {
    const int i0 = blockIdx.y * 8;
    const int kk = min(8, k - i0);
    double acc[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) acc[i] = 0.0;
    if (kk == 8) {
        for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < n; l += gridDim.x * blockDim.x) {
            const double wl = __ldg(w + l);
            double vv[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) vv[i] = __ldcs(V + (int64_t)(i0 + i) * n + l);
#pragma unroll
            for (int i = 0; i < 8; ++i) acc[i] += vv[i] * wl;
        }
    } else {   // the last group: no multiply-adds for absent vectors (FP64 is the scarce pipe)
        for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < n; l += gridDim.x * blockDim.x) {
            const double wl = __ldg(w + l);
#pragma unroll
            for (int i = 0; i < 8; ++i)
                if (i < kk) acc[i] += __ldcs(V + (int64_t)(i0 + i) * n + l) * wl;
        }
    }
    __shared__ double part[8][8];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    {
        const double a = warp_sum8(acc, lane);
        if ((lane & 3) == 0) part[wid][lane >> 2] = a;
    }
    __syncthreads();
    double *rg = red + (int64_t)blockIdx.y * gridDim.x * 8;
    if (threadIdx.x < 8) {
        double a = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) a += part[q][threadIdx.x];
        rg[(int64_t)blockIdx.x * 8 + threadIdx.x] = a;
    }
    __shared__ bool last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(cnt + blockIdx.y, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    if (wid < kk) {
        double t = 0.0;
#pragma unroll 8   // independent loads in flight; the sum order is unchanged
        for (int b = lane; b < (int)gridDim.x; b += 32) t += __ldcg(&rg[(int64_t)b * 8 + wid]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
        if (lane == 0) h[i0 + wid] = t;
    }
    if (threadIdx.x == 0) cnt[blockIdx.y] = 0u;
}

// y[l] += sign * sum_{i<k} c[i] V[i n + l]   (c on the device, k <= 128)
__global__ void k_multiaxpy(int n, int k, const double *__restrict__ V, const double *__restrict__ c, double sign,
                            double *__restrict__ y, const int *__restrict__ kdev) {
    if (kdev) k = min(k, *kdev);   // count known on the device only (GMRES inside a graph)
    __shared__ double cs[128];
    for (int i = threadIdx.x; i < k; i += blockDim.x) cs[i] = sign * c[i];
    __syncthreads();
    for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < n; l += gridDim.x * blockDim.x) {
        double a = y[l];
        int i = 0;
        for (; i + 8 <= k; i += 8) {   // eight vectors' loads in flight, summed in order
            double v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) v[u] = __ldcs(V + (int64_t)(i + u) * n + l);
#pragma unroll
            for (int u = 0; u < 8; ++u) a += cs[i + u] * v[u];
        }
        for (; i < k; ++i) a += cs[i] * V[(int64_t)i * n + l];
        y[l] = a;
    }
}

// y[l] += sign * sum_{i<k} c[i] V[i n + l], then ||y||_2 (the last
// Gram-Schmidt pass of an Arnoldi step and the new vector's norm in one read)
__global__ void k_multiaxpy_norm(int n, int k, const double *__restrict__ V, const double *__restrict__ c,
                                 double sign, double *__restrict__ y, double *red, unsigned int *cnt, double *norm_out) {
    __shared__ double cs[128];
    for (int i = threadIdx.x; i < k; i += blockDim.x) cs[i] = sign * c[i];
    __syncthreads();
    double ss = 0.0;
    for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < n; l += gridDim.x * blockDim.x) {
        double a = y[l];
        int i = 0;
        for (; i + 8 <= k; i += 8) {   // eight vectors' loads in flight, summed in order
            double v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) v[u] = __ldcs(V + (int64_t)(i + u) * n + l);
#pragma unroll
            for (int u = 0; u < 8; ++u) a += cs[i + u] * v[u];
        }
        for (; i < k; ++i) a += cs[i] * V[(int64_t)i * n + l];
        y[l] = a;
        ss += a * a;
    }
    finish_norm(block_sum(ss), red, cnt, norm_out);
}

__global__ void k_scale(int n, const double *__restrict__ x, double a, double *__restrict__ y) {
    for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < n; l += gridDim.x * blockDim.x) y[l] = a * x[l];
}

int stride_grid(int n) { return std::max(1, std::min((n + kThreads - 1) / kThreads, 4 * 152)); }
constexpr int kDotGroups = 16;   // up to 128 vectors in groups of 8
}  // namespace

int multidot_blocks(int n) { return stride_grid(n); }

void launch_multidot(int n, int k, const double *V, const double *w, double *red, unsigned int *cnt, double *h,
                     cudaStream_t st) {
    KernelScope ks_(st, "krylov_dot", (double)(k + 1) * n * 8);
    if (k <= 8 * kDotGroups) k_multidot8<<<dim3(stride_grid(n), (k + 7) / 8), kThreads, 0, st>>>(n, k, V, w, red, cnt, h);
    else k_multidot<<<stride_grid(n), kThreads, 0, st>>>(n, k, V, w, red, cnt, h);
    MS_CHECK_LAUNCH();
}

void launch_multiaxpy(int n, int k, const double *V, const double *c, double sign, double *y, cudaStream_t st,
                      const int *kdev) {
    KernelScope ks_(st, "krylov_axpy", (double)(k + 2) * n * 8);
    k_multiaxpy<<<2 * stride_grid(n), kThreads, 0, st>>>(n, k, V, c, sign, y, kdev);
    MS_CHECK_LAUNCH();
}

namespace {
__global__ void k_scale_dev(int n, const double *__restrict__ x, const double *__restrict__ a,
                            double *__restrict__ y) {
    const double f = *a;
    for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < n; l += gridDim.x * blockDim.x) y[l] = f * x[l];
}

// GMRES bookkeeping on the device (one thread), the same arithmetic as the
// host loop: restart begin, one Arnoldi step's Hessenberg column with its
// Givens rotations and convergence test, the small triangular solve, and the
// restart's true-residual test.  Each sets the graph condition that lets the
// next step (or restart) run.
__global__ void k_gmres_begin(GmresDev G, const double *beta_norm, const cudaGraphConditionalHandle *steps) {
    const double beta = *beta_norm;
    for (int i = 0; i <= G.m; ++i) G.g[i] = 0.0;
    G.g[0] = beta;
    *G.k = 0;
    *G.scal = beta > 0.0 ? 1.0 / beta : 0.0;
    const int stop = !(beta > 0.0) || *G.it >= G.max_iter;
    *G.stop = stop;
    cudaGraphSetConditional(steps[0], stop ? 0u : 1u);
    for (int i = 1; i < G.m; ++i) cudaGraphSetConditional(steps[i], 0u);   // each opened by its predecessor
}

__global__ void k_gmres_step(GmresDev G, int j, const double *h1, const double *h2, const double *hn_dev,
                             const cudaGraphConditionalHandle *steps) {
    const int m = G.m;
    double *H = G.H;
    for (int i = 0; i <= j; ++i) H[(size_t)i * m + j] = h1[i] + h2[i];
    const double hn = *hn_dev;
    if (!(hn == hn)) {
        *G.err = 1;
        *G.stop = 1;
        return;   // the next step stays closed
    }
    H[(size_t)(j + 1) * m + j] = hn;
    *G.scal = hn > 0.0 ? 1.0 / hn : 0.0;
    gmres_givens(H, m, j, G.cs, G.sn, G.g);
    *G.k = j + 1;
    const int it = *G.it + 1;
    *G.it = it;
    const double res = fabs(G.g[j + 1]) / G.nq;
    *G.res = res;
    if (G.hist) G.hist[it] = res;
    const int stop = res <= G.tol || hn == 0.0 || it >= G.max_iter;
    *G.stop = stop;
    if (j + 1 < m) cudaGraphSetConditional(steps[j + 1], stop ? 0u : 1u);
}

// H(0:k, 0:k) y = g(0:k) by back substitution
__global__ void k_gmres_solve(GmresDev G) { gmres_back_solve(G.H, G.m, *G.k, G.g, G.y); }

__global__ void k_gmres_restart(GmresDev G, const double *beta_norm, cudaGraphConditionalHandle outer) {
    const double beta = *beta_norm;
    const double res = beta / G.nq;
    *G.res = res;
    const int it = *G.it;
    if (G.hist) G.hist[it] = res;
    if (!(res == res)) *G.err = 1;
    // every restart advances the iteration count, so more than max_iter + 1
    // restarts cannot happen; the count stops the loop even if one did not
    const int r = ++*G.restarts;
    cudaGraphSetConditional(outer,
                            (res > G.tol && it < G.max_iter && res == res && !*G.err && r <= G.max_iter) ? 1u : 0u);
}
}  // namespace

void launch_multiaxpy_norm(int n, int k, const double *V, const double *c, double sign, double *y, double *red,
                           unsigned int *cnt, double *norm_out, cudaStream_t st) {
    KernelScope ks_(st, "krylov_axpy", (double)(k + 2) * n * 8);
    // one partial sum per block in red, which holds ceil(n / 256) of them:
    // the grid is the reduction grid (never more blocks than that)
    k_multiaxpy_norm<<<reduce_grid(n), kThreads, 0, st>>>(n, k, V, c, sign, y, red, cnt, norm_out);
    MS_CHECK_LAUNCH();
}

void launch_scale_dev(int n, const double *x, const double *a, double *y, cudaStream_t st) {
    k_scale_dev<<<stride_grid(n), kThreads, 0, st>>>(n, x, a, y);
    MS_CHECK_LAUNCH();
}

void launch_gmres_begin(const GmresDev &G, const double *beta_norm, const cudaGraphConditionalHandle *steps,
                        cudaStream_t st) {
    k_gmres_begin<<<1, 1, 0, st>>>(G, beta_norm, steps);
    MS_CHECK_LAUNCH();
}

void launch_gmres_step(const GmresDev &G, int j, const double *h1, const double *h2, const double *hn,
                       const cudaGraphConditionalHandle *steps, cudaStream_t st) {
    k_gmres_step<<<1, 1, 0, st>>>(G, j, h1, h2, hn, steps);
    MS_CHECK_LAUNCH();
}

void launch_gmres_solve(const GmresDev &G, cudaStream_t st) {
    k_gmres_solve<<<1, 1, 0, st>>>(G);
    MS_CHECK_LAUNCH();
}

void launch_gmres_restart(const GmresDev &G, const double *beta_norm, cudaGraphConditionalHandle outer,
                          cudaStream_t st) {
    k_gmres_restart<<<1, 1, 0, st>>>(G, beta_norm, outer);
    MS_CHECK_LAUNCH();
}

void launch_scale(int n, const double *x, double a, double *y, cudaStream_t st) {
    k_scale<<<stride_grid(n), kThreads, 0, st>>>(n, x, a, y);
    MS_CHECK_LAUNCH();
}

void launch_norm2(const double *v, int n, double *red, unsigned int *cnt, double *out, cudaStream_t st) {
    KernelScope ks_(st, "norm2", (double)n * 8);
    k_norm2<<<reduce_grid(n), kThreads, 0, st>>>(n, v, red, cnt, out);
    MS_CHECK_LAUNCH();
}

void launch_sub(const double *a, const double *b, double *c, int n, cudaStream_t st) {
    k_sub<<<blocks_for(n), kThreads, 0, st>>>(n, a, b, c);
    MS_CHECK_LAUNCH();
}

void launch_scatter_zero(double *v, int idx, cudaStream_t st) {
    k_set_zero_at<<<1, 32, 0, st>>>(v, idx);
    MS_CHECK_LAUNCH();
}

void launch_to_float(const double *a, float *b, int64_t n, cudaStream_t st) {
    if (n <= 0) return;
    int blocks = (int)std::min<int64_t>((n + kThreads - 1) / kThreads, 8192);
    k_to_float<<<blocks, kThreads, 0, st>>>(a, b, n);
    MS_CHECK_LAUNCH();
}

void launch_widen(const float *a, double *b, int64_t n, cudaStream_t st) {
    if (n <= 0) return;
    int blocks = (int)std::min<int64_t>((n + kThreads - 1) / kThreads, 8192);
    k_widen<<<blocks, kThreads, 0, st>>>(a, b, n);
    MS_CHECK_LAUNCH();
}

void launch_narrow(const double *a, float *b, int64_t n, cudaStream_t st) { launch_to_float(a, b, n, st); }

void build_column_chunks(const std::vector<int> &cptr, int M, int C, std::vector<int> &beg, std::vector<int> &col,
                         std::vector<int> &ptr, std::vector<int> *slot, int *multi) {
    beg.clear();
    col.clear();
    ptr.assign((size_t)M + 1, 0);
    if (slot) slot->clear();
    int nm = 0;
    for (int j = 0; j < M; ++j) {
        const int len = cptr[j + 1] - cptr[j];
        const int k = std::max(1, (len + C - 1) / C);
        ptr[j + 1] = ptr[j] + k;
        for (int t = 0; t < k; ++t) {
            beg.push_back(cptr[j] + t * C);
            col.push_back(j);
            if (slot) slot->push_back(k > 1 ? nm++ : -1);
        }
    }
    if (multi) *multi = nm;
}

void launch_restrict(const RestrictView &v, const double *r, double *d, cudaStream_t st) {
    KernelScope ks_(st, "restrict", (double)v.nnz * (4 + (v.cval ? 8 : 0) + 8) + (double)v.M * (8 + 4));
    const int g = (int)(((int64_t)v.n_chunks * 32 + kThreads - 1) / kThreads);
    k_restrict_ch<double, double, double, double><<<g, kThreads, 0, st>>>(
        v.n_chunks, v.ch_beg, v.ch_col, v.ch_ptr, v.cptr, v.ccell, v.cval, r, v.ch_part, v.ch_cnt, d);
    MS_CHECK_LAUNCH();
}

void launch_restrict32(const RestrictView &v, const float *r, float *d, cudaStream_t st) {
    KernelScope ks_(st, "restrict32", (double)v.nnz * (4 + (v.cval32 ? 4 : 0) + 4) + (double)v.M * (4 + 4));
    const int g = (int)(((int64_t)v.n_chunks * 32 + kThreads - 1) / kThreads);
    k_restrict_ch<float, float, float, float><<<g, kThreads, 0, st>>>(
        v.n_chunks, v.ch_beg, v.ch_col, v.ch_ptr, v.cptr, v.ccell, v.cval32, r, v.ch_part, v.ch_cnt, d);
    MS_CHECK_LAUNCH();
}

RestrictView restrict_view(const ms_coarse &c) {
    RestrictView v;
    v.M = c.M;
    if (c.restriction == MS_RESTRICT_FV) {
        v.nnz = c.fv_h_cptr.empty() ? 0 : c.fv_h_cptr.back();
        v.n_chunks = c.fv_n_chunks;
        v.ch_beg = c.fv_ch_beg.p; v.ch_col = c.fv_ch_col.p; v.ch_ptr = c.fv_ch_ptr.p;
        v.cptr = c.fv_cptr.p; v.ccell = c.fv_ccell.p;
        v.ch_part = c.fv_ch_part.p; v.ch_cnt = c.fv_ch_cnt.p;
        return v;
    }
    const ms_basis &b = *c.basis;
    v.nnz = b.nnz;
    v.n_chunks = b.n_chunks;
    v.ch_beg = b.ch_beg.p; v.ch_col = b.ch_col.p; v.ch_ptr = b.ch_ptr.p;
    v.cptr = b.cptr.p; v.ccell = b.ccell.p;
    v.cval = b.cval.p; v.cval32 = b.cval32.p;
    v.ch_part = b.ch_part.p; v.ch_cnt = b.ch_cnt.p;
    return v;
}

void launch_prolong(const ms_basis &b, int n, const double *xc, double *x, cudaStream_t st) {
    KernelScope ks_(st, "prolong", (double)b.B * n * (4 + 8) + (double)b.M * 8 + (double)n * 16);
    if (b.B <= 8) k_prolong<double, double, 8><<<blocks_for(n), kThreads, 0, st>>>(n, b.B, b.pid.p, b.pval.p, xc, x);
    else k_prolong<double, double, 0><<<blocks_for(n), kThreads, 0, st>>>(n, b.B, b.pid.p, b.pval.p, xc, x);
    MS_CHECK_LAUNCH();
}

void launch_prolong32(const ms_basis &b, int n, const float *xc, double *x, cudaStream_t st) {
    KernelScope ks_(st, "prolong32", (double)b.B * n * (4 + 4) + (double)b.M * 4 + (double)n * 16);
    if (b.B <= 8) k_prolong<float, float, 8><<<blocks_for(n), kThreads, 0, st>>>(n, b.B, b.pid.p, b.pval32.p, xc, x);
    else k_prolong<float, float, 0><<<blocks_for(n), kThreads, 0, st>>>(n, b.B, b.pid.p, b.pval32.p, xc, x);
    MS_CHECK_LAUNCH();
}

}  // namespace msgb
