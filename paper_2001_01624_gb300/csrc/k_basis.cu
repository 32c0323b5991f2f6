// Prolongation bases and Galerkin coarse operators.
//
// MsRSB smoothing (Sec. 5.1; Sec. 5 requirements 2-3): from the block
// indicator, every iteration updates each basis on its support from the old
// values,  P_ij <- P_ij - omega (A P_j)_i / A_ii  (i in S_j; 0 elsewhere),
// then renormalises every cell so that sum_j P_ij = 1.  One thread per cell
// does both steps for all bases covering the cell: the cell's slot list and
// its neighbours' slot lists are sorted by block id, so (A P_j)_i is a merge
// of at most 1 + W short sorted lists.  Supports are implicit in the slot
// pattern (a cell without a slot for block j is outside S_j), so confinement
// holds by construction.
//
// Galerkin operator (Eq. (10), R = P^T): (A P)_il is formed per cell as the
// merge of the slot lists of the cell and its neighbours; then row j of
// A_c = P^T (A P) is accumulated by one warp over the support of block j in
// shared memory, in a fixed order (deterministic), and A_c is symmetrised.
#include <cstdlib>

#include "ms_internal.h"
#include "msrsb_cell.cuh"

namespace msgb {

namespace {

constexpr int kThreads = 256;
inline int blocks_for(int64_t n, int t = kThreads) { return (int)((n + t - 1) / t); }

__global__ void k_basis_init(int64_t total, const unsigned char *__restrict__ is_home, double *pv) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (; e < total; e += (int64_t)gridDim.x * blockDim.x) pv[e] = is_home[e] ? 1.0 : 0.0;
}

__global__ void k_basis_init32(int64_t total, const unsigned char *__restrict__ is_home, float *pv) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (; e < total; e += (int64_t)gridDim.x * blockDim.x) pv[e] = is_home[e] ? 1.0f : 0.0f;
}

// One MsRSB iteration for all bases, fused with the partition-of-unity pass.
template <typename T, int BM>
__global__ void __launch_bounds__(kThreads) k_msrsb(int n, int W, int B, const int *__restrict__ col,
                                                    const T *__restrict__ off, const T *__restrict__ diag,
                                                    const int *__restrict__ pid, T *bufA, T *bufB,
                                                    const T *__restrict__ odiag, unsigned long long *ctl) {
    if (*(volatile const unsigned long long *)ctl) return;   // smoothing finished: no-op
    const bool odd = ctl[1] & 1ull;                            // iterations done so far
    const T *__restrict__ pin = odd ? bufB : bufA;
    T *__restrict__ pout = odd ? bufA : bufB;
    unsigned long long *maxinc = ctl + 2;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long inck = 0ull;   // key of the largest |increment|
    if (i < n) {
        int ids[BM];
        T v[BM], acc[BM];
        const T d = diag[i];
#pragma unroll
        for (int s = 0; s < BM; ++s) {
            ids[s] = s < B ? pid[(int64_t)s * n + i] : kSlotPad;
            v[s] = ids[s] != kSlotPad ? pin[(int64_t)s * n + i] : T(0);
            acc[s] = d * v[s];
        }
        for (int w = 0; w < W; ++w) {
            const int k = col[(int64_t)w * n + i];
            if (k == i) continue;
            const T a = off[(int64_t)w * n + i];
            int t = 0;
            int kid = pid[k];
#pragma unroll
            for (int s = 0; s < BM; ++s) {
                if (ids[s] != kSlotPad) {
                    while (kid < ids[s]) {
                        ++t;
                        kid = t < B ? pid[(int64_t)t * n + k] : kSlotPad;
                    }
                    if (kid == ids[s]) acc[s] += a * pin[(int64_t)t * n + k];
                }
            }
        }
        // omega / A_ii precomputed per smoothing run; one reciprocal for the
        // partition-of-unity scale
        const T od = odiag[i];
        T sum = 0;
#pragma unroll
        for (int s = 0; s < BM; ++s) {
            if (ids[s] != kSlotPad) {
                acc[s] = v[s] - od * acc[s];
                sum += acc[s];
            }
        }
        T rs;
        if constexpr (sizeof(T) == 8) rs = recip_series(sum);
        else rs = T(1) / sum;
#pragma unroll
        for (int s = 0; s < BM; ++s) {
            if (ids[s] != kSlotPad) {
                const T nv = acc[s] * rs;
                inck = max(inck, abs_key(nv - v[s]));
                pout[(int64_t)s * n + i] = nv;
            }
        }
    }
    // CTA max then one atomic per CTA (integer keys)
    __shared__ unsigned long long wmax[kThreads / 32];
    unsigned long long m = abs_key(key_value<T>(inck));   // key of the value as a double
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_down_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long mm = 0ull;
        for (int q = 0; q < kThreads / 32; ++q) mm = max(mm, wmax[q]);
        atomicMax(maxinc, mm);
    }
}

// Neighbour slot maps: one merge of sorted slot lists per (cell, A slot),
// done once per basis pattern.
__global__ void k_basis_maps(int n, int W, int B, const int *__restrict__ col, const int *__restrict__ pid,
                             unsigned *__restrict__ nmap, unsigned char *__restrict__ nslots) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int ids[8];
    int cnt = 0;
#pragma unroll
    for (int s = 0; s < 8; ++s) {
        ids[s] = s < B ? pid[(int64_t)s * n + i] : kSlotPad;
        cnt += ids[s] != kSlotPad;
    }
    nslots[i] = (unsigned char)cnt;
    for (int w = 0; w < W; ++w) {
        const int k = col[(int64_t)w * n + i];
        unsigned m = 0xffffffffu;
        if (k != i) {
            int t = 0;
            int kid = pid[k];
#pragma unroll
            for (int s = 0; s < 8; ++s) {
                if (ids[s] != kSlotPad) {
                    while (kid < ids[s]) {
                        ++t;
                        kid = t < B ? pid[(int64_t)t * n + k] : kSlotPad;
                    }
                    if (kid == ids[s]) m = (m & ~(15u << (4 * s))) | ((unsigned)t << (4 * s));
                }
            }
        }
        nmap[(int64_t)w * n + i] = m;
    }
}

// The smoothing's cell order: window w of kOrderWin cells (one CTA of 1024
// threads, 4 consecutive cells each) lists its cells by descending slot
// count, keeping the cell order within a count (a counting sort: one
// block-wide exclusive scan per count).
__global__ void __launch_bounds__(1024) k_slot_order(int n, const unsigned char *__restrict__ nslots,
                                                     int *__restrict__ order) {
    __shared__ int wsum[32];
    __shared__ int base;
    const int w0 = blockIdx.x * kOrderWin;
    const int c0 = w0 + 4 * threadIdx.x;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int cc[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) cc[e] = c0 + e < n ? (int)nslots[c0 + e] : -1;
    if (threadIdx.x == 0) base = 0;
    __syncthreads();
    for (int c = 8; c >= 0; --c) {
        int mine = 0;
#pragma unroll
        for (int e = 0; e < 4; ++e) mine += cc[e] == c;
        int inc = mine;   // inclusive warp scan
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, inc, d);
            if (lane >= d) inc += v;
        }
        if (lane == 31) wsum[wid] = inc;
        __syncthreads();
        int before = base;
        for (int q = 0; q < wid; ++q) before += wsum[q];
        int at = before + inc - mine;
#pragma unroll
        for (int e = 0; e < 4; ++e)
            if (cc[e] == c) order[w0 + at++] = c0 + e;
        __syncthreads();   // every thread has read base and wsum
        if (threadIdx.x == 0) {
            int tot = 0;
            for (int q = 0; q < 32; ++q) tot += wsum[q];
            base += tot;
        }
        __syncthreads();
    }
}

// MsRSB iteration with precomputed neighbour slot maps (B <= 8): every
// neighbour contribution is an independent load.  The slot loops of a warp
// stop at the largest slot count among its cells (2, 4 or 8): in FP64 a
// multiply-add that only some lanes need still takes the FP64 pipe for all,
// in FP32 the warp issues fewer instructions.  FP64: the rows come prescaled
// by omega / A_ii (diag and off hold 1 - omega-scaled diagonal and the negated
// scaled off-diagonals).
template <typename T, int WM>
__global__ void __launch_bounds__(kThreads, sizeof(T) == 4 ? 6 : 3) k_msrsb_mapped(int n, int W, const int *__restrict__ col,
                                                           const T *__restrict__ off, const T *__restrict__ diag,
                                                           const unsigned *__restrict__ nmap,
                                                           const unsigned char *__restrict__ nslots, T *bufA,
                                                           T *bufB, const T *__restrict__ odiag,
                                                           unsigned long long *ctl, const int *__restrict__ order) {
    if (*(volatile const unsigned long long *)ctl) return;   // smoothing finished: no-op
    const bool odd = ctl[1] & 1ull;                            // iterations done so far
    const T *__restrict__ pin = odd ? bufB : bufA;
    T *__restrict__ pout = odd ? bufA : bufB;
    unsigned long long *maxinc = ctl + 2;
    const int tix = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = order != nullptr && tix < n ? order[tix] : tix;   // the cell this thread updates
    const int cnt = i < n ? (int)nslots[i] : 0;
    unsigned long long inck = 0ull;   // key of the largest |increment|
    constexpr bool PRE = sizeof(T) == 8;   // FP64: prescaled rows (one multiply-add less per entry)
    const int cmax = __reduce_max_sync(0xffffffffu, cnt);
    if (i < n) {
        if (cmax <= 2) inck = msrsb_cell<T, WM, 2, PRE>(i, cnt, n, W, col, off, diag, nmap, pin, pout, odiag);
        else if (cmax <= 4) inck = msrsb_cell<T, WM, 4, PRE>(i, cnt, n, W, col, off, diag, nmap, pin, pout, odiag);
        else inck = msrsb_cell<T, WM, 8, PRE>(i, cnt, n, W, col, off, diag, nmap, pin, pout, odiag);
    }
    __shared__ unsigned long long wmax[kThreads / 32];
    unsigned long long m = abs_key(key_value<T>(inck));   // key of the value as a double
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_down_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long mm = 0ull;
        for (int q = 0; q < kThreads / 32; ++q) mm = max(mm, wmax[q]);
        atomicMax(maxinc, mm);
    }
}

// After each smoothing iteration: count it, keep its largest increment
// (ctl[3]) and stop once that is below tol, not a number, or the cap is
// reached.  ctl = {stopped, iterations, running max key, last max key}.
__global__ void k_smooth_control(unsigned long long *ctl, double tol, int max_iter) {
    if (ctl[0]) return;
    const unsigned long long it = ++ctl[1];
    const unsigned long long key = ctl[2];
    ctl[3] = key;
    ctl[2] = 0ull;
    const double inc = __longlong_as_double((long long)key);
    if (inc < tol || inc != inc || it >= (unsigned long long)max_iter) ctl[0] = 1ull;   // converged, NaN or capped
}

template <typename T>
__global__ void k_omega_over_diag(int n, const T *__restrict__ diag, T omega, T *__restrict__ od) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) od[i] = omega / diag[i];
}

// Rows of the Jacobi update P - (omega / A_ii) A P prescaled per smoothing run:
// c_i = 1 - (omega / A_ii) A_ii and b_ij = -(omega / A_ii) A_ij (slot layout of A).
__global__ void k_prescale_rows(int n, int W, const double *__restrict__ off, const double *__restrict__ diag,
                                double omega, double *__restrict__ c, double *__restrict__ bw) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double od = omega / diag[i];
    c[i] = 1.0 - od * diag[i];
    for (int w = 0; w < W; ++w) bw[(int64_t)w * n + i] = -(od * off[(int64_t)w * n + i]);
}

template <typename T>
__global__ void k_gather_columns(int64_t nnz, const int *__restrict__ csrc, const T *__restrict__ pval,
                                 T *__restrict__ cval) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (; e < nnz; e += (int64_t)gridDim.x * blockDim.x) cval[e] = pval[csrc[e]];
}

__global__ void k_widen(int64_t nnz, const float *a, double *b) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (; e < nnz; e += (int64_t)gridDim.x * blockDim.x) b[e] = (double)a[e];
}

// ---------------------------------------------------------------- (A P)
// Merge of the sorted slot lists of cell i (weight diag) and of its
// neighbours (weights off).  COUNT only counts distinct blocks; otherwise
// the union ids and values (A P)_il are written, padded to WAP.
constexpr int kMaxNbr = 32;

template <bool COUNT>
__global__ void __launch_bounds__(128) k_ap(int n, int W, int B, const int *__restrict__ col,
                                            const double *__restrict__ off, const double *__restrict__ diag,
                                            const int *__restrict__ pid, const double *__restrict__ pval, int WAP,
                                            int *__restrict__ apid, double *__restrict__ apval, int *cnt_max) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    int count = 0;
    if (i < n) {
        int src[kMaxNbr + 1];
        double wgt[kMaxNbr + 1];
        int pos[kMaxNbr + 1];
        int head[kMaxNbr + 1];
        int L = 0;
        src[L] = i; wgt[L] = diag[i]; pos[L] = 0; head[L] = pid[i]; ++L;
        for (int w = 0; w < W && L <= kMaxNbr; ++w) {
            const int k = col[(int64_t)w * n + i];
            if (k == i) continue;
            src[L] = k; wgt[L] = off[(int64_t)w * n + i]; pos[L] = 0; head[L] = pid[k]; ++L;
        }
        while (true) {
            int l = kSlotPad;
            for (int q = 0; q < L; ++q) l = min(l, head[q]);
            if (l == kSlotPad) break;
            double val = 0.0;
            for (int q = 0; q < L; ++q) {
                if (head[q] == l) {
                    if (!COUNT) val += wgt[q] * pval[(int64_t)pos[q] * n + src[q]];
                    ++pos[q];
                    head[q] = pos[q] < B ? pid[(int64_t)pos[q] * n + src[q]] : kSlotPad;
                }
            }
            if (!COUNT) {
                apid[(int64_t)count * n + i] = l;
                apval[(int64_t)count * n + i] = val;
            }
            ++count;
        }
        if (!COUNT)
            for (int c = count; c < WAP; ++c) {
                apid[(int64_t)c * n + i] = kSlotPad;
                apval[(int64_t)c * n + i] = 0.0;
            }
    }
    if (COUNT) {
        __shared__ int m;
        if (threadIdx.x == 0) m = 0;
        __syncthreads();
        atomicMax(&m, count);
        __syncthreads();
        if (threadIdx.x == 0) atomicMax(cnt_max, m);
    }
}

// Row j of A_c: warp-per-block accumulation over row j of R.
// A_c(j, :) = sum over row j of R of R_ji (A P)(i, :) (R = P^T: the support
// of block j with weights P_ij; finite volume: block j's cells, unit
// weights when cval is null), one warp
// per column chunk with a dense shared-memory row accumulator (lanes take the
// distinct entries of an (A P) row, cells in support order).  A column cut
// into several chunks writes each chunk's row to its partial slot; the last
// chunk to finish adds the partial rows in chunk order (deterministic).
__global__ void k_rap(int n, int M, int WAP, int nch, int C, const int *__restrict__ ch_beg,
                      const int *__restrict__ ch_col, const int *__restrict__ ch_ptr, const int *__restrict__ ch_slot,
                      const int *__restrict__ cptr, const int *__restrict__ ccell, const double *__restrict__ cval,
                      const int *__restrict__ apid, const double *__restrict__ apval, double *part, unsigned *cnt,
                      double *__restrict__ Ac) {
    extern __shared__ double acc_all[];
    const int warps = blockDim.x >> 5;
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int c = blockIdx.x * warps + wid;
    double *acc = acc_all + (size_t)wid * M;
    if (c >= nch) return;
    for (int l = lane; l < M; l += 32) acc[l] = 0.0;
    __syncwarp();
    const int j = ch_col[c];
    const int e0 = ch_beg[c], e1 = min(e0 + C, cptr[j + 1]);
    for (int e = e0; e < e1; ++e) {
        const int i = ccell[e];
        const double p = cval ? cval[e] : 1.0;
        for (int w = lane; w < WAP; w += 32) {
            const int l = apid[(int64_t)w * n + i];
            if (l != kSlotPad) acc[l] += p * apval[(int64_t)w * n + i];
        }
        __syncwarp();
    }
    const int q0 = ch_ptr[j], k = ch_ptr[j + 1] - q0;
    if (k == 1) {
        for (int l = lane; l < M; l += 32) Ac[(int64_t)j * M + l] = acc[l];
        return;
    }
    double *pp = part + (int64_t)ch_slot[c] * M;
    for (int l = lane; l < M; l += 32) pp[l] = acc[l];
    __threadfence();
    __syncwarp();
    unsigned t = 0;
    if (lane == 0) t = atomicAdd(&cnt[j], 1u);
    t = __shfl_sync(0xffffffffu, t, 0);
    if (t != (unsigned)(k - 1)) return;
    __threadfence();
    for (int l = lane; l < M; l += 32) {
        double v = 0.0;
#pragma unroll 4
        for (int q = q0; q < q0 + k; ++q) v += __ldcg(part + (int64_t)ch_slot[q] * M + l);
        Ac[(int64_t)j * M + l] = v;
    }
    if (lane == 0) cnt[j] = 0u;
}

__global__ void k_symmetrise(int M, double *Ac) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)M * M) return;
    const int r = (int)(e / M), c = (int)(e % M);
    if (c <= r) return;
    const double a = Ac[(int64_t)r * M + c], b = Ac[(int64_t)c * M + r];
    const double m = 0.5 * (a + b);
    Ac[(int64_t)r * M + c] = m;
    Ac[(int64_t)c * M + r] = m;
}

}  // namespace

void launch_basis_maps(const ms_system &s, ms_basis &b, cudaStream_t st) {
    b.has_map = false;
    if (b.B > 8 || s.W == 0) return;
    b.nmap.alloc((size_t)s.W * s.n);
    b.nslots.alloc(s.n);
    k_basis_maps<<<blocks_for(s.n), kThreads, 0, st>>>(s.n, s.W, b.B, s.col.p, b.pid.p, b.nmap.p, b.nslots.p);
    MS_CHECK_LAUNCH();
    b.order.alloc(s.n);
    k_slot_order<<<(s.n + kOrderWin - 1) / kOrderWin, 1024, 0, st>>>(s.n, b.nslots.p, b.order.p);
    MS_CHECK_LAUNCH();
    b.has_map = true;
}

void launch_basis_init(ms_basis &b, int n, cudaStream_t st) {
    const int64_t total = (int64_t)b.B * n;
    const int blocks = (int)std::min<int64_t>((total + kThreads - 1) / kThreads, 8192);
    KernelScope ks_(st, "basis_init", (double)total * (1 + (b.precision == MS_PREC_MIXED ? 4 : 8)));
    if (b.precision == MS_PREC_MIXED) k_basis_init32<<<blocks, kThreads, 0, st>>>(total, b.is_home.p, b.pval32.p);
    else k_basis_init<<<blocks, kThreads, 0, st>>>(total, b.is_home.p, b.pval.p);
    MS_CHECK_LAUNCH();
}

template <typename T>
static void msrsb_dispatch(const ms_system &s, const ms_basis &b, const int *pid, const T *off, const T *diag,
                           T *pin, T *pout, const T *omega, unsigned long long *maxinc, cudaStream_t st) {
    const int g = blocks_for(s.n);
    const int B = b.B;
    if (b.has_map) {
        // A (unpinned), omega / A_ii and the maps once, old slot values read once, new written
        KernelScope ks_(st, sizeof(T) == 8 ? "msrsb" : "msrsb32",
                        (double)s.n * (2 * sizeof(T) + 1) + (double)s.W * s.n * (4 + sizeof(T) + 4) +
                            (double)b.nnz * 2 * sizeof(T));
        // maxinc: the control block.  FP64 takes the prescaled rows.
        const int *order = nullptr;   // FP64: cells by slot count within windows
        if constexpr (sizeof(T) == 8) {
            off = b.pre_w64.p;
            diag = b.pre_c64.p;
            const char *e = std::getenv("MSGB_SMOOTH_ORDER");   // "0": natural cell order
            if (!(e && e[0] == '0')) order = b.order.p;
        }
        if (s.W <= 4)
            k_msrsb_mapped<T, 4><<<g, kThreads, 0, st>>>(s.n, s.W, s.col.p, off, diag, b.nmap.p, b.nslots.p, pin,
                                                         pout, omega, maxinc, order);
        else if (s.W <= 6)
            k_msrsb_mapped<T, 6><<<g, kThreads, 0, st>>>(s.n, s.W, s.col.p, off, diag, b.nmap.p, b.nslots.p, pin,
                                                         pout, omega, maxinc, order);
        else if (s.W <= 8)
            k_msrsb_mapped<T, 8><<<g, kThreads, 0, st>>>(s.n, s.W, s.col.p, off, diag, b.nmap.p, b.nslots.p, pin,
                                                         pout, omega, maxinc, order);
        else
            k_msrsb_mapped<T, 0><<<g, kThreads, 0, st>>>(s.n, s.W, s.col.p, off, diag, b.nmap.p, b.nslots.p, pin,
                                                         pout, omega, maxinc, order);
        MS_CHECK_LAUNCH();
        return;
    }
    // A (unpinned) and omega / A_ii once, slot ids and old values once, new values written
    KernelScope ks_(st, sizeof(T) == 8 ? "msrsb" : "msrsb32",
                    (double)s.n * 2 * sizeof(T) + (double)s.W * s.n * (4 + sizeof(T)) +
                        (double)B * s.n * (4 + 2 * sizeof(T)));
    if (B <= 4) k_msrsb<T, 4><<<g, kThreads, 0, st>>>(s.n, s.W, B, s.col.p, off, diag, pid, pin, pout, omega, maxinc);
    else if (B <= 8) k_msrsb<T, 8><<<g, kThreads, 0, st>>>(s.n, s.W, B, s.col.p, off, diag, pid, pin, pout, omega, maxinc);
    else if (B <= 16) k_msrsb<T, 16><<<g, kThreads, 0, st>>>(s.n, s.W, B, s.col.p, off, diag, pid, pin, pout, omega, maxinc);
    else if (B <= 32) k_msrsb<T, 32><<<g, kThreads, 0, st>>>(s.n, s.W, B, s.col.p, off, diag, pid, pin, pout, omega, maxinc);
    else throw Error{MS_ERR_INVALID_ARG, "basis overlap above 32 per cell is not supported"};
    MS_CHECK_LAUNCH();
}

// omega / A_ii of the unpinned A for one smoothing run (A fixed during it).
void launch_basis_scale(const ms_system &s, ms_basis &b, bool fp32, cudaStream_t st) {
    const int g = blocks_for(s.n);
    KernelScope ks_(st, "basis_scale", (double)s.n * (fp32 ? 8 : 16));
    if (fp32) {
        b.od32.alloc(s.n);
        k_omega_over_diag<float><<<g, kThreads, 0, st>>>(s.n, s.diag32.p, (float)b.omega, b.od32.p);
    } else {
        b.od64.alloc(s.n);
        k_omega_over_diag<double><<<g, kThreads, 0, st>>>(s.n, s.diag.p, b.omega, b.od64.p);
        b.pre_c64.alloc(s.n);
        b.pre_w64.alloc(std::max<size_t>((size_t)s.W * s.n, 1));
        k_prescale_rows<<<g, kThreads, 0, st>>>(s.n, s.W, s.off_u.p, s.diag.p, b.omega, b.pre_c64.p, b.pre_w64.p);
    }
    MS_CHECK_LAUNCH();
}

// One iteration under the device control block ctl (k_smooth_control after
// it): reads pval / pval_tmp by the parity of the iterations done, and does
// nothing once the smoothing has stopped.  The caller swaps the buffers when
// an odd number of iterations ran.
void launch_msrsb_iter(const ms_system &s, ms_basis &b, bool fp32, unsigned long long *ctl, double tol, int max_iter,
                       cudaStream_t st) {
    if (fp32) msrsb_dispatch<float>(s, b, b.pid.p, s.off_u32.p, s.diag32.p, b.pval32.p, b.pval32_tmp.p, b.od32.p, ctl, st);
    else msrsb_dispatch<double>(s, b, b.pid.p, s.off_u.p, s.diag.p, b.pval.p, b.pval_tmp.p, b.od64.p, ctl, st);
    k_smooth_control<<<1, 1, 0, st>>>(ctl, tol, max_iter);
    MS_CHECK_LAUNCH();
}

// Column view values from the cell-major slots (and an FP64 copy of FP32
// bases, used by the Galerkin product).
void launch_basis_columns(ms_basis &b, cudaStream_t st) {
    const int blocks = (int)std::min<int64_t>((b.nnz + kThreads - 1) / kThreads, 8192);
    if (b.nnz == 0) return;
    KernelScope ks_(st, "basis_columns", (double)b.nnz * 16);
    if (b.precision == MS_PREC_MIXED) {
        k_gather_columns<float><<<blocks, kThreads, 0, st>>>(b.nnz, b.csrc.p, b.pval32.p, b.cval32.p);
        k_widen<<<blocks, kThreads, 0, st>>>(b.nnz, b.cval32.p, b.cval.p);
        const int64_t tot = (int64_t)b.B * (int64_t)(b.pval.n / std::max(b.B, 1));   // FP64 slot copy for the Galerkin product
        const int bb = (int)std::min<int64_t>((tot + kThreads - 1) / kThreads, 8192);
        if (tot) k_widen<<<bb, kThreads, 0, st>>>(tot, b.pval32.p, b.pval.p);
    } else {
        k_gather_columns<double><<<blocks, kThreads, 0, st>>>(b.nnz, b.csrc.p, b.pval.p, b.cval.p);
    }
    MS_CHECK_LAUNCH();
}

int launch_ap_count(const ms_system &s, const ms_basis &b, int *cnt_max, int *host_pinned, cudaStream_t st) {
    MS_REQUIRE(s.W <= kMaxNbr, MS_ERR_INVALID_ARG, "too many connections per cell for the Galerkin kernel");
    MS_CUDA(cudaMemsetAsync(cnt_max, 0, sizeof(int), st));
    KernelScope ks_(st, "ap_count", 0.0);
    k_ap<true><<<blocks_for(s.n, 128), 128, 0, st>>>(s.n, s.W, b.B, s.col.p, s.off_p.p, s.diag.p, b.pid.p, b.pval.p,
                                                      0, nullptr, nullptr, cnt_max);
    MS_CHECK_LAUNCH();
    MS_CUDA(cudaMemcpyAsync(host_pinned, cnt_max, sizeof(int), cudaMemcpyDeviceToHost, st));
    MS_CUDA(cudaStreamSynchronize(st));
    return *host_pinned;
}

void launch_ap_fill(const ms_system &s, const ms_basis &b, ms_coarse &c, cudaStream_t st) {
    KernelScope ks_(st, "ap_fill", 0.0);
    k_ap<false><<<blocks_for(s.n, 128), 128, 0, st>>>(s.n, s.W, b.B, s.col.p, s.off_p.p, s.diag.p, b.pid.p,
                                                       b.pval.p, c.WAP, c.apid.p, c.apval.p, nullptr);
    MS_CHECK_LAUNCH();
}

void launch_rap(const ms_system &s, const std::vector<int> &h_cptr, const int *cptr, const int *ccell,
                const double *cval, bool symmetrise, ms_coarse &c, cudaStream_t st) {
    const int M = c.M;
    const size_t per_warp = (size_t)M * sizeof(double);
    MS_REQUIRE(per_warp <= 200 * 1024, MS_ERR_INVALID_ARG, "coarse system too large for the Galerkin kernel");
    if (c.gchunk == 0) {
        // chunk size: the partial rows of split columns stay within 256 MB
        std::vector<int> cb, cc, cp, sl;
        int multi = 0;
        int C = kColChunk;
        for (;; C *= 2) {
            build_column_chunks(h_cptr, M, C, cb, cc, cp, &sl, &multi);
            if ((double)multi * M * 8.0 <= 256.0 * 1024 * 1024 || C >= (1 << 30) / 2) break;
        }
        c.gchunk = C;
        c.n_gchunks = (int)cb.size();
        c.gch_beg.upload(cb, st);
        c.gch_col.upload(cc, st);
        c.gch_ptr.upload(cp, st);
        c.gch_slot.upload(sl, st);
        c.gpart.alloc(std::max<size_t>((size_t)multi * M, 1));
        c.gcnt.alloc(std::max(M, 1));
        c.gcnt.zero(st);
    }
    int warps = (int)std::max<size_t>(1, std::min<size_t>(8, (200 * 1024) / per_warp));
    size_t smem = per_warp * warps;
    static size_t smem_set = 48 * 1024;
    MS_CUDA(raise_smem_limit(k_rap, smem, smem_set));
    KernelScope ks_(st, "rap", 0.0);
    k_rap<<<(c.n_gchunks + warps - 1) / warps, 32 * warps, smem, st>>>(
        s.n, M, c.WAP, c.n_gchunks, c.gchunk, c.gch_beg.p, c.gch_col.p, c.gch_ptr.p, c.gch_slot.p, cptr, ccell,
        cval, c.apid.p, c.apval.p, c.gpart.p, c.gcnt.p, c.Ac.p);
    MS_CHECK_LAUNCH();
    if (symmetrise) {
        const int64_t MM = (int64_t)M * M;
        k_symmetrise<<<(int)((MM + kThreads - 1) / kThreads), kThreads, 0, st>>>(M, c.Ac.p);
        MS_CHECK_LAUNCH();
    }
}

}  // namespace msgb
