// Batched MsRSB basis smoothing (Sec. 5.1) for many independent systems in
// one persistent launch.
//
// Work items are (member, tile) pairs: one iteration of one member's
// smoothing over `tile` consecutive cells.  A member's iteration k + 1 may
// start only when all tiles of its iteration k are done, and only if
// iteration k did not stop it.  So the queue is filled as the work goes: the
// block that finishes the last tile of a member's iteration runs the member's
// iteration control (the same as the per-system path: count, keep the largest
// increment, stop below tol, on NaN or at the cap) and, if the member goes on,
// appends the tiles of its next iteration.  Blocks take items in ticket order
// from a ring of 64-bit slots [position + 1 : 31 | consumed : 1 | item : 32];
// an item never waits for another item, so the launch needs no co-residency
// and cannot deadlock; a block whose ticket has no item yet waits for one
// (or for every member to stop).  Slots are reused only after their previous
// item was consumed.  Every wait is bounded (2 s) and records an error.
//
// The cell update is msrsb_cell, the one the per-system kernel runs.  The slot
// values another block wrote in this launch are read with weak L1-cached
// loads after the acquire of the item's slot (thread 0, then the block
// barrier), which the memory model orders after the writes the finishing
// block released.
// Results are bitwise those of smoothing each member alone.
#include <algorithm>
#include <cstring>

#include "ms_internal.h"
#include "msrsb_cell.cuh"

namespace msgb {

namespace {

constexpr int kBT = 256;                       // threads per block (cells per pass of a tile)
constexpr unsigned long long kConsumed = 1ull << 32;
constexpr unsigned long long kBatchWaitNs = 2000000000ull;
// slot values: weak loads cached in L1 after the item's acquire (ldp policy 2)
constexpr int kLd = 2;

template <typename T>
struct SmJob {
    const int *col;
    const T *off;
    const T *diag;
    const unsigned *nmap;
    const unsigned char *nslots;
    T *bufA;
    T *bufB;
    const T *odiag;
    unsigned long long *ctl;   // {stopped, iterations, running max key, last max key}
    double tol;
    int n, W, ntiles, max_iter;
};

struct BatchQueue {
    unsigned long long head, tail;   // next ticket, next free position
    int active;                      // members still smoothing
    int err;                         // 1: a wait ran out
};

__device__ __forceinline__ unsigned long long bq_now() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned long long ld_acq64(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_rel64(unsigned long long *p, unsigned long long v) {
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ int ld_vol32(const int *p) { return *(volatile const int *)p; }

// Append the tiles of member m's next iteration (the whole block).
__device__ void bq_push(BatchQueue *q, unsigned long long *slots, unsigned long long mask, int m, int ntiles,
                        unsigned long long base) {
    const unsigned long long R = mask + 1;
    for (int j = threadIdx.x; j < ntiles; j += blockDim.x) {
        const unsigned long long p = base + (unsigned long long)j;
        unsigned long long *slot = &slots[p & mask];
        // the slot's previous occupant (position p - R) must have been consumed
        unsigned long long t0 = 0;
        for (int spins = 0;; ++spins) {
            const unsigned long long v = ld_acq64(slot);
            if (v == 0ull || (p >= R && (v >> 33) == p - R + 1 && (v & kConsumed))) break;
            if (ld_vol32(&q->err)) return;
            if ((spins & 31) == 31) {
                const unsigned long long now = bq_now();
                if (t0 == 0) t0 = now;
                else if (now - t0 > kBatchWaitNs) { atomicExch(&q->err, 1); return; }
            }
        }
        st_rel64(slot, ((p + 1) << 33) | ((unsigned long long)m << 20) | (unsigned long long)j);
    }
}

template <typename T>
__global__ void __launch_bounds__(kBT, sizeof(T) == 4 ? 6 : 3) k_msrsb_batch(const SmJob<T> *__restrict__ jobs, int tile, BatchQueue *q,
                                                     unsigned long long *slots, unsigned long long mask,
                                                     int *done) {
    __shared__ unsigned s_item;
    __shared__ int s_state;                      // 0 exit, 1 item
    __shared__ int s_push;                       // member to enqueue, or -1
    __shared__ unsigned long long s_base;
    __shared__ unsigned long long wmax[kBT / 32];
    const int tid = threadIdx.x;
    for (;;) {
        if (tid == 0) {
            const unsigned long long t = atomicAdd(&q->head, 1ull);
            unsigned long long *slot = &slots[t & mask];
            int state = 0;
            unsigned long long t0 = 0;
            for (int spins = 0;; ++spins) {
                const unsigned long long v = ld_acq64(slot);
                if ((v >> 33) == t + 1 && !(v & kConsumed)) {
                    s_item = (unsigned)v;
                    st_rel64(slot, v | kConsumed);
                    state = 1;
                    break;
                }
                if (ld_vol32(&q->active) == 0 || ld_vol32(&q->err)) break;
                if (spins > 8) __nanosleep(64);
                if ((spins & 31) == 31) {
                    const unsigned long long now = bq_now();
                    if (t0 == 0) t0 = now;
                    else if (now - t0 > kBatchWaitNs) { atomicExch(&q->err, 1); break; }
                }
            }
            s_state = state;
            s_push = -1;
        }
        __syncthreads();
        if (!s_state) break;
        const int m = (int)(s_item >> 20), tl = (int)(s_item & 0xFFFFFu);
        const SmJob<T> J = jobs[m];
        const bool odd = __ldcg(&J.ctl[1]) & 1ull;           // iterations done so far
        const T *pin = odd ? J.bufB : J.bufA;
        T *pout = odd ? J.bufA : J.bufB;
        const int i0 = tl * tile, i1 = min(J.n, i0 + tile);
        unsigned long long inck = 0ull;
        for (int b0 = i0; b0 < i1; b0 += kBT) {
            const int i = b0 + tid;
            const int cnt = i < i1 ? (int)J.nslots[i] : 0;
            // slot loops bounded by the warp's largest slot count; FP64 rows prescaled
            constexpr bool PRE = sizeof(T) == 8;
            const int cmax = __reduce_max_sync(0xffffffffu, cnt);
            if (i < i1) {
                unsigned long long k;
                if (cmax <= 2) k = msrsb_cell<T, 8, 2, PRE, kLd>(i, cnt, J.n, J.W, J.col, J.off, J.diag, J.nmap, pin, pout, J.odiag);
                else if (cmax <= 4) k = msrsb_cell<T, 8, 4, PRE, kLd>(i, cnt, J.n, J.W, J.col, J.off, J.diag, J.nmap, pin, pout, J.odiag);
                else k = msrsb_cell<T, 8, 8, PRE, kLd>(i, cnt, J.n, J.W, J.col, J.off, J.diag, J.nmap, pin, pout, J.odiag);
                inck = max(inck, k);
            }
        }
        unsigned long long km = abs_key(key_value<T>(inck));   // key of the value as a double
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) km = max(km, __shfl_down_sync(0xffffffffu, km, o));
        if ((tid & 31) == 0) wmax[tid >> 5] = km;
        __syncthreads();
        if (tid == 0) {
            unsigned long long mm = 0ull;
            for (int w = 0; w < kBT / 32; ++w) mm = max(mm, wmax[w]);
            atomicMax(&J.ctl[2], mm);
            __threadfence();
            if (atomicAdd(&done[m], 1) == J.ntiles - 1) {
                // last tile of this iteration: the iteration control
                __threadfence();
                done[m] = 0;
                const unsigned long long it = __ldcg(&J.ctl[1]) + 1ull;
                const unsigned long long key = atomicExch(&J.ctl[2], 0ull);
                J.ctl[3] = key;
                J.ctl[1] = it;
                const double inc = __longlong_as_double((long long)key);
                if (inc < J.tol || inc != inc || it >= (unsigned long long)J.max_iter) {
                    J.ctl[0] = 1ull;
                    __threadfence();
                    atomicSub(&q->active, 1);
                } else {
                    __threadfence();
                    s_base = atomicAdd(&q->tail, (unsigned long long)J.ntiles);
                    s_push = m;
                }
            }
        }
        __syncthreads();
        if (s_push >= 0) bq_push(q, slots, mask, s_push, jobs[s_push].ntiles, s_base);
        __syncthreads();
    }
}

template <typename T>
SmJob<T> make_job(const ms_system &s, ms_basis &b) {
    SmJob<T> j{};
    j.col = s.col.p;
    if constexpr (sizeof(T) == 8) {   // prescaled rows, as in the per-system path
        j.off = b.pre_w64.p;
        j.diag = b.pre_c64.p;
        j.bufA = b.pval.p;
        j.bufB = b.pval_tmp.p;
        j.odiag = b.od64.p;
    } else {
        j.off = s.off_u32.p;
        j.diag = s.diag32.p;
        j.bufA = b.pval32.p;
        j.bufB = b.pval32_tmp.p;
        j.odiag = b.od32.p;
    }
    j.nmap = b.nmap.p;
    j.nslots = b.nslots.p;
    j.tol = b.tol;
    j.n = s.n;
    j.W = s.W;
    j.max_iter = b.max_iter;
    return j;
}

// One persistent launch for the members `idx` (one precision).
template <typename T>
void run_batch(ms_ctx *ctx, const std::vector<ms_system *> &sys, const std::vector<ms_basis *> &bases,
               const std::vector<int> &idx) {
    cudaStream_t st = ctx->stream;
    const int nj = (int)idx.size();
    const int tile = ctx->batch_tile;
    const bool fp32 = sizeof(T) == 4;
    BatchScratch &B = *ctx->batch;
    std::vector<SmJob<T>> jobs(nj);
    B.ctl.alloc((size_t)4 * nj);
    B.done.alloc(nj);
    MS_CUDA(cudaMemsetAsync(B.ctl.p, 0, (size_t)4 * nj * sizeof(unsigned long long), st));
    MS_CUDA(cudaMemsetAsync(B.done.p, 0, (size_t)nj * sizeof(int), st));
    int64_t first = 0;
    int active = 0;
    for (int q = 0; q < nj; ++q) {
        ms_system &s = *sys[idx[q]];
        ms_basis &b = *bases[idx[q]];
        launch_basis_init(b, s.n, st);
        jobs[q] = make_job<T>(s, b);
        jobs[q].ctl = B.ctl.p + 4 * (size_t)q;
        jobs[q].ntiles = (s.n + tile - 1) / tile;
        if (b.max_iter > 0) {
            launch_basis_scale(s, b, fp32, st);
            jobs[q] = make_job<T>(s, b);   // the prescaled rows may have been (re)allocated
            jobs[q].ctl = B.ctl.p + 4 * (size_t)q;
            jobs[q].ntiles = (s.n + tile - 1) / tile;
            first += jobs[q].ntiles;
            ++active;
        }
    }
    int dev = 0, sms = 0;
    MS_CUDA(cudaGetDevice(&dev));
    MS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int G = std::max(1, sms * std::max(1, ctx->batch_ctas_per_sm));
    unsigned long long R = 1024;
    while (R < (unsigned long long)(2 * first + 2 * G + 1024)) R <<= 1;
    // initial items: the first iteration of every member, largest first
    std::vector<int> order(nj);
    for (int q = 0; q < nj; ++q) order[q] = q;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b2) { return jobs[a].n > jobs[b2].n; });
    std::vector<unsigned long long> init((size_t)first);
    unsigned long long p = 0;
    for (int q : order) {
        if (bases[idx[q]]->max_iter <= 0) continue;
        for (int t = 0; t < jobs[q].ntiles; ++t, ++p)
            init[p] = ((p + 1) << 33) | ((unsigned long long)q << 20) | (unsigned long long)t;
    }
    B.slots.alloc(R);
    MS_CUDA(cudaMemsetAsync(B.slots.p, 0, R * sizeof(unsigned long long), st));
    if (first) MS_CUDA(cudaMemcpyAsync(B.slots.p, init.data(), first * sizeof(unsigned long long), cudaMemcpyHostToDevice, st));
    B.queue.alloc(3);
    const unsigned long long qh[3] = {0ull, (unsigned long long)first, (unsigned long long)(unsigned)active};
    MS_CUDA(cudaMemcpyAsync(B.queue.p, qh, sizeof(qh), cudaMemcpyHostToDevice, st));
    B.jobs.alloc(sizeof(SmJob<T>) * nj);
    MS_CUDA(cudaMemcpyAsync(B.jobs.p, jobs.data(), sizeof(SmJob<T>) * nj, cudaMemcpyHostToDevice, st));
    if (active > 0) {
        int64_t cells = 0, nnz = 0, wn = 0;
        for (int q = 0; q < nj; ++q) {
            cells += jobs[q].n;
            nnz += bases[idx[q]]->nnz;
            wn += (int64_t)jobs[q].W * jobs[q].n;
        }
        // bytes: added once the iteration counts are known (below)
        KernelScope ks_(st, fp32 ? "msrsb_batch32" : "msrsb_batch", 0.0);
        (void)cells;
        (void)nnz;
        (void)wn;
        k_msrsb_batch<T><<<G, kBT, 0, st>>>((const SmJob<T> *)B.jobs.p, tile, (BatchQueue *)B.queue.p, B.slots.p,
                                            R - 1, B.done.p);
        MS_CHECK_LAUNCH();
    }
    // read back the control blocks and the queue's error word
    std::vector<unsigned long long> h((size_t)4 * nj + 3);
    MS_CUDA(cudaMemcpyAsync(h.data(), B.ctl.p, (size_t)4 * nj * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
    MS_CUDA(cudaMemcpyAsync(h.data() + 4 * nj, B.queue.p, 3 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
    MS_CUDA(cudaStreamSynchronize(st));
    const int qerr = (int)(h[4 * (size_t)nj + 2] >> 32);
    if (qerr) throw Error{MS_ERR_TIMEOUT, "a batched basis smoothing wait ran out"};
    {
        // algorithmic bytes of the launch: per member and iteration, as the
        // per-system kernel (rows and slot maps, old slot values read, new written)
        double bytes = 0.0;
        for (int q = 0; q < nj; ++q) {
            if (bases[idx[q]]->max_iter <= 0) continue;
            const double it = (double)h[4 * (size_t)q + 1];
            bytes += it * ((double)jobs[q].n * (2 * sizeof(T) + 1) + (double)jobs[q].W * jobs[q].n * (4 + sizeof(T) + 4) +
                           (double)bases[idx[q]]->nnz * 2 * sizeof(T));
        }
        profile_add_bytes(fp32 ? "msrsb_batch32" : "msrsb_batch", bytes);
    }
    for (int q = 0; q < nj; ++q) {
        ms_system &s = *sys[idx[q]];
        ms_basis &b = *bases[idx[q]];
        int it = 0;
        double inc = 0.0;
        if (b.max_iter > 0) {
            it = (int)h[4 * (size_t)q + 1];
            std::memcpy(&inc, &h[4 * (size_t)q + 3], sizeof(double));
            if (it & 1) {
                if (fp32) std::swap(b.pval32.p, b.pval32_tmp.p);
                else std::swap(b.pval.p, b.pval_tmp.p);
            }
            if (!(inc == inc)) throw Error{MS_ERR_INVALID_ARG, "basis smoothing produced NaN"};
        }
        b.iters = it;
        b.last_inc = inc;
        b.assembly_id = s.assembly_id;
        launch_basis_columns(b, st);
    }
}

}  // namespace

void smooth_batch(ms_ctx *ctx, const std::vector<ms_system *> &sys, const std::vector<ms_basis *> &bases,
                  std::vector<char> &taken) {
    const int n = (int)sys.size();
    taken.assign(n, 0);
    if (!ctx->batch) ctx->batch.reset(new BatchScratch());
    std::vector<int> g64, g32;
    const int tile = ctx->batch_tile;
    for (int m = 0; m < n; ++m) {
        ms_system &s = *sys[m];
        ms_basis &b = *bases[m];
        if (b.rule == MS_SUPPORT_BLOCK || !b.has_map || s.W > 8 || (s.n + tile - 1) / tile >= (1 << 20)) continue;
        (b.precision == MS_PREC_MIXED ? g32 : g64).push_back(m);
    }
    if ((int)g64.size() >= (1 << 12) || (int)g32.size() >= (1 << 12)) return;   // item ids hold 12 bits of member
    if (!g64.empty()) run_batch<double>(ctx, sys, bases, g64);
    if (!g32.empty()) run_batch<float>(ctx, sys, bases, g32);
    for (int m : g64) taken[m] = 1;
    for (int m : g32) taken[m] = 1;
}

}  // namespace msgb
