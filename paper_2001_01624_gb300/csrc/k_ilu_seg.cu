// ILU(0) triangular sweeps on structured grids with each line split into
// segments of 64 cells, one warp per segment.
//
// Natural-order ILU(0) on the 7-point pattern (the smoother of the multistage
// cycle, Sec. 3): the forward sweep is
//     y(x,j,k) = r - Lx y(x-1,j,k) - Ly y(x,j-1,k) - Lz y(x,j,k-1),
// the backward sweep its mirror image with U and the reciprocal diagonal.
// With the neighbouring lines (j-1,k) and (j,k-1) known, a line is the
// first-order recurrence v(x) = A(x) v(x-1) + B(x).  Each k-row of lines is
// walked along j; rows drift into a wavefront, so a sweep costs about
// (lines per row + rows) line steps.  Walking the shorter grid direction
// (y-lines on transposed vectors when nx < ny) shortens that chain, but a
// long line costs one warp many dependent FP64 instructions per step, and on
// this part a warp's FP64 instruction occupies its sub-partition for about 64
// cycles whether one lane or 32 are active.  So a line is cut into segments
// of 64 cells (2 per lane), one warp each, placed on different
// sub-partitions: a segment solves its recurrence from a zero start with a
// shuffle scan, then adds P(x) c, where c is the value leaving the segment
// before it and P(x) the product of the multipliers from the segment's start
// to x (constant for the factor, precomputed with the scan multipliers in
// FP64).  Only that one value travels between the segments of a line.
//
// Hand-overs (a finished line segment to the same segment of the next row,
// a segment's last value to the next segment of its line) are 8-byte tagged
// words in the receiver's shared memory: the payload in the low half (an FP64
// value as two words, one per half) and the line's number in the high half.
// The receiver polls its own words with plain loads until every tag matches,
// and tells the sender how far it has read with a progress word in the
// sender's shared memory, so a ring slot is rewritten only after it was read.
// Rows at the last CTA of a cluster hand their lines to the next cluster
// through a global ring of tagged words (one slot per line, the launch's tag),
// which a relay warp of the receiving cluster polls ahead and forwards.  A
// producer warp streams each row's inputs (coefficients, scan tables and the
// right-hand side, two lines per bulk copy) into a ring of slots guarded by
// mbarriers.  Every wait is bounded in device time and reports a timeout.
#include <algorithm>
#include <atomic>
#include <cstdlib>
#include <string>

#include "ms_internal.h"
#include "line_sync.cuh"

namespace msgb {

namespace {

constexpr int SE = 2;              // cells per lane
constexpr int SLW = 32 * SE;       // cells per segment
constexpr int SRF = 2;             // input slots per row
constexpr int SRL = 4;             // lines per input slot (one barrier wait per 4 line steps)
constexpr int SNX = 8;             // k-exchange ring: lines a row may run ahead of the next
constexpr int SNC = 8;             // carry ring: lines a segment may run ahead of the next
constexpr int SNL = 5;             // scan levels over 32 lanes
constexpr int kMaxSeg = 4;         // lines of up to 256 cells

// scan table of one line: per segment the multipliers of the 5 levels x 32
// lanes, then (more than one segment) the 64 carry multipliers P
__host__ __device__ constexpr int seg_span(int S) { return SNL * 32 + (S > 1 ? SLW : 0); }
__host__ __device__ constexpr int seg_table(int S) { return S * seg_span(S); }

// tagged words: payload in the low 32 bits, tag in the high 32.  The data a
// word guards travels in the word itself, so these accesses need no ordering
// against other memory operations (no memory clobber); being volatile they
// keep their order among themselves.
__device__ __forceinline__ unsigned long long tw_lo(unsigned payload, unsigned tag) {
    return (unsigned long long)payload | ((unsigned long long)tag << 32);
}
__device__ __forceinline__ void tw_put2(unsigned caddr, unsigned long long a, unsigned long long b) {
    asm volatile("st.relaxed.cluster.shared::cluster.v2.u64 [%0], {%1, %2};" ::"r"(caddr), "l"(a), "l"(b));
}
__device__ __forceinline__ void tw_put1(unsigned caddr, unsigned long long a) {
    asm volatile("st.relaxed.cluster.shared::cluster.u64 [%0], %1;" ::"r"(caddr), "l"(a));
}
__device__ __forceinline__ void tw_get2(unsigned saddr, unsigned long long &a, unsigned long long &b) {
    asm volatile("ld.relaxed.cluster.shared::cta.v2.u64 {%0, %1}, [%2];" : "=l"(a), "=l"(b) : "r"(saddr));
}
__device__ __forceinline__ unsigned long long tw_get1(unsigned saddr) {
    unsigned long long a;
    asm volatile("ld.relaxed.cluster.shared::cta.u64 %0, [%1];" : "=l"(a) : "r"(saddr));
    return a;
}
__device__ __forceinline__ void prog_put(unsigned caddr, unsigned v) {
    asm volatile("st.relaxed.cluster.shared::cluster.u32 [%0], %1;" ::"r"(caddr), "r"(v));
}
__device__ __forceinline__ unsigned prog_get(unsigned saddr) {
    unsigned v;
    asm volatile("ld.relaxed.cluster.shared::cta.u32 %0, [%1];" : "=r"(v) : "r"(saddr));
    return v;
}
__device__ __forceinline__ bool tag_is(unsigned long long w, unsigned tag) { return (unsigned)(w >> 32) == tag; }

// one lane's SE values as tagged words (FP64: 2 words per value)
__device__ __forceinline__ void tw_encode(const float (&v)[SE], unsigned tag, unsigned long long (&w)[SE]) {
#pragma unroll
    for (int e = 0; e < SE; ++e) w[e] = tw_lo(__float_as_uint(v[e]), tag);
}
__device__ __forceinline__ void tw_encode(const double (&v)[SE], unsigned tag, unsigned long long (&w)[2 * SE]) {
#pragma unroll
    for (int e = 0; e < SE; ++e) {
        const unsigned long long b = (unsigned long long)__double_as_longlong(v[e]);
        w[2 * e] = tw_lo((unsigned)(b & 0xffffffffull), tag);
        w[2 * e + 1] = tw_lo((unsigned)(b >> 32), tag);
    }
}
__device__ __forceinline__ float tw_decode1(unsigned long long w) { return __uint_as_float((unsigned)w); }
__device__ __forceinline__ double tw_decode2(unsigned long long lo, unsigned long long hi) {
    return __longlong_as_double((long long)((lo & 0xffffffffull) | (hi << 32)));
}

// poll N words at saddr (N = 2 or 4, 16-byte aligned) until all carry `tag`;
// false on timeout (recorded in err)
template <int N>
__device__ __forceinline__ bool tw_wait(unsigned saddr, unsigned tag, unsigned long long (&w)[N], int *err) {
    static_assert(N == 2 || N == 4, "2 or 4 words");
    unsigned long long t0 = 0;
    int spins = 0;
    for (;;) {
        bool ok;
        if constexpr (N == 2) {
            tw_get2(saddr, w[0], w[1]);
            ok = tag_is(w[0], tag) && tag_is(w[1], tag);
        } else {
            tw_get2(saddr, w[0], w[1]);
            tw_get2(saddr + 16, w[2], w[3]);
            ok = tag_is(w[0], tag) && tag_is(w[1], tag) && tag_is(w[2], tag) && tag_is(w[3], tag);
        }
        if (ok) return true;
        if ((++spins & 63) == 0) {
            const unsigned long long now = global_ns();
            if (t0 == 0) t0 = now;
            else if (now - t0 > wait_limit_ns(err)) {
                atomicOr(err, kErrTimeout);
                return false;
            }
        }
    }
}

// wait until the progress word at saddr reaches `need`; `seen` keeps the
// last value read, so the word is read only when that is not enough
__device__ __forceinline__ bool prog_wait(unsigned saddr, unsigned need, unsigned &seen, int *err) {
    if (seen >= need) return true;
    unsigned long long t0 = 0;
    int spins = 0;
    while ((seen = prog_get(saddr)) < need) {
        if ((++spins & 63) == 0) {
            const unsigned long long now = global_ns();
            if (t0 == 0) t0 = now;
            else if (now - t0 > wait_limit_ns(err)) {
                atomicOr(err, kErrTimeout);
                return false;
            }
        }
    }
    return true;
}

// shared-memory layout of the segmented sweep (bytes), for a layout of
// lines of Lx cells in S segments, TK rows per CTA
struct SegSmem {
    size_t coef, tab, rhs, xin, cin, pv, prog, bars, total;
};
// PP warps per segment take the lines in turn (PP = 2: one warp's bookkeeping
// overlaps the other's dependency chain)
template <typename T, typename TR>
__host__ __device__ SegSmem seg_smem(int Lx, int S, int TK, int PP) {
    constexpr int RW = sizeof(T) == 8 ? 2 : 1;
    SegSmem m{};
    size_t off = 0;
    m.coef = off;
    off += (size_t)SRF * TK * SRL * Lx * 4 * sizeof(T);
    m.tab = off;
    off += sizeof(T) == 8 ? (size_t)SRF * TK * SRL * seg_table(S) * sizeof(T) : 0;
    m.rhs = off;
    off += (size_t)SRF * TK * rhs_win(SRL * Lx, sizeof(TR)) * sizeof(TR);
    m.xin = off;                                   // [TK][S][SNX] lines from the previous row
    off += (size_t)TK * S * SNX * SLW * RW * 8;
    m.cin = off;                                   // [TK][S][PP][SNC] carries, padded to 16 bytes
    off += (size_t)TK * S * PP * SNC * 2 * 8;
    m.pv = off;                                    // [TK][S][PP][2] the previous line, from the other warp
    off += PP > 1 ? (size_t)TK * S * PP * 2 * SLW * RW * 8 : 0;
    m.prog = off;                                  // progress: xprog [TK S PP] | cprog [TK S PP] | rprog [S PP]
    off += ((size_t)(2 * TK * S + S) * PP * 4 + 15) / 16 * 16;
    m.bars = off;
    off += (size_t)2 * SRF * TK * 8;
    m.total = off;
    return m;
}

}  // namespace

namespace {

// Warps: PP x TK rows x S segments compute (warp (p TK + r) S + s: phase p,
// row r, segment s, so the segments of a row, and the two phases of one
// segment, sit on different sub-partitions' turns), then the producer, then
// (rows spanning several clusters) one relay warp per segment.  Phase p takes
// the lines tj = p, p + PP, ... of its row and segment.  The rows may span NC
// clusters of gridDim.x / NC CTAs; each cluster takes a ticket when it
// starts, and the ticket decides its block of rows, so a cluster only waits
// for one that started before it.
constexpr int kSegMaxWarps = 14;   // compute warps + producer + relays

template <typename T, typename TR, bool BWD, int PP>
__global__ void __launch_bounds__(32 * kSegMaxWarps, 1)
    k_line_seg(int Lx, int Ny, int Nz, int S, int TK, int NC, const T *__restrict__ coef4, const T *__restrict__ scanm,
               const TR *__restrict__ rhs, T *__restrict__ out, unsigned long long *tick, unsigned long long *ring,
               int *err) {
    constexpr int RW = sizeof(T) == 8 ? 2 : 1;   // tagged words per value
    constexpr int NW = SE * RW;                  // tagged words of one lane's values
    constexpr bool TAB = sizeof(T) == 8;         // FP64: scan and carry multipliers from the table
    constexpr unsigned FULL = 0xffffffffu;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const unsigned K = cluster_rank();
    const SegSmem lay = seg_smem<T, TR>(Lx, S, TK, PP);
    extern __shared__ __align__(16) unsigned char smraw[];
    T *cwin = reinterpret_cast<T *>(smraw + lay.coef);
    T *twin = reinterpret_cast<T *>(smraw + lay.tab);
    TR *rwin = reinterpret_cast<TR *>(smraw + lay.rhs);
    unsigned long long *xin = reinterpret_cast<unsigned long long *>(smraw + lay.xin);
    unsigned long long *cin = reinterpret_cast<unsigned long long *>(smraw + lay.cin);
    unsigned long long *pvin = reinterpret_cast<unsigned long long *>(smraw + lay.pv);
    unsigned *prog = reinterpret_cast<unsigned *>(smraw + lay.prog);   // xprog [TK S PP] | cprog | rprog [S PP]
    const int NCW = TK * S * PP;   // compute warps
    const unsigned full_f = smem_u32(smraw + lay.bars);
    const unsigned empty_f = full_f + 8 * SRF * TK;
    const int CLN = Lx * 4;
    const int TBW = seg_table(S);
    const int WR = rhs_win(SRL * Lx, sizeof(TR));

    // every hand-over word starts with a tag no line carries, every progress
    // word at zero; the cluster barrier below publishes them
    for (size_t i = tid; i < (lay.prog - lay.xin) / 8; i += blockDim.x) xin[i] = ~0ull;
    for (int i = tid; i < (2 * TK * S + S) * PP; i += blockDim.x) prog[i] = 0u;
    if (tid < TK) {
        for (int q = 0; q < SRF; ++q) {
            mb_init(full_f + 8 * (q * TK + tid), 1);
            mb_init(empty_f + 8 * (q * TK + tid), (unsigned)(S * PP));   // each compute warp of the row frees it
        }
    }
    __shared__ unsigned long long s_tick;
    if (NC > 1 && K == 0 && tid == 0) s_tick = atomicAdd(tick, 1ull);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    cluster_sync_all();
    unsigned long long tk = 0;
    if (NC > 1) {
        const unsigned a = map_cta(smem_u32(&s_tick), 0);
        asm volatile("ld.shared::cluster.u64 %0, [%1];" : "=l"(tk) : "r"(a) : "memory");
    }
    const int NKC = (int)gridDim.x / NC;                 // CTAs per cluster
    const int v = (int)(tk % (unsigned long long)NC);    // this cluster's block of rows
    const unsigned ltag = (unsigned)(tk / (unsigned long long)NC) + 1u;   // the launch's tag in the global ring
    const int KG = v * NKC + (int)K;                     // CTA position in the row order
    const long long plane = (long long)Lx * Ny;
    const int nblk = (Ny + SRL - 1) / SRL;
    const int SW = S * SLW;                              // values of one line in the global ring

    if (w == NCW) {
        // producer warp: lane r streams the input blocks of row r (SRL lines each)
        const int g = KG * TK + lane;
        int tb = (lane < TK && g < Nz) ? 0 : nblk;
        const int kr = BWD ? Nz - 1 - g : g;
        const long long rowbase = plane * kr;
        unsigned long long t0 = 0;
        int idle = 0;
        while (__any_sync(FULL, tb < nblk)) {
            bool issued = false;
            if (tb < nblk) {
                const int q = tb % SRF;
                const unsigned u = (unsigned)(tb / SRF);
                if (tb < SRF || mb_test(empty_f + 8 * (q * TK + lane), (u - 1) & 1u)) {
                    const int nl = min(SRL, Ny - tb * SRL);
                    const int j0 = BWD ? Ny - tb * SRL - nl : tb * SRL;   // first real line of the block
                    const long long base = rowbase + (long long)Lx * j0;
                    const unsigned fb = full_f + 8 * (q * TK + lane);
                    const unsigned lc = (unsigned)(nl * CLN * sizeof(T));
                    const unsigned lt = TAB ? (unsigned)(nl * TBW * sizeof(T)) : 0u;
                    // the rhs block rounded out to 16-byte granules (inside the allocation)
                    const unsigned long long ar = (unsigned long long)(size_t)(rhs + base);
                    const unsigned long long a0 = ar & ~15ull;
                    const unsigned lr =
                        (unsigned)(((ar + (unsigned long long)nl * Lx * sizeof(TR) + 15ull) & ~15ull) - a0);
                    mb_expect(fb, lc + lt + lr);
                    bulk_g2s(smem_u32(cwin + (size_t)(q * TK + lane) * SRL * CLN), coef4 + base * 4, lc, fb);
                    if (TAB)
                        bulk_g2s(smem_u32(twin + (size_t)(q * TK + lane) * SRL * TBW),
                                 scanm + ((long long)kr * Ny + j0) * TBW, lt, fb);
                    bulk_g2s(smem_u32(rwin + (size_t)(q * TK + lane) * WR), (const void *)(size_t)a0, lr, fb);
                    ++tb;
                    issued = true;
                }
            }
            if (__any_sync(FULL, issued)) {
                t0 = 0;
            } else {
                __nanosleep(32);
                if ((++idle & 63) == 0) {
                    const unsigned long long now = __shfl_sync(FULL, global_ns(), 0);
                    if (t0 == 0) t0 = now;
                    else if (now - t0 > wait_limit_ns(err)) {
                        if (lane == 0) atomicOr(err, kErrTimeout);
                        break;
                    }
                }
            }
        }
    } else if (w > NCW && w <= NCW + S) {
        // relay warps, one per segment: the first CTA of a cluster other than
        // the first takes its segment of the previous cluster's last row from
        // the global ring (two lines per round trip) and forwards it, retagged,
        // into row 0's exchange slots, each segment as soon as it is there
        constexpr int D = 2;
        const int s2 = w - NCW - 1;
        if (NC > 1 && K == 0 && v > 0 && KG * TK < Nz) {
            const unsigned long long *rin =
                ring + ((size_t)(v - 1) * Ny * SW + (size_t)s2 * SLW + (size_t)lane * SE) * RW;
            const unsigned rp0 = smem_u32(prog + (2 * TK * S + s2) * PP);   // + 4 p: phase p's reads
            const unsigned xo = map_cta(smem_u32(xin + (size_t)s2 * SNX * SLW * RW + (size_t)lane * NW), K);
            int tj = 0;
            unsigned long long t0 = 0;
            unsigned rseen0 = 0, rseen1 = 0;   // per phase of the lines
            bool ok = true;
            while (tj < Ny && ok) {
                unsigned long long wv[D][NW];
#pragma unroll
                for (int d = 0; d < D; ++d)
#pragma unroll
                    for (int k = 0; k < NW; ++k)
                        wv[d][k] = tj + d < Ny ? *(const volatile unsigned long long *)(rin + (size_t)(tj + d) * SW * RW + k)
                                               : 0ull;
                int ready = 0;
#pragma unroll
                for (int d = 0; d < D; ++d) {
                    bool here = tj + d < Ny;
#pragma unroll
                    for (int k = 0; k < NW; ++k) here = here && tag_is(wv[d][k], ltag);
                    if (here && ready == d) ready = d + 1;
                }
                ready = (int)__reduce_min_sync(FULL, (unsigned)ready);
                if (ready == 0) {
                    const unsigned long long now = __shfl_sync(FULL, global_ns(), 0);
                    if (t0 == 0) t0 = now;
                    else if (now - t0 > wait_limit_ns(err)) {
                        if (lane == 0) atomicOr(err, kErrTimeout);
                        ok = false;
                    }
                    continue;
                }
                t0 = 0;
#pragma unroll
                for (int d = 0; d < D; ++d) {
                    if (d >= ready || !ok) continue;
                    const int line = tj + d;
                    if (line >= SNX) {
                        const bool odd = PP > 1 && (line & 1);
                        unsigned sn = odd ? rseen1 : rseen0;
                        ok = prog_wait(rp0 + (odd ? 4u : 0u), (unsigned)(line - SNX + 1), sn, err);
                        if (odd) rseen1 = sn;
                        else rseen0 = sn;
                    }
                    if (!__all_sync(FULL, ok)) {
                        ok = false;
                        continue;
                    }
                    unsigned long long o[NW];
#pragma unroll
                    for (int k = 0; k < NW; ++k) o[k] = tw_lo((unsigned)wv[d][k], (unsigned)line + 1u);
                    const unsigned a = xo + (unsigned)((line % SNX) * SLW * RW * 8);
                    tw_put2(a, o[0], o[1]);
                    if constexpr (NW == 4) tw_put2(a + 16, o[2], o[3]);
                }
                tj += ready;
            }
        }
    } else if (w < NCW) {
        const int p = w / (TK * S), r = (w % (TK * S)) / S, s = w % S;
        const int g = KG * TK + r;
        const int rs = r * S + s;   // row and segment within the CTA
        if (g < Nz) {
            const int gl = lane;
            const int kr = BWD ? Nz - 1 - g : g;
            const long long rowbase = plane * kr;
            const bool has_src = g > 0, has_dst = g + 1 < Nz;
            const bool src_remote = r == 0, dst_remote = r == TK - 1;
            // the previous row arrives from the row above in this CTA, from the
            // previous CTA of the cluster, or (first CTA of a cluster) from the relay
            const bool src_relay = has_src && src_remote && K == 0;
            const bool dst_global = has_dst && dst_remote && (int)K == NKC - 1;
            const unsigned my_x = smem_u32(xin + (size_t)rs * SNX * SLW * RW + (size_t)gl * NW);
            const unsigned my_xprog = smem_u32(prog + rs * PP + p);   // how far the next row's phase p has read
            unsigned src_prog = 0u;                                   // where I report how far I have read
            if (has_src) {
                if (src_relay) src_prog = map_cta(smem_u32(prog + (2 * TK * S + s) * PP + p), K);
                else if (src_remote) src_prog = map_cta(smem_u32(prog + ((TK - 1) * S + s) * PP + p), K - 1);
                else src_prog = map_cta(smem_u32(prog + (rs - S) * PP + p), K);
            }
            unsigned dst_x = 0u;
            if (has_dst && !dst_global) {
                const int dst_rs = dst_remote ? s : rs + S;
                dst_x = map_cta(smem_u32(xin + (size_t)dst_rs * SNX * SLW * RW + (size_t)gl * NW), dst_remote ? K + 1 : K);
            }
            unsigned long long *ring_out =
                dst_global ? ring + ((size_t)v * Ny * SW + (size_t)s * SLW + (size_t)gl * SE) * RW : nullptr;
            // the carry from segment s - 1 and to segment s + 1 (same phase: same lines)
            const bool has_cin = s > 0, has_cout = s + 1 < S;
            const unsigned my_c = smem_u32(cin + (size_t)(rs * PP + p) * SNC * 2);
            const unsigned nxt_c = has_cout ? map_cta(smem_u32(cin + (size_t)((rs + 1) * PP + p) * SNC * 2), K) : 0u;
            const unsigned my_cprog = smem_u32(prog + (TK * S + rs) * PP + p);   // how far segment s + 1 has read
            const unsigned prv_cprog = has_cin ? map_cta(smem_u32(prog + (TK * S + rs - 1) * PP + p), K) : 0u;
            // the previous line of this segment, from the other phase (PP = 2)
            const unsigned my_pv = smem_u32(pvin + (size_t)(rs * PP + p) * 2 * SLW * RW + (size_t)gl * NW);
            const unsigned oth_pv =
                PP > 1 ? map_cta(smem_u32(pvin + (size_t)(rs * PP + (PP - 1 - p)) * 2 * SLW * RW + (size_t)gl * NW), K)
                       : 0u;
            T prev[SE];
#pragma unroll
            for (int e = 0; e < SE; ++e) prev[e] = T(0);
            unsigned xseen = 0, cseen = 0;   // last progress read of my receivers
            int cur_blk = -1;
            bool done = true;
            for (int tj = p; tj < Ny; tj += PP) {
                const int blk = tj / SRL, q = blk % SRF;
                const int nl = min(SRL, Ny - blk * SRL);
                bool ok = true;
                if (blk != cur_blk) {   // a new input block: free the last one, wait for this one
                    if (cur_blk >= 0 && gl == 0) mb_arrive_relaxed(empty_f + 8 * ((cur_blk % SRF) * TK + r));
                    ok = wait_lane(full_f + 8 * (q * TK + r), (unsigned)(blk / SRF) & 1u, err);
                    cur_blk = blk;
                }
                if (!__all_sync(FULL, ok)) {
                    done = false;
                    break;
                }
                // the slot keeps its lines in real order; this line's place in it
                const int li = BWD ? nl - 1 - (tj - blk * SRL) : tj - blk * SRL;
                const int j = BWD ? Ny - 1 - tj : tj;
                const int j0 = BWD ? Ny - blk * SRL - nl : blk * SRL;
                const long long bbase = rowbase + (long long)Lx * j0;
                const int shr = (int)((((unsigned)(size_t)rhs + (unsigned)bbase * (unsigned)sizeof(TR)) & 15u) / sizeof(TR));
                const T *cl = cwin + ((size_t)(q * TK + r) * SRL + li) * CLN;
                const TR *rl = rwin + (size_t)(q * TK + r) * WR + shr + (size_t)li * Lx;
                // what does not depend on the neighbours or the carry first
                T A[SE], B[SE], BR[SE], CB[SE], CK[SE], P[SE];
                T sv[SNL];
                if (TAB) {
                    const T *tl = twin + ((size_t)(q * TK + r) * SRL + li) * TBW + (size_t)s * seg_span(S);
#pragma unroll
                    for (int lv = 0; lv < SNL; ++lv) sv[lv] = tl[lv * 32 + gl];
#pragma unroll
                    for (int e = 0; e < SE; ++e) P[e] = S > 1 ? tl[SNL * 32 + gl * SE + e] : T(0);
                }
#pragma unroll
                for (int e = 0; e < SE; ++e) {
                    const int at = s * SLW + gl * SE + e;
                    A[e] = T(1);
                    BR[e] = T(0);
                    CB[e] = T(0);
                    CK[e] = T(0);
                    if (at < Lx) {
                        const int x = BWD ? Lx - 1 - at : at;   // real x of the cell
                        const Coef4<T> c = load_coef(cl + 4 * x);
                        // backward coefficients come scaled by 1 / U_ii (d = 1 / U_ii)
                        BR[e] = BWD ? c.d * (T)rl[x] : (T)rl[x];
                        A[e] = -c.a;
                        CB[e] = c.b;
                        CK[e] = c.c;
                    }
                }
                const unsigned xtag = (unsigned)tj + 1u;
                // the previous line of this segment (the other phase's last line)
                if (PP > 1 && tj > 0) {
                    unsigned long long wv[NW];
                    ok = tw_wait<NW>(my_pv + (unsigned)(((tj / PP) & 1) * SLW * RW * 8), (unsigned)tj, wv, err);
#pragma unroll
                    for (int e = 0; e < SE; ++e) {
                        if constexpr (RW == 2) prev[e] = (T)tw_decode2(wv[2 * e], wv[2 * e + 1]);
                        else prev[e] = (T)tw_decode1(wv[e]);
                    }
                }
#pragma unroll
                for (int e = 0; e < SE; ++e) B[e] = BR[e] - CB[e] * prev[e];
                // k-neighbour: the same segment of this line in the previous row
                if (has_src) {
                    unsigned long long wv[NW];
                    const bool okx = tw_wait<NW>(my_x + (unsigned)((tj % SNX) * SLW * RW * 8), xtag, wv, err);
                    ok = ok && okx;
                    T nk[SE];
#pragma unroll
                    for (int e = 0; e < SE; ++e) {
                        if constexpr (RW == 2) nk[e] = (T)tw_decode2(wv[2 * e], wv[2 * e + 1]);
                        else nk[e] = (T)tw_decode1(wv[e]);
                    }
#pragma unroll
                    for (int e = 0; e < SE; ++e)
                        if (s * SLW + gl * SE + e < Lx) B[e] = B[e] - CK[e] * nk[e];
                }
                if (!__all_sync(FULL, ok)) {
                    done = false;
                    break;
                }
                if (has_src && gl == 0) prog_put(src_prog, xtag);   // every lane has its words
                // the segment's recurrence from a zero start: lanes compose their
                // cells' maps, a shuffle scan composes the lanes (FP64: the scan's
                // multiplier products come precomputed with the line)
                T LB = B[0], LA = A[0];
#pragma unroll
                for (int e = 1; e < SE; ++e) {
                    LB = A[e] * LB + B[e];
                    if (!TAB) LA = A[e] * LA;
                }
                if (TAB) {
#pragma unroll
                    for (int d = 1, lv = 0; d < 32; d <<= 1, ++lv) {
                        const T pb = __shfl_up_sync(FULL, LB, d);
                        if (gl >= d) LB = sv[lv] * pb + LB;
                    }
                } else {
#pragma unroll
                    for (int d = 1; d < 32; d <<= 1) {
                        const T pa = __shfl_up_sync(FULL, LA, d), pb = __shfl_up_sync(FULL, LB, d);
                        if (gl >= d) {
                            LB = LA * pb + LB;
                            LA = LA * pa;
                        }
                    }
                    if (S > 1) {   // carry multipliers: products of A from the segment's start
                        T le = __shfl_up_sync(FULL, LA, 1);
                        if (gl == 0) le = T(1);
#pragma unroll
                        for (int e = 0; e < SE; ++e) {
                            le = le * A[e];
                            P[e] = le;
                        }
                    }
                }
                T vin = __shfl_up_sync(FULL, LB, 1);
                if (gl == 0) vin = T(0);
                T val[SE];
#pragma unroll
                for (int e = 0; e < SE - 1; ++e) {
                    vin = A[e] * vin + B[e];
                    val[e] = vin;
                }
                val[SE - 1] = LB;   // the scan's value at the lane's last cell (one dependent step fewer)
                // the value entering the segment, from segment s - 1 of this line
                if (has_cin) {
                    unsigned long long cw[2];
                    ok = tw_wait<2>(my_c + (unsigned)(((tj / PP) % SNC) * 16), xtag, cw, err);
                    if (!__all_sync(FULL, ok)) {
                        done = false;
                        break;
                    }
                    T c;
                    if constexpr (RW == 2) c = (T)tw_decode2(cw[0], cw[1]);
                    else c = (T)tw_decode1(cw[0]);
#pragma unroll
                    for (int e = 0; e < SE; ++e) val[e] = P[e] * c + val[e];
                    if (gl == 0) prog_put(prv_cprog, xtag);
                }
                // this line to the other phase (its next line's j-neighbour), then
                // to the next row, ahead of the carry: a row waits on the row
                // before it once per row, on the segment before it only once
                // per row of segments
                if (PP > 1 && tj + 1 < Ny) {
                    unsigned long long wv[NW];
                    tw_encode(val, xtag, wv);
                    const unsigned a = oth_pv + (unsigned)((((tj + 1) / PP) & 1) * SLW * RW * 8);
                    tw_put2(a, wv[0], wv[1]);
                    if constexpr (NW == 4) tw_put2(a + 16, wv[2], wv[3]);
                }
                if (has_dst) {
                    unsigned long long wv[NW];
                    tw_encode(val, dst_global ? ltag : xtag, wv);
                    if (dst_global) {
                        unsigned long long *ro = ring_out + (size_t)tj * SW * RW;
#pragma unroll
                        for (int k = 0; k < NW; ++k) *(volatile unsigned long long *)(ro + k) = wv[k];
                    } else {
                        bool ok2 = true;
                        if (tj >= SNX) ok2 = prog_wait(my_xprog, (unsigned)(tj - SNX + 1), xseen, err);
                        if (!__all_sync(FULL, ok2)) {
                            done = false;
                            break;
                        }
                        const unsigned a = dst_x + (unsigned)((tj % SNX) * SLW * RW * 8);
                        tw_put2(a, wv[0], wv[1]);
                        if constexpr (NW == 4) tw_put2(a + 16, wv[2], wv[3]);
                    }
                }
                // the value leaving the segment, to segment s + 1 (its last lane's last cell)
                bool okc = true;
                if (has_cout && gl == 31) {
                    if (tj >= PP * SNC) okc = prog_wait(my_cprog, (unsigned)(tj - PP * SNC + 1), cseen, err);
                    if (okc) {
                        unsigned long long cw[2];
                        if constexpr (RW == 2) {
                            const unsigned long long b = (unsigned long long)__double_as_longlong((double)val[SE - 1]);
                            cw[0] = tw_lo((unsigned)(b & 0xffffffffull), xtag);
                            cw[1] = tw_lo((unsigned)(b >> 32), xtag);
                        } else {
                            cw[0] = cw[1] = tw_lo(__float_as_uint((float)val[SE - 1]), xtag);
                        }
                        tw_put2(nxt_c + (unsigned)(((tj / PP) % SNC) * 16), cw[0], cw[1]);
                    }
                }
                if (!__all_sync(FULL, okc)) {
                    done = false;
                    break;
                }
                T *ob = out + rowbase + (long long)Lx * j;
#pragma unroll
                for (int e = 0; e < SE; ++e) {
                    const int at = s * SLW + gl * SE + e;
                    if (at < Lx) ob[BWD ? Lx - 1 - at : at] = val[e];
                    if (PP == 1) prev[e] = val[e];
                }
            }
            // the last block this warp read: every lane's reads of it fed a scan
            if (done && cur_blk >= 0 && gl == 0) mb_arrive_relaxed(empty_f + 8 * ((cur_blk % SRF) * TK + r));
        }
    }
    cluster_sync_all();   // no CTA leaves while a neighbour may still touch its shared memory
}

}  // namespace

namespace {

// Scan and carry multipliers of every (line, segment) of one FP64 sweep
// direction, in the sweep's order of operations: lane gl's product of its SE
// cells' multipliers A (A = -L_x forward, -U_x / U_ii backward as stored, 1
// past the line's end), the running product the shuffle scan holds before
// each level, and (several segments) each cell's product of A from the
// segment's start.  One warp per (line, segment).
template <bool BWD>
__global__ void k_pack_seg_scan(int Lx, long long lines, int S, const double *__restrict__ coef4,
                                double *__restrict__ table) {
    const long long item = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int gl = threadIdx.x & 31;
    if (item >= lines * S) return;   // whole warps
    const long long line = item / S;
    const int s = (int)(item % S);
    const double *cl = coef4 + line * Lx * 4;
    double A[SE];
#pragma unroll
    for (int e = 0; e < SE; ++e) {
        const int at = s * SLW + gl * SE + e;
        A[e] = 1.0;
        if (at < Lx) A[e] = -cl[4 * (BWD ? Lx - 1 - at : at)];
    }
    double LA = A[0];
#pragma unroll
    for (int e = 1; e < SE; ++e) LA = A[e] * LA;
    double *o = table + line * seg_table(S) + (size_t)s * seg_span(S);
#pragma unroll
    for (int d = 1, lv = 0; d < 32; d <<= 1, ++lv) {
        o[lv * 32 + gl] = LA;
        const double pa = __shfl_up_sync(0xffffffffu, LA, d);
        if (gl >= d) LA = LA * pa;
    }
    if (S > 1) {
        double le = __shfl_up_sync(0xffffffffu, LA, 1);
        if (gl == 0) le = 1.0;
#pragma unroll
        for (int e = 0; e < SE; ++e) {
            le = le * A[e];
            o[SNL * 32 + gl * SE + e] = le;
        }
    }
}

template <typename T, typename TR, bool BWD, int PP>
cudaError_t launch_seg_pp(const int dims[3], int S, int TK, int NK, int NC, const T *coef4, const T *scanm,
                          const TR *rhs, T *out, unsigned long long *tick, unsigned long long *ring, int *err,
                          cudaStream_t st, bool query_only, int *clusters) {
    auto kern = k_line_seg<T, TR, BWD, PP>;
    const size_t smem = seg_smem<T, TR>(dims[0], S, TK, PP).total;
    static size_t smem_set = 0;                      // per instantiation: attributes are raised once
    static std::atomic<bool> nonportable{false};
    cudaError_t e = raise_smem_limit(kern, smem, smem_set);
    if (e != cudaSuccess) return e;
    if (NK > 8 && !nonportable) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
        nonportable = true;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(NK * NC, 1, 1);
    cfg.blockDim = dim3(32 * (TK * S * PP + 1 + (NC > 1 ? S : 0)), 1, 1);   // + producer (+ relay per segment)
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = NK;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (query_only) return cudaOccupancyMaxActiveClusters(clusters, kern, &cfg);
    return cudaLaunchKernelEx(&cfg, kern, dims[0], dims[1], dims[2], S, TK, NC, coef4, scanm, rhs, out, tick, ring, err);
}

template <typename T, typename TR, bool BWD>
cudaError_t launch_seg(const int dims[3], int S, int TK, int PP, int NK, int NC, const T *coef4, const T *scanm,
                       const TR *rhs, T *out, unsigned long long *tick, unsigned long long *ring, int *err,
                       cudaStream_t st, bool query_only = false, int *clusters = nullptr) {
    return PP > 1 ? launch_seg_pp<T, TR, BWD, 2>(dims, S, TK, NK, NC, coef4, scanm, rhs, out, tick, ring, err, st,
                                                 query_only, clusters)
                  : launch_seg_pp<T, TR, BWD, 1>(dims, S, TK, NK, NC, coef4, scanm, rhs, out, tick, ring, err, st,
                                                 query_only, clusters);
}

template <typename T, typename TR>
bool seg_fits(const int dims[3], int S, int TK, int PP, int NK, int NC) {
    if (TK * S * PP + 1 + (NC > 1 ? S : 0) > kSegMaxWarps) return false;
    if (seg_smem<T, TR>(dims[0], S, TK, PP).total > 220 * 1024 || seg_smem<T, T>(dims[0], S, TK, PP).total > 220 * 1024)
        return false;
    int c1 = 0, c2 = 0;
    if (launch_seg<T, TR, false>(dims, S, TK, PP, NK, NC, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr,
                                 nullptr, true, &c1) != cudaSuccess ||
        launch_seg<T, T, true>(dims, S, TK, PP, NK, NC, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr,
                               nullptr, true, &c2) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return c1 >= NC && c2 >= NC;
}

}  // namespace

// Segmented sweep layout for precision p (0 FP64, 1 FP32; the right-hand side
// of the FP32 forward sweep is FP64 or FP32, both are checked): the walked
// direction (y-lines on transposed vectors when nx < ny), segments per line,
// rows per CTA (FP64 rows of several segments one per CTA, so no two rows'
// FP64 scans share a sub-partition), and the clusters the rows span.
bool plan_ilu_seg(ms_system &s, int p) {
    // both precisions by default (on the 60x220x85 grid FP32 0.110 / 0.111 ms
    // per forward / backward sweep against 0.123 / 0.119 ms with one warp per
    // line); MSGB_ILU_SEG=0 never, =1 FP64 only
    const char *e = std::getenv("MSGB_ILU_SEG");
    if (e && e[0] == '0') return false;
    if (p == 1 && e && e[0] == '1') return false;
    // MSGB_SEG_LINES=x or =y forces the walked direction (y: where ny <= 256)
    const char *ld = std::getenv("MSGB_SEG_LINES");
    bool ylines = s.ny > s.nx && s.ny <= kMaxSeg * SLW;
    if (ld && ld[0] == 'x') ylines = false;
    if (ld && ld[0] == 'y') ylines = s.ny <= kMaxSeg * SLW;
    const int dims[3] = {ylines ? s.ny : s.nx, ylines ? s.nx : s.ny, s.nz};
    if (dims[0] > kMaxSeg * SLW || dims[1] < 1 || dims[2] < 1) return false;
    const int S = (dims[0] + SLW - 1) / SLW;
    // one warp per segment; MSGB_SEG_PP=2 gives each segment two warps that
    // take the lines in turn (the previous line then travels between them
    // through shared memory: on the 60x220x85 grid 0.189 / 0.189 ms FP64
    // against 0.183 / 0.191 ms with one warp, as a hand-off between warps
    // costs about what the bookkeeping it overlaps does)
    int PP = 1;
    if (const char *t = std::getenv("MSGB_SEG_PP")) PP = std::atoi(t) >= 2 ? 2 : 1;
    int tk = (p == 0 && S > 1) || PP > 1 ? 1 : 2;
    if (const char *t = std::getenv("MSGB_SEG_TK")) tk = std::max(1, std::atoi(t));
    const int NKtot = (dims[2] + tk - 1) / tk;
    const int NC = (NKtot + 15) / 16;
    const int NK = (NKtot + NC - 1) / NC;
    const int TK = (dims[2] + NK * NC - 1) / (NK * NC);
    const bool fits = p == 0 ? seg_fits<double, double>(dims, S, TK, PP, NK, NC)
                             : seg_fits<float, double>(dims, S, TK, PP, NK, NC) &&
                                   seg_fits<float, float>(dims, S, TK, PP, NK, NC);
    if (!fits) return false;
    s.sg_S[p] = S;
    s.sg_PP[p] = PP;
    s.sg_TK[p] = TK;
    s.sg_NK[p] = NK;
    s.sg_NC[p] = NC;
    s.cl_T[p] = ylines;
    if (NC > 1) {
        s.sg_ring[p].alloc((size_t)(NC - 1) * dims[1] * S * SLW * (p == 0 ? 2 : 1));
        s.sg_ring[p].zero(nullptr);
    }
    s.sg_tick.alloc(2);
    s.sg_tick.zero(nullptr);
    s.sg_ok[p] = true;
    return true;
}

size_t seg_table_size(const ms_system &s) {
    const int Lx = s.cl_T[0] ? s.ny : s.nx;
    return (size_t)2 * (s.n / Lx) * seg_table(s.sg_S[0]);
}

void pack_seg_tables(ms_system &s, const double *coef4, double *table, cudaStream_t st) {
    const int Lx = s.cl_T[0] ? s.ny : s.nx;
    const long long lines = s.n / Lx;
    const int S = s.sg_S[0];
    const int g = (int)((lines * S + 7) / 8);
    k_pack_seg_scan<false><<<g, 256, 0, st>>>(Lx, lines, S, coef4, table);
    k_pack_seg_scan<true><<<g, 256, 0, st>>>(Lx, lines, S, coef4 + (size_t)4 * s.n, table + (size_t)lines * seg_table(S));
    MS_CHECK_LAUNCH();
}

template <typename T, typename TR>
void seg_fwd(ms_system &s, int p, const T *coef4, const T *scanm, const TR *rhs, T *out, cudaStream_t st) {
    const bool yl = s.cl_T[p];
    const int dims[3] = {yl ? s.ny : s.nx, yl ? s.nx : s.ny, s.nz};
    MS_CUDA((launch_seg<T, TR, false>(dims, s.sg_S[p], s.sg_TK[p], s.sg_PP[p], s.sg_NK[p], s.sg_NC[p], coef4, scanm, rhs, out,
                                      s.sg_tick.p + p, s.sg_ring[p].p, s.sync.p + 3, st)));
}

template <typename T>
void seg_bwd(ms_system &s, int p, const T *coef4, const T *scanm, const T *rhs, T *out, cudaStream_t st) {
    const bool yl = s.cl_T[p];
    const int dims[3] = {yl ? s.ny : s.nx, yl ? s.nx : s.ny, s.nz};
    MS_CUDA((launch_seg<T, T, true>(dims, s.sg_S[p], s.sg_TK[p], s.sg_PP[p], s.sg_NK[p], s.sg_NC[p], coef4, scanm, rhs, out,
                                    s.sg_tick.p + p, s.sg_ring[p].p, s.sync.p + 3, st)));
}

template void seg_fwd<double, double>(ms_system &, int, const double *, const double *, const double *, double *,
                                      cudaStream_t);
template void seg_fwd<float, double>(ms_system &, int, const float *, const float *, const double *, float *,
                                     cudaStream_t);
template void seg_fwd<float, float>(ms_system &, int, const float *, const float *, const float *, float *,
                                    cudaStream_t);
template void seg_bwd<double>(ms_system &, int, const double *, const double *, const double *, double *, cudaStream_t);
template void seg_bwd<float>(ms_system &, int, const float *, const float *, const float *, float *, cudaStream_t);

}  // namespace msgb
