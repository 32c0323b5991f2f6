// ILU(0) triangular sweeps on structured grids: line scan pipelined across
// one thread-block cluster.
//
// Natural-order ILU(0) on the 7-point pattern (the smoother of the second
// stage of the multistage cycle, Sec. 3): the forward sweep is
//     y(x,j,k) = r - Lx y(x-1,j,k) - Ly y(x,j-1,k) - Lz y(x,j,k-1),
// the backward sweep the mirror image with U and the reciprocal diagonal.
// Given the neighbouring x-lines (j-1,k) and (j,k-1), the x-line (j,k) is the
// first-order recurrence v(x) = A(x) v(x-1) + B(x), which one warp solves with
// an affine shuffle scan (E consecutive cells per lane).
//
// Every k-row of x-lines is owned by one warp, which walks its row along j
// and keeps the previous line (the j-neighbour) in registers.  Row g needs
// line j of row g-1 (the k-neighbour): rows hand finished lines to the next
// row through a small ring of shared-memory buffers guarded by mbarriers
// (full / empty), so each row waits only for its own neighbour instead of for
// a block-wide barrier, and rows drift into a natural wavefront.  The rows are
// split over the CTAs of one cluster (TK rows per CTA).  A line is handed over
// with asynchronous stores into the next row's buffer (in the next CTA for the
// last row of a CTA, through distributed shared memory) that count as
// transaction bytes on the receiver's barrier, so no release fence is needed
// and a CTA boundary costs the same as a warp boundary; the receiver re-arms
// its barrier with the expected byte count when it frees the buffer.  A
// producer warp per CTA streams each row's inputs (the packed coefficient line
// and the right-hand-side line, one bulk copy each) into a ring of
// shared-memory slots, independently per row.
//
// Coefficients are packed four per cell (x, y, z neighbour and a fourth
// entry: zero forward, the reciprocal diagonal backward), so a coefficient
// line starts on a 16-byte boundary and is one bulk copy.  All waits are
// bounded in device time and report a timeout instead of hanging.
#include <atomic>

#include <cstdlib>

#include <string>

#include "ms_internal.h"
#include "line_sync.cuh"

namespace msgb {

namespace {

constexpr int RF = 4;    // fetch ring: lines in flight per row
// warps per CTA when the rows span several clusters, for grids deep enough
// that one cluster would hold at least kClusterSplitFrom warps per CTA (the
// 60x220x85 sweeps: 340 / 357 us FP64 with 6 warps per CTA in one cluster,
// 312 / 329 us with 2 per CTA over three)
constexpr int kClusterTK64 = 2;
constexpr int kClusterTK32 = 2;
constexpr int kClusterSplitFrom = 4;
constexpr int NBX = 4;   // row-exchange ring: lines a row may run ahead of the next


// G k-rows per warp, in lane groups of L = 32 / G lanes; E cells per lane.
// The rows may span several clusters (NC of them, gridDim.x / NC CTAs each):
// each cluster takes a ticket when it starts, and the ticket, not the launch
// position, decides which block of rows it owns, so a cluster only ever waits
// for one that started before it; at a cluster boundary the line goes through
// a global ring (one tagged slot per line), so the sender never waits.
// Warp step t: group h solves line t - h of its row, so the k-neighbour of
// groups h > 0 is the line group h - 1 finished in step t - 1 (passed by a
// shuffle); group 0 receives its k-neighbour from the previous warp's last
// row through the exchange ring, and group G - 1 sends to the next warp's.
template <typename T, typename TR, bool BWD, int E, int G>
__global__ void __launch_bounds__(544, 1)
    k_line_cluster(int nx, int ny, int nz, int TK, int NC, const T *__restrict__ coef4, const T *__restrict__ scanm,
                   const TR *__restrict__ rhs, T *__restrict__ out, unsigned long long *tick,
                   unsigned long long *ring, int *err) {
    constexpr int L = 32 / G;
    constexpr int LW = L * E;
    // FP64 only: the FP64 pipe bounds those sweeps; FP32 multiplies are cheap and
    // table loads would only add shared-memory latency to the scan
    constexpr bool TAB = sizeof(T) == 8;
    constexpr int SCN = TAB ? scan_table(L) : 0;
    constexpr unsigned FULL = 0xffffffffu;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const unsigned K = cluster_rank();
    const int RPC = TK * G;   // rows per CTA
    const int WR = rhs_win(nx, sizeof(TR));
    const int CLN = nx * 4;   // packed coefficient line (elements of T)
    const int CLS = CLN + SCN;   // a coefficient slot: the line's coefficients, then its scan multipliers
    // shared: coefficient slots [RF][RPC][CLS] T | rhs slots [RF][RPC][WR] TR | exchange [TK][NBX][LW] T |
    //         barriers full_f, empty_f [RF][RPC], full_x, empty_x [NBX][TK]
    extern __shared__ __align__(16) unsigned char smraw[];
    T *cwin = reinterpret_cast<T *>(smraw);
    size_t off = (size_t)RF * RPC * CLS * sizeof(T);
    TR *rwin = reinterpret_cast<TR *>(smraw + off);
    off += (size_t)RF * RPC * WR * sizeof(TR);
    T *xin = reinterpret_cast<T *>(smraw + off);
    off += (size_t)TK * NBX * LW * sizeof(T);
    const unsigned full_f = smem_u32(smraw + off);
    const unsigned empty_f = full_f + 8 * RF * RPC;
    const unsigned full_x = empty_f + 8 * RF * RPC;
    const unsigned empty_x = full_x + 8 * NBX * TK;
    const unsigned empty_r = empty_x + 8 * NBX * TK;     // [NBX]: warp 0 frees a slot the relay warp filled

    __shared__ unsigned long long s_tick;
    if (NC > 1 && K == 0 && tid == 0) s_tick = atomicAdd(tick, 1ull);
    if (tid < RPC) {
        for (int q = 0; q < RF; ++q) {
            mb_init(full_f + 8 * (q * RPC + tid), 1);
            mb_init(empty_f + 8 * (q * RPC + tid), 1);
        }
    }
    if (tid < TK) {
        for (int b = 0; b < NBX; ++b) {
            mb_init(full_x + 8 * (b * TK + tid), 1);
            mb_init(empty_x + 8 * (b * TK + tid), 1);
        }
    }
    if (tid < NBX) mb_init(empty_r + 8 * tid, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    cluster_sync_all();
    // this cluster's block of rows (v) and the launch's tag, from rank 0's ticket
    unsigned long long tk = 0;
    if (NC > 1) {
        const unsigned a = map_cta(smem_u32(&s_tick), 0);
        asm volatile("ld.shared::cluster.u64 %0, [%1];" : "=l"(tk) : "r"(a) : "memory");
    }
    const int NKC = (int)gridDim.x / NC;                 // CTAs per cluster
    const int v = (int)(tk % (unsigned long long)NC);
    const unsigned tag = (unsigned)(tk / (unsigned long long)NC) + 1u;
    const int KG = v * NKC + (int)K;                     // CTA position in the row order

    const long long plane = (long long)nx * ny;
    const long long dj = BWD ? -(long long)nx : (long long)nx;   // real index step from line j to j+1 (mirrored)
    if (w == TK) {
        // producer warp: lane r streams the inputs of row r, each row on its own
        const int g = KG * RPC + lane;
        int tj = (lane < RPC && g < nz) ? 0 : ny;
        const int kr = BWD ? nz - 1 - g : g;
        const long long base0 = (long long)nx * (BWD ? ny - 1 : 0) + plane * kr;
        const unsigned lc = (unsigned)nx * 4 * sizeof(T);
        constexpr unsigned ls = (unsigned)SCN * sizeof(T);
        unsigned long long t0 = 0;
        int idle = 0;
        while (__any_sync(FULL, tj < ny)) {
            bool issued = false;
            if (tj < ny) {
                const int q = tj % RF;
                const unsigned u = (unsigned)(tj / RF);
                if (tj < RF || mb_test(empty_f + 8 * (q * RPC + lane), (u - 1) & 1u)) {
                    const long long base = base0 + dj * tj;
                    const unsigned fb = full_f + 8 * (q * RPC + lane);
                    // the rhs line rounded out to 16-byte granules (never leaving the
                    // granule of a valid address, so inside the mapped allocation)
                    const unsigned long long ar = (unsigned long long)(size_t)(rhs + base);
                    const unsigned long long a0 = ar & ~15ull;
                    const unsigned lr = (unsigned)(((ar + (unsigned long long)nx * sizeof(TR) + 15ull) & ~15ull) - a0);
                    mb_expect(fb, lc + ls + lr);
                    bulk_g2s(smem_u32(cwin + (size_t)(q * RPC + lane) * CLS), coef4 + base * 4, lc, fb);
                    if (TAB)
                        bulk_g2s(smem_u32(cwin + (size_t)(q * RPC + lane) * CLS + CLN), scanm + (base / nx) * SCN, ls,
                                 fb);
                    bulk_g2s(smem_u32(rwin + (size_t)(q * RPC + lane) * WR), (const void *)(size_t)a0, lr, fb);
                    ++tj;
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
    } else if (w == TK + 1) {
        // relay warp (rows spanning several clusters): the first CTA of a cluster
        // other than the first takes the previous cluster's last row from the
        // global ring and hands each line to its warp 0 through the exchange
        // ring, so the ring's polling stays off warp 0's steps.  Loads for the
        // next D lines stay in flight; the lines that have arrived, in order,
        // are forwarded after each round trip.
        if constexpr (G == 1) {
            constexpr int RW = ring_words<T>();
            constexpr int D = 8 / E > 0 ? 8 / E : 1;
            constexpr int NWD = E * RW;                   // words of one lane's values of a line
            if (K == 0 && v > 0 && KG * TK < nz) {
                const unsigned long long *rin = ring + ((size_t)(v - 1) * ny * LW + lane * E) * RW;
                const unsigned xo0 = map_cta(smem_u32(xin + (size_t)lane * E), K);   // warp 0's slots
                const unsigned fb0 = map_cta(full_x, K);
                int tj = 0;
                unsigned long long t0 = 0;
                bool ok = true;
                while (tj < ny && ok) {
                    unsigned long long wv[D][NWD];
#pragma unroll
                    for (int d = 0; d < D; ++d)
#pragma unroll
                        for (int k = 0; k < NWD; ++k)
                            wv[d][k] = tj + d < ny ? *(const volatile unsigned long long *)(rin + (size_t)(tj + d) * LW * RW + k)
                                                   : 0ull;
                    int ready = 0;
#pragma unroll
                    for (int d = 0; d < D; ++d) {
                        bool here = tj + d < ny;
#pragma unroll
                        for (int k = 0; k < NWD; ++k) here = here && (unsigned)(wv[d][k] >> 32) == tag;
                        if (here && ready == d) ready = d + 1;
                    }
                    ready = (int)__reduce_min_sync(0xffffffffu, (unsigned)ready);
                    if (ready == 0) {
                        const unsigned long long now = __shfl_sync(0xffffffffu, global_ns(), 0);
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
                        if (d >= ready) break;
                        const int line = tj + d;
                        const int bs = line % NBX;
                        const unsigned ubs = (unsigned)(line / NBX);
                        if (line >= NBX) ok = wait_lane(empty_r + 8 * bs, (ubs - 1) & 1u, err);
                        if (!__all_sync(0xffffffffu, ok)) {
                            ok = false;
                            break;
                        }
                        T val[E];
#pragma unroll
                        for (int e = 0; e < E; ++e) {
                            if (RW == 2) {
                                const unsigned long long bits = (wv[d][2 * e] & 0xffffffffull) | (wv[d][2 * e + 1] << 32);
                                val[e] = (T)__longlong_as_double((long long)bits);
                            } else {
                                val[e] = (T)__uint_as_float((unsigned)(wv[d][e] & 0xffffffffull));
                            }
                        }
                        const unsigned xo = xo0 + (unsigned)(bs * LW * sizeof(T)), fb = fb0 + 8 * bs * TK;
#pragma unroll
                        for (int e = 0; e < E; e += 2) st_async2(xo + e * (unsigned)sizeof(T), val[e], val[e + 1], fb);
                    }
                    tj += ready;
                }
            }
        }
    } else if (w < TK && (KG * TK + w) * G < nz) {
        const int grp = lane / L, gl = lane % L;
        const int wrow0 = (KG * TK + w) * G;                 // first row of this warp
        const int g = wrow0 + grp;                           // row of this lane's group
        const int rl = w * G + grp;                          // row within the CTA
        const bool live = g < nz;
        const int kr = BWD ? nz - 1 - g : g;
        const long long base0 = (long long)nx * (BWD ? ny - 1 : 0) + plane * kr;
        const bool has_src = wrow0 > 0;                      // the previous warp's last row exists
        const bool has_dst = wrow0 + G < nz;                 // the next warp's first row exists (this warp full)
        const bool src_remote = w == 0, dst_remote = w == TK - 1;
        // across a cluster boundary: through the global ring (received by the
        // relay warp of this CTA, which fills warp 0's exchange ring)
        const bool src_relay = has_src && src_remote && K == 0;
        const bool dst_global = has_dst && dst_remote && (int)K == NKC - 1;
        // a line handed to the next warp: LW values (cells past nx are padding)
        constexpr unsigned XB = LW * sizeof(T);
        constexpr int RW = ring_words<T>();
        if (has_src && lane == 0)
            for (int b = 0; b < NBX && b < ny; ++b) mb_expect_relaxed(full_x + 8 * (b * TK + w), XB);
        const unsigned dst_rank = dst_remote && !dst_global ? K + 1 : K;
        const int dst_w = dst_remote ? 0 : w + 1;
        const unsigned dst_xin = dst_global ? 0u : map_cta(smem_u32(xin + (size_t)dst_w * NBX * LW + gl * E), dst_rank);
        const unsigned dst_full = dst_global ? 0u : map_cta(full_x + 8 * dst_w, dst_rank);
        const unsigned src_empty =
            !has_src ? 0u
                     : (src_relay ? empty_r : map_cta(empty_x + 8 * (src_remote ? TK - 1 : w - 1), src_remote ? K - 1 : K));
        // ring slots: [boundary][line][LW values][RW words]; the last row of a cluster writes boundary v
        unsigned long long *ring_out = dst_global ? ring + ((size_t)v * ny * LW + gl * E) * RW : nullptr;
        T prev[E];
#pragma unroll
        for (int e = 0; e < E; ++e) prev[e] = T(0);
        const int steps = ny + G - 1;
        for (int t = 0; t < steps; ++t) {
            const int tj = t - grp;
            const bool act = live && tj >= 0 && tj < ny;
            const int q = act ? tj % RF : 0;
            const unsigned u = act ? (unsigned)(tj / RF) : 0u;
            bool ok = true;
            if (act) ok = wait_lane(full_f + 8 * (q * RPC + rl), u & 1u, err);
            // everything that does not depend on the k-neighbour first: the
            // multipliers, the scan table and the offsets' in-row terms
            T A[E], B[E], CK[E];
#pragma unroll
            for (int e = 0; e < E; ++e) {
                A[e] = T(1);
                B[e] = T(0);
                CK[e] = T(0);
            }
            constexpr int NLV = scan_levels(L);
            T sv[NLV];                      // this lane's scan multipliers from the line's table (FP64)
            if (TAB) {
                const T *sm = cwin + (size_t)(q * RPC + rl) * CLS + CLN + gl;
#pragma unroll
                for (int lv = 0; lv < NLV; ++lv) sv[lv] = act ? sm[lv * L] : T(0);
            }
            long long base = 0;
            if (act) {
                base = base0 + dj * tj;
                const int shr =
                    (int)((((unsigned)(size_t)rhs + (unsigned)base * (unsigned)sizeof(TR)) & 15u) / sizeof(TR));
                const T *cl = cwin + (size_t)(q * RPC + rl) * CLS;
                const TR *rl_ = rwin + (size_t)(q * RPC + rl) * WR + shr;
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    const int at = gl * E + e;
                    if (at < nx) {
                        const int x = BWD ? nx - 1 - at : at;   // real x of the cell
                        const Coef4<T> c = load_coef(cl + 4 * x);
                        // backward coefficients come scaled by 1 / U_ii (d = 1 / U_ii)
                        B[e] = (BWD ? c.d * (T)rl_[x] : (T)rl_[x]) - c.b * prev[e];
                        A[e] = -c.a;
                        CK[e] = c.c;
                    }
                }
            }
            // k-neighbour: the group below finished this line in the previous step
            T nk[E];
#pragma unroll
            for (int e = 0; e < E; ++e) nk[e] = G > 1 ? __shfl_up_sync(FULL, prev[e], L) : T(0);
            const int b = t % NBX;
            const unsigned ub = (unsigned)(t / NBX);
            const bool recv = grp == 0 && has_src && act;
            if (grp == 0) {
#pragma unroll
                for (int e = 0; e < E; ++e) nk[e] = T(0);
            }
            if (recv) {
                ok = ok && wait_lane(full_x + 8 * (b * TK + w), ub & 1u, err);
                const T *xi = xin + ((size_t)w * NBX + b) * LW + gl * E;
#pragma unroll
                for (int e = 0; e < E; ++e) nk[e] = xi[e];
            }
            if (!__all_sync(FULL, ok)) break;
            if (act) {
#pragma unroll
                for (int e = 0; e < E; ++e)
                    if (gl * E + e < nx) B[e] = B[e] - CK[e] * nk[e];
            }
            // lanes compose their cells' maps, then a shuffle scan composes the
            // lanes.  The products of the multipliers the scan needs at each level
            // do not depend on the right-hand side: in FP64 they come precomputed
            // with the line, so only the offsets are scanned.
            T LB = B[0];
            if (TAB) {
#pragma unroll
                for (int e = 1; e < E; ++e) LB = A[e] * LB + B[e];
#pragma unroll
                for (int d = 1, lv = 0; d < L; d <<= 1, ++lv) {
                    const T pb = __shfl_up_sync(FULL, LB, d, L);
                    if (gl >= d) LB = sv[lv] * pb + LB;
                }
            } else {
                T LA = A[0];
#pragma unroll
                for (int e = 1; e < E; ++e) {
                    LB = A[e] * LB + B[e];
                    LA = A[e] * LA;
                }
#pragma unroll
                for (int d = 1; d < L; d <<= 1) {
                    const T pa = __shfl_up_sync(FULL, LA, d, L), pb = __shfl_up_sync(FULL, LB, d, L);
                    if (gl >= d) {
                        LB = LA * pb + LB;
                        LA = LA * pa;
                    }
                }
            }
            T v = __shfl_up_sync(FULL, LB, 1, L);
            if (gl == 0) v = T(0);
            T val[E];
#pragma unroll
            for (int e = 0; e < E; ++e) {
                v = A[e] * v + B[e];
                val[e] = v;
            }
            // every lane's reads of its slot and of the exchange buffer fed the scan
            // (a warp-wide shuffle), so they are complete: hand both back
            if (act && gl == 0) mb_arrive_relaxed(empty_f + 8 * (q * RPC + rl));
            if (recv && gl == 0) {
                if (t + NBX < ny) mb_expect_relaxed(full_x + 8 * (b * TK + w), XB);
                if (src_relay) mb_arrive_relaxed(src_empty + 8 * b);
                else if (src_remote) mb_arrive_relaxed_remote(src_empty + 8 * b * TK);
                else mb_arrive_relaxed(src_empty + 8 * b * TK);
            }
            if (act) {
#pragma unroll
                for (int e = 0; e < E; ++e) prev[e] = val[e];
            }
            // the last group passes its line to the next warp
            const bool send = has_dst && grp == G - 1 && act;
            bool ok2 = true;
            if (send && dst_global) {
                unsigned long long *ro = ring_out + (size_t)tj * LW * RW;
#pragma unroll
                for (int e = 0; e < E; ++e) ring_put(ro + e * RW, val[e], tag);
            } else if (send) {
                const int bs = tj % NBX;
                const unsigned ubs = (unsigned)(tj / NBX);
                if (tj >= NBX) ok2 = wait_lane(empty_x + 8 * (bs * TK + w), (ubs - 1) & 1u, err);
                if (ok2) {
                    const unsigned xo = dst_xin + (unsigned)(bs * LW * sizeof(T)), fb = dst_full + 8 * bs * TK;
#pragma unroll
                    for (int e = 0; e < E; e += 2) st_async2(xo + e * (unsigned)sizeof(T), val[e], val[e + 1], fb);
                }
            }
            if (act) {
                T *ob = out + base;
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    const int at = gl * E + e;
                    if (at < nx) ob[BWD ? nx - 1 - at : at] = val[e];
                }
            }
            if (!__all_sync(FULL, ok2)) break;
        }
    }
    cluster_sync_all();   // no CTA leaves while a neighbour may still touch its shared memory
}

// Packed sweep coefficients.  x-lines: cell i keeps (Lx, Ly, Lz, 0) and
// (Ux, Uy, Uz, 1/U_ii).  y-lines (transposed = 1): the cell moves to
// t = y + ny (x + nx z) and keeps (Ly, Lx, Lz, 0) and (Uy, Ux, Uz, 1/U_ii), so
// that the in-line neighbour comes first, then the previous line's.
// ILU(0) factorisation of the 7-point pattern in natural order: no fill, so
// U keeps A's upper entries, L_ik = A_ik / u_k, and only the pivots follow a
// recurrence, u_i = A_ii - sum over the lower neighbours k of A_ik A_ki / u_k.
// Its dependencies are those of the forward sweep, so the same cluster line
// pipeline computes it: a warp per k-row, lines walked along j, the j- and
// k-neighbour pivots (as 1/u) from registers and the exchange ring; within a
// line the x-recurrence is a composition of projective maps, scanned across
// the lanes.
// Input per cell (c_x, c_y, c_z, A_ii) with c_d = A_ik A_ki; output 1/u.
template <int E>
__global__ void __launch_bounds__(544, 1)
    k_factor_cluster(int nx, int ny, int nz, int TK, const double *__restrict__ fac4, double *__restrict__ dinv,
                     int *err) {
    constexpr int LW = 32 * E;
    constexpr unsigned FULL = 0xffffffffu;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const unsigned K = cluster_rank();
    const int CLN = nx * 4;
    // shared: coefficient slots [RF][TK][CLN] | exchange [TK][NBX][LW] |
    //         barriers full_f, empty_f [RF][TK], full_x, empty_x [NBX][TK]
    extern __shared__ __align__(16) unsigned char smraw[];
    double *cwin = reinterpret_cast<double *>(smraw);
    size_t off = (size_t)RF * TK * CLN * sizeof(double);
    double *xin = reinterpret_cast<double *>(smraw + off);
    off += (size_t)TK * NBX * LW * sizeof(double);
    const unsigned full_f = smem_u32(smraw + off);
    const unsigned empty_f = full_f + 8 * RF * TK;
    const unsigned full_x = empty_f + 8 * RF * TK;
    const unsigned empty_x = full_x + 8 * NBX * TK;
    if (tid < TK) {
        for (int q = 0; q < RF; ++q) {
            mb_init(full_f + 8 * (q * TK + tid), 1);
            mb_init(empty_f + 8 * (q * TK + tid), 1);
        }
        for (int b = 0; b < NBX; ++b) {
            mb_init(full_x + 8 * (b * TK + tid), 1);
            mb_init(empty_x + 8 * (b * TK + tid), 1);
        }
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    cluster_sync_all();
    const long long plane = (long long)nx * ny;
    if (w == TK) {
        // producer warp: lane r streams the packed lines of row r
        const int g = (int)K * TK + lane;
        int tj = (lane < TK && g < nz) ? 0 : ny;
        const unsigned lc = (unsigned)nx * 32;
        unsigned long long t0 = 0;
        int idle = 0;
        while (__any_sync(FULL, tj < ny)) {
            bool issued = false;
            if (tj < ny) {
                const int q = tj % RF;
                const unsigned u = (unsigned)(tj / RF);
                if (tj < RF || mb_test(empty_f + 8 * (q * TK + lane), (u - 1) & 1u)) {
                    const long long base = (long long)nx * tj + plane * g;
                    const unsigned fb = full_f + 8 * (q * TK + lane);
                    mb_expect(fb, lc);
                    bulk_g2s(smem_u32(cwin + (size_t)(q * TK + lane) * CLN), fac4 + base * 4, lc, fb);
                    ++tj;
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
    } else if (w < TK && (int)K * TK + w < nz) {
        const int g = (int)K * TK + w;
        const bool has_src = g > 0, has_dst = g + 1 < nz;
        const bool src_remote = w == 0, dst_remote = w == TK - 1;
        constexpr unsigned XB = LW * sizeof(double);
        if (has_src && lane == 0)
            for (int b = 0; b < NBX && b < ny; ++b) mb_expect_relaxed(full_x + 8 * (b * TK + w), XB);
        const unsigned dst_rank = dst_remote ? K + 1 : K;
        const int dst_w = dst_remote ? 0 : w + 1;
        const unsigned dst_xin = map_cta(smem_u32(xin + (size_t)dst_w * NBX * LW + lane * E), dst_rank);
        const unsigned dst_full = map_cta(full_x + 8 * dst_w, dst_rank);
        const unsigned src_empty = has_src ? map_cta(empty_x + 8 * (src_remote ? TK - 1 : w - 1), src_remote ? K - 1 : K) : 0u;
        double prev[E];
#pragma unroll
        for (int e = 0; e < E; ++e) prev[e] = 0.0;
        for (int tj = 0; tj < ny; ++tj) {
            const int q = tj % RF, b = tj % NBX;
            const unsigned u = (unsigned)(tj / RF), ub = (unsigned)(tj / NBX);
            bool ok = wait_lane(full_f + 8 * (q * TK + w), u & 1u, err);
            double nk[E];
#pragma unroll
            for (int e = 0; e < E; ++e) nk[e] = 0.0;
            if (has_src) {
                ok = ok && wait_lane(full_x + 8 * (b * TK + w), ub & 1u, err);
                const double *xi = xin + ((size_t)w * NBX + b) * LW + lane * E;
#pragma unroll
                for (int e = 0; e < E; ++e) nk[e] = xi[e];
            }
            if (!__all_sync(FULL, ok)) break;
            // u_x = a'_x - c_x / u_{x-1} is the projective map v -> M_x v on
            // v = (u, 1), M_x = [[a'_x, -c_x], [1, 0]]: lanes compose their cells'
            // maps, a shuffle scan composes the lanes (each product rescaled by a
            // power of two, exact, so the entries stay near 1), and each lane
            // applies the maps to the vector coming from the cells before it.
            const double *cl = cwin + (size_t)(q * TK + w) * CLN;
            double ma[E], mc[E];
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int x = lane * E + e;
                ma[e] = 1.0;   // padding cells are skipped below
                mc[e] = 0.0;
                if (x < nx) {
                    const double4 c = reinterpret_cast<const double4 *>(cl)[x];
                    ma[e] = c.w - c.y * prev[e] - c.z * nk[e];   // A_ii minus the j- and k-neighbour terms
                    mc[e] = c.x;
                }
            }
            // lane product P = M_{E-1} ... M_0 (padding cells contribute the identity)
            double p00 = 1.0, p01 = 0.0, p10 = 0.0, p11 = 1.0;
#pragma unroll
            for (int e = 0; e < E; ++e) {
                if (lane * E + e < nx) {
                    const double n00 = ma[e] * p00 - mc[e] * p10, n01 = ma[e] * p01 - mc[e] * p11;
                    p10 = p00;
                    p11 = p01;
                    p00 = n00;
                    p01 = n01;
                }
            }
            auto rescale = [](double &a, double &b, double &c, double &d) {
                const double m = fmax(fmax(fabs(a), fabs(b)), fmax(fabs(c), fabs(d)));
                if (m > 0.0 && m < INFINITY) {
                    const int k = ilogb(m);
                    a = scalbn(a, -k);
                    b = scalbn(b, -k);
                    c = scalbn(c, -k);
                    d = scalbn(d, -k);
                }
            };
            rescale(p00, p01, p10, p11);
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const double q00 = __shfl_up_sync(FULL, p00, d), q01 = __shfl_up_sync(FULL, p01, d);
                const double q10 = __shfl_up_sync(FULL, p10, d), q11 = __shfl_up_sync(FULL, p11, d);
                if (lane >= d) {   // P <- P Q (the earlier lanes' maps act first)
                    const double n00 = p00 * q00 + p01 * q10, n01 = p00 * q01 + p01 * q11;
                    const double n10 = p10 * q00 + p11 * q10, n11 = p10 * q01 + p11 * q11;
                    p00 = n00;
                    p01 = n01;
                    p10 = n10;
                    p11 = n11;
                    rescale(p00, p01, p10, p11);
                }
            }
            // vector entering this lane: earlier lanes' product applied to (1, 0) (u_{-1} infinite)
            double v0 = __shfl_up_sync(FULL, p00, 1), v1 = __shfl_up_sync(FULL, p10, 1);
            if (lane == 0) {
                v0 = 1.0;
                v1 = 0.0;
            }
            double val[E];
            bool bad = false;
#pragma unroll
            for (int e = 0; e < E; ++e) {
                val[e] = 0.0;
                if (lane * E + e < nx) {
                    const double n0 = ma[e] * v0 - mc[e] * v1;
                    v1 = v0;
                    v0 = n0;
                    const double m = fmax(fabs(v0), fabs(v1));
                    if (m > 0.0 && m < INFINITY) {
                        const int k = ilogb(m);
                        v0 = scalbn(v0, -k);
                        v1 = scalbn(v1, -k);
                    }
                    val[e] = v1 / v0;   // 1 / u_x
                    bad |= !(val[e] > 0.0);
                }
            }
            if (bad) atomicOr(err, kErrSingular);
            if (lane == 0) {
                mb_arrive_relaxed(empty_f + 8 * (q * TK + w));
                if (has_src) {
                    if (tj + NBX < ny) mb_expect_relaxed(full_x + 8 * (b * TK + w), XB);
                    if (src_remote) mb_arrive_relaxed_remote(src_empty + 8 * b * TK);
                    else mb_arrive_relaxed(src_empty + 8 * b * TK);
                }
            }
#pragma unroll
            for (int e = 0; e < E; ++e) prev[e] = val[e];
            bool ok2 = true;
            if (has_dst) {
                if (tj >= NBX) ok2 = wait_lane(empty_x + 8 * (b * TK + w), (ub - 1) & 1u, err);
                if (ok2) {
                    const unsigned xo = dst_xin + (unsigned)(b * LW * sizeof(double)), fb = dst_full + 8 * b * TK;
#pragma unroll
                    for (int e = 0; e < E; e += 2) st_async2(xo + e * (unsigned)sizeof(double), val[e], val[e + 1], fb);
                }
            }
            double *ob = dinv + (long long)nx * tj + plane * g;
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int x = lane * E + e;
                if (x < nx) ob[x] = val[e];
            }
            if (!__all_sync(FULL, ok2)) break;
        }
    }
    cluster_sync_all();
}

// (c_x, c_y, c_z, A_ii) per cell from the pinned ELL matrix: c_d = A_ik A_ki for
// the lower neighbour k in direction d (0 where there is none)
__global__ void k_pack_factor(int n, const int8_t *__restrict__ dslot, const int *__restrict__ col,
                              const double *__restrict__ off, const double *__restrict__ diag, double *__restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double c[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        c[d] = 0.0;
        const int wl = dslot[(int64_t)d * n + i];
        if (wl >= 0) {
            const int k = col[(int64_t)wl * n + i];
            const int wu = dslot[(int64_t)(d + 3) * n + k];   // k's slot pointing back to i
            if (wu >= 0) c[d] = off[(int64_t)wl * n + i] * off[(int64_t)wu * n + k];
        }
    }
    double *o = out + (size_t)i * 4;
    o[0] = c[0];
    o[1] = c[1];
    o[2] = c[2];
    o[3] = diag[i];
}

// L_ik = A_ik / u_k in the lower slots, A's entries in the upper slots
__global__ void k_factor_finish(int n, int W, const int *__restrict__ col, const double *__restrict__ off,
                                const double *__restrict__ dinv, double *__restrict__ lu) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int w = 0; w < W; ++w) {
        const int64_t at = (int64_t)w * n + i;
        const int k = col[at];
        lu[at] = k < i ? off[at] * dinv[k] : off[at];
    }
}

template <typename T>
__global__ void k_pack_coef4(int n, int nx, int ny, int transposed, const T *__restrict__ dcoef,
                             const T *__restrict__ dinv, T *__restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int t = i, a = 0, b = 1;
    if (transposed) {
        const int x = i % nx, y = (i / nx) % ny, z = i / (nx * ny);
        t = y + ny * (x + nx * z);
        a = 1;
        b = 0;
    }
    T *l = out + (size_t)t * 4, *u = out + ((size_t)n + t) * 4;
    l[0] = dcoef[(size_t)a * n + i];
    l[1] = dcoef[(size_t)b * n + i];
    l[2] = dcoef[(size_t)2 * n + i];
    l[3] = T(0);
    const T di = dinv[i];   // backward sweep: x_i = d (y_i - sum U_ij x_j), the U_ij stored times d
    u[0] = dcoef[(size_t)(3 + a) * n + i] * di;
    u[1] = dcoef[(size_t)(3 + b) * n + i] * di;
    u[2] = dcoef[(size_t)5 * n + i] * di;
    u[3] = di;
}

// Scan multipliers of every line of one sweep direction: lane gl's product of
// its E cells' multipliers A (A = -L_x forward, -U_x / U_ii backward as stored, 1 past
// the line's end) and the running products the sweep's shuffle scan forms
// before each level, in the sweep's order of operations (so the sweep's
// results do not change).  One warp per line; table [line][level][lane].
template <typename T, bool BWD, int E>
__global__ void k_pack_scan(int nx, long long lines, const T *__restrict__ coef4, T *__restrict__ table) {
    constexpr int L = 32;
    const long long line = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int gl = threadIdx.x & 31;
    if (line >= lines) return;                // whole warps
    const T *cl = coef4 + line * nx * 4;
    T A[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int at = gl * E + e;
        A[e] = T(1);
        if (at < nx) {
            const int x = BWD ? nx - 1 - at : at;
            A[e] = -cl[4 * x];    // backward coefficients are stored scaled by 1 / U_ii
        }
    }
    T LA = A[0];
#pragma unroll
    for (int e = 1; e < E; ++e) LA = A[e] * LA;
    T *o = table + line * scan_table(L) + gl;
#pragma unroll
    for (int d = 1, lv = 0; d < L; d <<= 1, ++lv) {
        o[lv * L] = LA;
        const T pa = __shfl_up_sync(0xffffffffu, LA, d);
        if (gl >= d) LA = LA * pa;
    }
}

// out[y + ny (x + nx z)] = in[x + nx (y + ny z)] (inverse = 1: the other way),
// 32 x 32 tiles of each z plane through shared memory
template <typename TI, typename TO>
__global__ void k_transpose_xy(int nx, int ny, int inverse, const TI *__restrict__ in, TO *__restrict__ out) {
    __shared__ TO tile[32][33];
    const int z = blockIdx.z;
    // tile of the source plane: rows r (slow index), columns c (fast index)
    const int R = inverse ? nx : ny, Cn = inverse ? ny : nx;
    const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    const size_t plane = (size_t)nx * ny * z;
    for (int dr = threadIdx.y; dr < 32; dr += blockDim.y) {
        const int r = r0 + dr, c = c0 + threadIdx.x;
        if (r < R && c < Cn) tile[dr][threadIdx.x] = (TO)in[plane + (size_t)r * Cn + c];
    }
    __syncthreads();
    for (int dc = threadIdx.y; dc < 32; dc += blockDim.y) {
        const int c = c0 + dc, r = r0 + threadIdx.x;
        if (r < R && c < Cn) out[plane + (size_t)c * R + r] = tile[threadIdx.x][dc];
    }
}

template <typename TI, typename TO>
void transpose_xy(const ms_system &s, bool inverse, const TI *in, TO *out, cudaStream_t st) {
    const int R = inverse ? s.nx : s.ny, Cn = inverse ? s.ny : s.nx;
    const dim3 grid((Cn + 31) / 32, (R + 31) / 32, s.nz), block(32, 8);
    KernelScope ks_(st, "transpose", (double)s.n * (sizeof(TI) + sizeof(TO)));
    k_transpose_xy<TI, TO><<<grid, block, 0, st>>>(s.nx, s.ny, inverse ? 1 : 0, in, out);
    MS_CHECK_LAUNCH();
}

// Lane layout of a line: G rows per warp (lanes per line L = 32 / G) and E
// cells per lane.  One row per warp: with G = 4 (8 lanes of 8 cells per line)
// the lanes' 128-byte strided reads of the packed coefficient line conflict on
// the same shared-memory banks, and the 60x220x85 sweep measured 0.9 ms FP32
// against 0.19 ms with G = 1.
struct LineShape {
    int G, E;
};
inline LineShape line_shape(int nx, bool) { return {1, nx <= 64 ? 2 : nx <= 128 ? 4 : 8}; }

template <typename T, typename TR>
size_t cluster_smem(int nx, int TK) {
    const LineShape ls = line_shape(nx, sizeof(T) == 4);
    const int RPC = TK * ls.G, LW = (32 / ls.G) * ls.E;
    return (size_t)RF * RPC * (nx * 4 + (sizeof(T) == 8 ? scan_table(32 / ls.G) : 0)) * sizeof(T) +
           (size_t)RF * RPC * rhs_win(nx, sizeof(TR)) * sizeof(TR) + (size_t)8 * NBX +
           (size_t)TK * NBX * LW * sizeof(T) + (size_t)8 * 2 * RF * RPC + (size_t)8 * 2 * NBX * TK;
}

template <typename T, typename TR, bool BWD, int E, int G>
cudaError_t launch_cluster_e(const ms_system &s, const int dims[3], int TK, int NK, int NC, const T *coef4,
                             const T *scanm, const TR *rhs, T *out, unsigned long long *tick,
                             unsigned long long *ring, cudaStream_t st, bool query_only, int *clusters) {
    auto kern = k_line_cluster<T, TR, BWD, E, G>;
    const size_t smem = cluster_smem<T, TR>(dims[0], TK);
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
    cfg.blockDim = dim3(32 * (TK + 1 + (NC > 1 ? 1 : 0)), 1, 1);   // + producer warp (+ relay warp)
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
    return cudaLaunchKernelEx(&cfg, kern, dims[0], dims[1], dims[2], TK, NC, coef4, scanm, rhs, out, tick, ring,
                              s.sync.p + 3);
}

// dims: (line length, lines walked per row, rows) of the sweep's layout
template <typename T, typename TR, bool BWD>
cudaError_t launch_cluster(const ms_system &s, const int dims[3], int TK, int NK, int NC, const T *coef4,
                           const T *scanm, const TR *rhs, T *out, unsigned long long *tick, unsigned long long *ring,
                           cudaStream_t st, bool query_only = false, int *clusters = nullptr) {
    switch (line_shape(dims[0], sizeof(T) == 4).E) {
        case 2:
            return launch_cluster_e<T, TR, BWD, 2, 1>(s, dims, TK, NK, NC, coef4, scanm, rhs, out, tick, ring, st,
                                                      query_only, clusters);
        case 4:
            return launch_cluster_e<T, TR, BWD, 4, 1>(s, dims, TK, NK, NC, coef4, scanm, rhs, out, tick, ring, st,
                                                      query_only, clusters);
        default:
            return launch_cluster_e<T, TR, BWD, 8, 1>(s, dims, TK, NK, NC, coef4, scanm, rhs, out, tick, ring, st,
                                                      query_only, clusters);
    }
}

inline void sweep_dims(const ms_system &s, int p, int dims[3]) {
    dims[0] = s.cl_T[p] ? s.ny : s.nx;
    dims[1] = s.cl_T[p] ? s.nx : s.ny;
    dims[2] = s.nz;
}

template <typename T, typename TR>
void cluster_apply(ms_system &s, const T *coef4, const T *scanm, const TR *r, T *y, T *z, cudaStream_t st) {
    const int64_t n = s.n;
    const int p = sizeof(T) == 8 ? 0 : 1;
    const double nl = (double)s.nnz_lower;
    int dims[3];
    sweep_dims(s, p, dims);
    const TR *rin = r;
    T *zout = z;
    if (s.cl_T[p]) {   // y-lines: sweeps on transposed copies of the vectors
        TR *rt = reinterpret_cast<TR *>(sizeof(TR) == 8 ? (void *)s.w_T64.p : (void *)s.w_T32.p);
        transpose_xy<TR, TR>(s, false, r, rt, st);
        rin = rt;
        zout = reinterpret_cast<T *>(sizeof(T) == 8 ? (void *)s.w_T64b.p : (void *)s.w_T32b.p);
    }
    if (s.sg_ok[p]) {   // lines in segments
        const long long lines = (long long)dims[1] * dims[2];
        {
            KernelScope ks_(st, sizeof(T) == 8 ? "ilu_fwd" : "ilu_fwd32",
                            nl * sizeof(T) + (double)n * (sizeof(TR) + sizeof(T)));
            seg_fwd<T, TR>(s, p, coef4, scanm, rin, y, st);
        }
        {
            KernelScope ks_(st, sizeof(T) == 8 ? "ilu_bwd" : "ilu_bwd32", nl * sizeof(T) + (double)n * 3 * sizeof(T));
            seg_bwd<T>(s, p, coef4 + (size_t)4 * n, scanm ? scanm + (size_t)lines * (seg_table_size(s) / 2 / lines) : nullptr,
                       y, zout, st);
        }
        if (s.cl_T[p]) transpose_xy<T, T>(s, true, zout, z, st);
        return;
    }
    {
        KernelScope ks_(st, sizeof(T) == 8 ? "ilu_fwd" : "ilu_fwd32", nl * sizeof(T) + (double)n * (sizeof(TR) + sizeof(T)));
        const cudaError_t e = launch_cluster<T, TR, false>(s, dims, s.cl_TK[p], s.cl_NK[p], s.cl_NC[p], coef4, scanm,
                                                           rin, y, s.cl_tick.p + p, s.cl_ring[p].p, st);
        MS_CUDA(e);
    }
    {
        KernelScope ks_(st, sizeof(T) == 8 ? "ilu_bwd" : "ilu_bwd32", nl * sizeof(T) + (double)n * 3 * sizeof(T));
        const long long lines = (long long)dims[1] * dims[2];
        const cudaError_t e = launch_cluster<T, T, true>(s, dims, s.cl_TK[p], s.cl_NK[p], s.cl_NC[p],
                                                         coef4 + (size_t)4 * n,
                                                         scanm ? scanm + lines * scan_table(32) : nullptr, y, zout,
                                                         s.cl_tick.p + p, s.cl_ring[p].p, st);
        MS_CUDA(e);
    }
    if (s.cl_T[p]) transpose_xy<T, T>(s, true, zout, z, st);
}

// Warps per CTA and cluster size for one precision and sweep layout dims: the
// cluster spans all k-rows (G per warp), at most 16 CTAs (more than 8 needs the
// non-portable size) of at most 16 warps and 32 rows, within the shared-memory
// limit, and the launch must be schedulable.  Fewer warps per CTA come first
// (one warp per SM sub-partition keeps each warp's dependency chain unshared).
template <typename T, typename TR>
bool plan_fits(ms_system &s, const int dims[3], int TK, int NK, int NC) {
    if (cluster_smem<T, TR>(dims[0], TK) > 220 * 1024 || cluster_smem<T, T>(dims[0], TK) > 220 * 1024) return false;
    int c1 = 0, c2 = 0;
    if (launch_cluster<T, TR, false>(s, dims, TK, NK, NC, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr,
                                     true, &c1) != cudaSuccess ||
        launch_cluster<T, T, true>(s, dims, TK, NK, NC, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr,
                                   true, &c2) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return c1 >= NC && c2 >= NC;
}

template <typename T, typename TR>
bool plan_precision(ms_system &s, int p, const int dims[3], bool sweep_only = false) {
    if (dims[0] > 256 || dims[1] < 1 || dims[2] < 1) return false;
    const LineShape ls = line_shape(dims[0], sizeof(T) == 4);
    const int warps = (dims[2] + ls.G - 1) / ls.G;
    if (sweep_only) {
        // a sweep layout only (the factorisation keeps its own): rows over
        // several clusters of the default warps per CTA
        const int tk = sizeof(T) == 8 ? kClusterTK64 : kClusterTK32;
        const int NKtot = (warps + tk - 1) / tk;
        const int NC = (NKtot + 15) / 16;
        const int NK = (NKtot + NC - 1) / NC;
        const int TK = (warps + NK * NC - 1) / (NK * NC);
        if (TK > 16 || TK * ls.G > 32 || !plan_fits<T, TR>(s, dims, TK, NK, NC)) return false;
        s.cl_TK[p] = TK;
        s.cl_NK[p] = NK;
        s.cl_NC[p] = NC;
        if (NC > 1) {
            s.cl_ring[p].alloc((size_t)(NC - 1) * dims[1] * (32 / ls.G) * ls.E * (sizeof(T) == 8 ? 2 : 1));
            s.cl_ring[p].zero(nullptr);
        }
        s.cl_tick.alloc(2);
        s.cl_tick.zero(nullptr);
        return true;
    }
    // one cluster over all rows (also the factorisation's layout)
    bool one = false;
    for (int C : {16, 8}) {
        const int TK = (warps + C - 1) / C;
        if (TK > 16 || TK * ls.G > 32) continue;
        const int NK = (warps + TK - 1) / TK;
        if (plan_fits<T, TR>(s, dims, TK, NK, 1)) {
            s.cl_TK[p] = s.cl_fTK[p] = TK;
            s.cl_NK[p] = s.cl_fNK[p] = NK;
            s.cl_NC[p] = 1;
            one = true;
            break;
        }
    }
    if (!one) return false;
    // rows over several clusters, so that fewer warps share an SM: TK warps per
    // CTA (MSGB_ILU_TK overrides the default for this precision)
    int tk = s.cl_TK[p] >= kClusterSplitFrom ? (sizeof(T) == 8 ? kClusterTK64 : kClusterTK32) : 0;
    if (const char *e = std::getenv("MSGB_ILU_TK")) tk = std::atoi(e);
    if (tk >= 1 && tk < s.cl_TK[p] && tk <= 15) {
        const int NKtot = (warps + tk - 1) / tk;
        const int NC = (NKtot + 15) / 16;
        const int NK = (NKtot + NC - 1) / NC;
        const int TK = (warps + NK * NC - 1) / (NK * NC);
        if (NC > 1 && plan_fits<T, TR>(s, dims, TK, NK, NC)) {
            s.cl_TK[p] = TK;
            s.cl_NK[p] = NK;
            s.cl_NC[p] = NC;
            s.cl_ring[p].alloc((size_t)(NC - 1) * dims[1] * (32 / ls.G) * ls.E * (sizeof(T) == 8 ? 2 : 1));
            s.cl_ring[p].zero(nullptr);
        }
    }
    s.cl_tick.alloc(2);
    s.cl_tick.zero(nullptr);
    return true;
}

}  // namespace

// Sweep layouts: x-lines (critical path ny + nz - 1 line steps) or y-lines on
// transposed vectors (critical path nx + nz - 1, 8 cells per lane when
// ny > 128).  FP32 takes y-lines when ny > nx: on the 60x220x85 benchmark grid
// its sweeps take 0.12 ms against 0.175 ms on x-lines.  FP64 keeps x-lines:
// a y-line step's offset scan is about 3 E + 4 dependent FP64 instructions
// per lane, and at this part's FP64 rate the longer steps cost more than the
// fewer steps save (0.41 against 0.32 ms).  MSGB_ILU_LINES=x keeps FP32 on
// x-lines, =yy puts both precisions on y-lines.
void plan_ilu_cluster(ms_system &s) {
    const char *e = std::getenv("MSGB_ILU_LINES");
    const std::string lines_env = e ? std::string(e) : std::string();
    const bool want_y = lines_env != "x";                            // FP32 sweeps on y-lines
    const bool want_y64 = lines_env == "y64" || lines_env == "yy";  // FP64 sweeps on y-lines
    int d[3] = {s.nx, s.ny, s.nz};
    s.cl_T[0] = false;
    s.cl_ok[0] = plan_precision<double, double>(s, 0, d);   // also the factorisation's layout
    if (want_y64 && s.cl_ok[0] && s.ny > s.nx && s.ny <= 256) {
        const int fTK = s.cl_fTK[0], fNK = s.cl_fNK[0];
        int dt[3] = {s.ny, s.nx, s.nz};
        if (plan_precision<double, double>(s, 0, dt, true)) {
            s.cl_T[0] = true;
            s.w_T64.alloc(s.n);
            s.w_T64b.alloc(s.n);
        } else {
            s.cl_ok[0] = plan_precision<double, double>(s, 0, d);
        }
        s.cl_fTK[0] = fTK;   // the factorisation runs on x-lines
        s.cl_fNK[0] = fNK;
    }
    s.cl_T[1] = want_y && s.ny > s.nx && s.ny <= 256;
    if (s.cl_T[1]) {
        int dt[3] = {s.ny, s.nx, s.nz};
        s.cl_ok[1] = plan_precision<float, double>(s, 1, dt) && plan_precision<float, float>(s, 1, dt);
        if (!s.cl_ok[1]) s.cl_T[1] = false;
    }
    if (!s.cl_T[1]) s.cl_ok[1] = plan_precision<float, double>(s, 1, d) && plan_precision<float, float>(s, 1, d);
    // segmented sweeps where their layout fits (they choose the walked direction)
    for (int p = 0; p < 2; ++p)
        if (s.cl_ok[p]) plan_ilu_seg(s, p);
    if (s.cl_T[0]) {
        s.w_T64.alloc(s.n);
        s.w_T64b.alloc(s.n);
    }
    if (s.cl_T[1] && s.cl_ok[1]) {
        s.w_T64.alloc(s.n);
        s.w_T32.alloc(s.n);
        s.w_T64b.alloc(s.n);
        s.w_T32b.alloc(s.n);
    }
}

// Structured ILU(0) factors (FP64) with the cluster line pipeline; false when
// the layout cannot be launched (the caller uses the level-ordered kernel).
bool launch_ilu_factor_cluster(ms_system &s, cudaStream_t st) {
    if (!s.structured || !s.cl_ok[0] || s.nx > 256) return false;
    const int E = s.nx <= 64 ? 2 : s.nx <= 128 ? 4 : 8;
    const int TK = s.cl_fTK[0], NK = s.cl_fNK[0];   // one cluster over all rows
    const int LW = 32 * E;
    const size_t smem = (size_t)RF * TK * s.nx * 32 + (size_t)TK * NBX * LW * 8 + (size_t)8 * 2 * (RF + NBX) * TK;
    if (smem > 220 * 1024) return false;
    s.w_fac4.alloc((size_t)4 * s.n);
    const int g = (s.n + 255) / 256;
    KernelScope ks_(st, "ilu_factor", (double)s.n * (8 + 8 + 8) + (double)s.W * s.n * (4 + 8 + 8));
    k_pack_factor<<<g, 256, 0, st>>>(s.n, s.dir_slot.p, s.col.p, s.off_p.p, s.diag.p, s.w_fac4.p);
    MS_CHECK_LAUNCH();
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(NK, 1, 1);
    cfg.blockDim = dim3(32 * (TK + 1), 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = NK;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t e = cudaSuccess;
    auto go = [&](auto kern) {
        static size_t smem_set = 0;
        e = raise_smem_limit(kern, smem, smem_set);
        if (e == cudaSuccess && NK > 8) e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e == cudaSuccess)
            e = cudaLaunchKernelEx(&cfg, kern, s.nx, s.ny, s.nz, TK, (const double *)s.w_fac4.p, s.dinv64.p,
                                   s.sync.p + 3);
    };
    if (E == 2) go(k_factor_cluster<2>);
    else if (E == 4) go(k_factor_cluster<4>);
    else go(k_factor_cluster<8>);
    if (e != cudaSuccess) {   // not launchable here: the level-ordered factorisation runs instead
        cudaGetLastError();
        return false;
    }
    k_factor_finish<<<g, 256, 0, st>>>(s.n, s.W, s.col.p, s.off_p.p, s.dinv64.p, s.lu64.p);
    MS_CHECK_LAUNCH();
    return true;
}

template <typename T>
void pack_scan_tables(ms_system &s, int p, const T *coef4, T *table, cudaStream_t st) {
    int dims[3];
    sweep_dims(s, p, dims);
    const long long lines = (long long)dims[1] * dims[2];
    const int g = (int)((lines + 7) / 8);
    const int E = line_shape(dims[0], sizeof(T) == 4).E;
    for (int dir = 0; dir < 2; ++dir) {
        const T *c = coef4 + (size_t)dir * 4 * s.n;
        T *o = table + (size_t)dir * lines * scan_table(32);
        if (dir == 0) {
            if (E == 2) k_pack_scan<T, false, 2><<<g, 256, 0, st>>>(dims[0], lines, c, o);
            else if (E == 4) k_pack_scan<T, false, 4><<<g, 256, 0, st>>>(dims[0], lines, c, o);
            else k_pack_scan<T, false, 8><<<g, 256, 0, st>>>(dims[0], lines, c, o);
        } else {
            if (E == 2) k_pack_scan<T, true, 2><<<g, 256, 0, st>>>(dims[0], lines, c, o);
            else if (E == 4) k_pack_scan<T, true, 4><<<g, 256, 0, st>>>(dims[0], lines, c, o);
            else k_pack_scan<T, true, 8><<<g, 256, 0, st>>>(dims[0], lines, c, o);
        }
    }
}

void launch_ilu_pack_coef4(ms_system &s, bool fp32, cudaStream_t st) {
    const int g = (s.n + 255) / 256;
    const size_t tab = (size_t)2 * s.n / (size_t)std::max(1, fp32 ? (s.cl_T[1] ? s.ny : s.nx) : (s.cl_T[0] ? s.ny : s.nx)) *
                       scan_table(32);
    if (fp32) {
        s.coef4_32.alloc((size_t)8 * s.n);
        k_pack_coef4<float><<<g, 256, 0, st>>>(s.n, s.nx, s.ny, s.cl_T[1] ? 1 : 0, s.dcoef32.p, s.dinv32.p,
                                               s.coef4_32.p);

    } else {
        s.coef4_64.alloc((size_t)8 * s.n);
        k_pack_coef4<double><<<g, 256, 0, st>>>(s.n, s.nx, s.ny, s.cl_T[0] ? 1 : 0, s.dcoef64.p, s.dinv64.p,
                                                s.coef4_64.p);
        if (s.sg_ok[0]) {
            s.scan_64.alloc(seg_table_size(s));
            pack_seg_tables(s, s.coef4_64.p, s.scan_64.p, st);
        } else {
            s.scan_64.alloc(tab);
            pack_scan_tables<double>(s, 0, s.coef4_64.p, s.scan_64.p, st);
        }
    }
    MS_CHECK_LAUNCH();
}

void launch_ilu_cluster64(ms_system &s, const double *r, double *y, double *z, cudaStream_t st) {
    cluster_apply<double, double>(s, s.coef4_64.p, s.scan_64.p, r, y, z, st);
}

void launch_ilu_cluster32(ms_system &s, const double *r, float *y, float *z, cudaStream_t st) {
    cluster_apply<float, double>(s, s.coef4_32.p, nullptr, r, y, z, st);
}

void launch_ilu_cluster32f(ms_system &s, const float *r, float *y, float *z, cudaStream_t st) {
    cluster_apply<float, float>(s, s.coef4_32.p, nullptr, r, y, z, st);
}

}  // namespace msgb
