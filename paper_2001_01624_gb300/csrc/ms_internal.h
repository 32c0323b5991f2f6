// Internal declarations of the GB300 multiscale pressure solver library.
// Host orchestration (ms_api.cu), host analysis (ms_analysis.cpp) and the
// kernel translation units share these structures.  Nothing here is part of
// the public ABI (include/ms.h).
#pragma once

#include <cuda_runtime.h>

#include <cmath>
#include <stdint.h>

#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "ms.h"

namespace msgb {

// ----------------------------------------------------------------- errors
struct Error {
    ms_status status;
    std::string what;
};

#define MS_CUDA(call)                                                                        \
    do {                                                                                     \
        cudaError_t e__ = (call);                                                            \
        if (e__ != cudaSuccess)                                                              \
            throw ::msgb::Error{e__ == cudaErrorMemoryAllocation ? MS_ERR_OOM : MS_ERR_CUDA, \
                                std::string(#call) + ": " + cudaGetErrorString(e__)};        \
    } while (0)

#define MS_REQUIRE(cond, st, msg)                           \
    do {                                                    \
        if (!(cond)) throw ::msgb::Error{(st), (msg)};      \
    } while (0)

#define MS_CHECK_LAUNCH() MS_CUDA(cudaGetLastError())

// ------------------------------------------------------------ device buffer
// Every device allocation of the library goes through DBuf: this records its
// bytes for the calling host thread and counts it for the process
// (ms_allocation_stats).
void note_device_alloc(size_t bytes);

template <typename T>
struct DBuf {
    T *p = nullptr;
    size_t n = 0;
    DBuf() = default;
    DBuf(const DBuf &) = delete;
    DBuf &operator=(const DBuf &) = delete;
    ~DBuf() { release(); }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
    }
    // Grow-only: keeps the buffer when it already holds `count` elements.
    void alloc(size_t count) {
        if (count <= n && p) return;
        release();
        if (count == 0) return;
        MS_CUDA(cudaMalloc(&p, count * sizeof(T)));
        n = count;
        note_device_alloc(count * sizeof(T));
    }
    void upload(const std::vector<T> &h, cudaStream_t s) {
        alloc(h.size());
        if (!h.empty()) MS_CUDA(cudaMemcpyAsync(p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, s));
    }
    void zero(cudaStream_t s) {
        if (n) MS_CUDA(cudaMemsetAsync(p, 0, n * sizeof(T), s));
    }
};

// Pinned host scratch for small device->host reads (norms, flags).
struct HostScratch {
    void *p = nullptr;
    size_t bytes = 0;
    ~HostScratch() {
        if (p) cudaFreeHost(p);
    }
    void *get(size_t b) {
        if (b > bytes) {
            if (p) cudaFreeHost(p);
            p = nullptr;
            MS_CUDA(cudaMallocHost(&p, b));
            bytes = b;
        }
        return p;
    }
};

constexpr int kSlotPad = 0x7fffffff;   // padding block id in basis slot lists (sorts last)

// Device-side synchronisation words of the level-ordered sweeps:
// [0] sweep counter, [1] ticket (a CTA's, or a warp's in the segment sweeps), [2] CTAs done,
// [3] error flags, [4] bound of one device-side wait of this system's sweeps in
// microseconds (0: kDefaultWaitNs).
constexpr int kSyncWords = 8;
constexpr unsigned long long kDefaultWaitNs = 2000000000ull;

#ifdef __CUDACC__
// Bound of a device-side wait, read (only once a wait is already long) from
// the word after a system's error word `errw` (sync word 3).
__device__ __forceinline__ unsigned long long wait_limit_ns(const int *errw) {
    const int us = *((volatile const int *)(errw + 1));
    return us > 0 ? (unsigned long long)us * 1000ull : kDefaultWaitNs;
}
#endif
constexpr int kSegMax = 64;        // rows per segment of the segment sweeps (2 per lane)
constexpr int kSegPlanMax = 256;   // longest run the host analysis entry point accepts
constexpr int kSegMaxKG = 8;       // couplings per row leaving its segment, per direction
constexpr int kErrTimeout = 1;
constexpr int kErrSingular = 2;
constexpr int kErrNaN = 4;

// Kernel tracing scope: counts the launch made inside it and, when tracing is
// enabled, brackets it with CUDA events on its stream.
class KernelScope {
  public:
    KernelScope(cudaStream_t st, const char *name, double bytes);
    ~KernelScope();
    KernelScope(const KernelScope &) = delete;
    KernelScope &operator=(const KernelScope &) = delete;

  private:
    cudaStream_t st_;
    const char *name_;
    double bytes_;
    cudaEvent_t a_ = nullptr;
};
// Raise a kernel's dynamic shared-memory limit to at least `bytes`; `cur`
// (one per kernel) remembers the limit set.  Thread-safe, never lowers it.
std::mutex &attr_mutex();
template <typename K>
cudaError_t raise_smem_limit(K kern, size_t bytes, size_t &cur) {
    std::lock_guard<std::mutex> g(attr_mutex());
    if (bytes <= cur) return cudaSuccess;
    const cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) cur = bytes;
    return e;
}

void profile_enable(bool on);
// Add algorithmic bytes to the latest traced launch of kernel family `name`
// (for a launch whose work is known only after it ran).
void profile_add_bytes(const char *name, double bytes);
bool profile_enabled();
// graph capture: list the launches captured (counted once at capture), then
// add them again per extra replay of the graph
void profile_record_begin();
std::vector<std::string> profile_record_end();
void profile_add_launches(const std::vector<std::string> &names, int64_t times);
void profile_reset();
int profile_read(ms_kernel_stat *out, int cap, int64_t *total);

// Device scratch of the batched basis smoothing (k_msrsb_batch): member
// descriptors, the work queue and its ring of slots, per-member tile counters
// and iteration-control blocks.
struct BatchScratch {
    DBuf<unsigned char> jobs;
    DBuf<unsigned long long> queue, slots, ctl;
    DBuf<int> done;
};

}  // namespace msgb

// ------------------------------------------------------------------ handles
struct ms_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t capture = nullptr;   // private stream that graphs are captured on (never executes)
    bool owns_stream = false;         // worker contexts of batched solves own their stream
    std::vector<std::unique_ptr<ms_ctx>> workers;
    ~ms_ctx() {
        workers.clear();
        if (capture) cudaStreamDestroy(capture);
        if (owns_stream && stream) cudaStreamDestroy(stream);
    }
    int sm_count = 0;
    std::string err;
    msgb::HostScratch pinned;
    // batched smoothing: cells per work item and resident blocks per SM
    // (ms_set_batch_tuning), and its device scratch
    int batch_tile = 1024, batch_ctas_per_sm = 4;
    std::unique_ptr<msgb::BatchScratch> batch;
};

// Host-side analysis products of a grid (built once per grid).
struct ms_system {
    int device = 0;
    int nx = 0, ny = 0, nz = 0;
    double dx = 0, dy = 0, dz = 0;
    int n = 0;       // active cells
    int ref = 0;     // pinned reference cell
    std::vector<int> cells;   // grid index of each active cell
    std::vector<int> g2a;     // active index of each grid cell (-1 inactive)

    // two-point connections
    int nf = 0;
    std::vector<int> h_fa, h_fb;          // active indices
    msgb::DBuf<int> f_ga, f_gb;           // grid indices (permeability lookup)
    msgb::DBuf<int> f_a, f_b;             // active indices
    msgb::DBuf<int8_t> f_axis;
    msgb::DBuf<double> f_mult;
    msgb::DBuf<double> f_T;               // transmissibility with mobility
    // row -> incident connections (for deterministic row assembly)
    msgb::DBuf<int> rf_ptr, rf_face;
    msgb::DBuf<uint8_t> rf_slot;

    // ELL storage of A: slot w of row i at [w*n + i]; padding col = i, val = 0
    int W = 0;
    std::vector<int> h_col;
    msgb::DBuf<int> col;
    msgb::DBuf<double> off_u, off_p, diag;    // unpinned / pinned off-diagonals, diagonal
    msgb::DBuf<float> off_p32, diag32;        // single-precision copies (mixed solve)
    msgb::DBuf<float> off_u32;                // single-precision unpinned (mixed basis)

    // natural-order wavefront levels, each padded to a multiple of 32 rows
    int n_levels = 0;
    int ntot = 0;
    int64_t nnz_lower = 0;   // structural entries below / above the diagonal

    // structured (Cartesian, all active, no non-neighbour connection) grids:
    // slot of each direction (-x,-y,-z,+x,+y,+z) per cell, -1 when absent, and
    // the tiled-wavefront ILU(0) sweep data
    bool structured = false;
    msgb::DBuf<int8_t> dir_slot;              // [d*n + i]
    int TJ = 0, TK = 0, NJ = 0, NK = 0;
    msgb::DBuf<int> tile_order;
    msgb::DBuf<unsigned long long> face_j, face_k;   // tagged tile-face exchange buffers
    msgb::DBuf<unsigned long long> tile_progress;    // tagged per-tile progress hints
    // line-scan sweeps: TK warps per CTA walk TJ x TK tiles of x-lines
    int LTJ = 0, LTK = 0, LNJ = 0, LNK = 0;
    // sweep kernel per precision ([0] FP64, [1] FP32): 0 level-ordered, 1 pencil tiles,
    // 2 line scan over CTA tiles, 3 line scan pipelined across one cluster,
    // 4 level-synchronous (cooperative), 5 segment dataflow
    int ilu_kind[2] = {0, 0};
    // cluster line scan per precision: feasible, rows per CTA, CTAs (= cluster size)
    bool cl_ok[2] = {false, false};
    bool cl_T[2] = {false, false};            // y-lines on transposed vectors (x fastest -> y fastest)
    msgb::DBuf<double> w_T64, w_T64b;         // transposed right-hand side / result
    msgb::DBuf<float> w_T32, w_T32b;
    msgb::DBuf<double> w_fac4;                // structured factorisation input (c_x, c_y, c_z, A_ii) per cell
    int cl_TK[2] = {0, 0}, cl_NK[2] = {0, 0};
    int cl_NC[2] = {1, 1};                    // clusters the sweep's rows span
    int cl_fTK[2] = {0, 0}, cl_fNK[2] = {0, 0};   // single-cluster layout (factorisation)
    msgb::DBuf<unsigned long long> cl_tick;   // cluster tickets per precision
    msgb::DBuf<unsigned long long> cl_ring[2];  // lines crossing cluster boundaries (tagged words)
    // segmented line sweeps (lines cut into 64-cell segments, one warp each)
    bool sg_ok[2] = {false, false};
    int sg_S[2] = {1, 1}, sg_PP[2] = {1, 1}, sg_TK[2] = {0, 0}, sg_NK[2] = {0, 0}, sg_NC[2] = {1, 1};
    msgb::DBuf<unsigned long long> sg_tick;   // cluster tickets per precision
    msgb::DBuf<unsigned long long> sg_ring[2];
    msgb::DBuf<double> coef4_64;              // [2][n][4]: (Lx, Ly, Lz, 0), (Ux/d, Uy/d, Uz/d, 1/d) per cell, d = U_ii
    msgb::DBuf<float> coef4_32;
    msgb::DBuf<double> scan_64;               // [2][lines][levels][32]: scan multipliers of each FP64 sweep line
    msgb::DBuf<int> line_order;
    msgb::DBuf<unsigned long long> lface_j, lface_k, line_progress;
    msgb::DBuf<double> dcoef64;               // [6*n]: L(-x,-y,-z), U(+x,+y,+z)
    msgb::DBuf<float> dcoef32;
    msgb::DBuf<int> lperm;
    msgb::DBuf<int> lev_off;                  // [n_levels + 1] level offsets into lperm
    msgb::DBuf<unsigned long long> lev_bar;   // grid barrier of the level-synchronous sweeps (counter, base)
    // segment sweeps (any grid): runs of consecutive rows chained by their (i-1, i)
    // couplings; per direction a hand-out order by wavefront level
    int n_seg = 0;
    int seg_width = 0;                        // most segments on one level (either direction)
    int seg_kg[2] = {0, 0};                   // couplings per row leaving its segment: lower, upper
    msgb::DBuf<int> seg_off;                  // [n_seg + 1] first row of each segment
    msgb::DBuf<int> seg_id;                   // [n] segment of each row
    msgb::DBuf<int> seg_ord;                  // [2 n_seg] forward order, backward order
    msgb::DBuf<unsigned long long> seg_tag;   // [2 n] results as tagged words (sweep counter | value bits)
    msgb::DBuf<int> seg_gc;                   // [(kg0 + kg1) n] columns of the leaving couplings, -1 padding
    msgb::DBuf<double> seg_v64;               // [(2 + kg0 + kg1) n] chain a (fwd, bwd), coupling values
    msgb::DBuf<float> seg_v32;

    // ILU(0) factors on A's pattern (L in lower slots, U in upper slots)
    bool ilu64_valid = false, ilu32_valid = false;
    msgb::DBuf<double> lu64, dinv64;
    msgb::DBuf<float> lu32, dinv32;

    // sweep synchronisation
    msgb::DBuf<int> flags;
    msgb::DBuf<int> sync;

    bool assembled = false;
    bool pinned = true;         // reference cell pinned (TPFA); false for a CPR pressure system
    bool symmetric = true;      // TPFA matrices are; CPR pressure systems are not
    msgb::DBuf<double> w_cpr;   // CPR per-cell state functions and accumulation terms
    uint64_t assembly_id = 0;   // bumped by every assembly

    // solve workspace (grown on demand)
    msgb::DBuf<double> w_q, w_x, w_r, w_z, w_xprev, w_d, w_xc, w_rc, w_part;
    msgb::DBuf<float> w_y32, w_z32, w_r32, w_d32, w_xc32, w_rin32;
    msgb::DBuf<double> w_y;
    msgb::DBuf<double> w_kry;                 // GMRES: V [(m+1) n], Z [m n], w, q copy; dot scratch
    msgb::DBuf<double> w_kred, w_kh;
    msgb::DBuf<double> w_kgd;                 // graph-driven GMRES: Hessenberg, rotations, g, y, history
    msgb::DBuf<int> w_kgi;                    //   and its counters
    msgb::DBuf<unsigned long long> w_kgh;     //   and the handles of its conditional steps
    msgb::DBuf<unsigned int> w_kcnt;
    msgb::DBuf<double> w_tu, w_ts, w_tq;      // transport: face fluxes, saturation buffer, sources
    msgb::DBuf<double> w_tc;                  //   upstream weights of a step: src [n], dg [n], inflow fluxes [W][n]
    msgb::DBuf<int> w_tci;                    //   inflow counts [n], upstream cells [W][n]
    msgb::DBuf<unsigned long long> w_tbar;    //   grid barrier of the one-launch substeps
    bool tbar_ready = false;
    int rf_max = 0;                           // most faces of one cell
    msgb::DBuf<double> w_red;                 // reduction partials
    msgb::DBuf<unsigned int> w_cnt;           // reduction counters
    msgb::DBuf<unsigned long long> w_max;     // max reductions
    msgb::DBuf<int> w_i0, w_i1, w_i2;         // integer scratch (partitions)
};

struct ms_basis {
    int M = 0;
    int B = 0;                  // slots per cell (max overlap)
    int64_t nnz = 0;
    int rule = 0;
    int precision = 0;
    double omega = 2.0 / 3.0, tol = 1e-3;
    int max_iter = 500;
    int iters = 0;
    double last_inc = 0;
    uint64_t assembly_id = 0;   // assembly the values were smoothed with
    std::vector<int> h_part;
    msgb::DBuf<int> part;       // block of each cell
    // cell-major slots: [s*n + i], block ids ascending, padding kSlotPad
    msgb::DBuf<int> pid;
    msgb::DBuf<double> pval, pval_tmp;
    msgb::DBuf<float> pval32, pval32_tmp;
    msgb::DBuf<double> od64;             // omega / A_ii for the current smoothing run
    msgb::DBuf<double> pre_c64, pre_w64; // prescaled rows of that run: 1 - omega, -(omega / A_ii) A_ij (FP64)
    msgb::DBuf<float> od32;
    // column view (CSC)
    msgb::DBuf<int> cptr, ccell, csrc;
    msgb::DBuf<double> cval;
    msgb::DBuf<float> cval32;
    msgb::DBuf<unsigned char> is_home;   // 1 where the slot's block is the cell's own block
    // neighbour slot maps (B <= 8): for slot w of A's row i, 4 bits per basis
    // slot s of cell i = slot of the same block in neighbour col[w][i] (15: none)
    bool has_map = false;
    msgb::DBuf<unsigned> nmap;
    msgb::DBuf<unsigned char> nslots;    // number of real slots of each cell
    // cells in the order the FP64 smoothing takes them: within each window of
    // kOrderWin cells, by descending slot count (stable), so that the lanes
    // of a warp mostly share a slot count (a multiply-add that only some
    // lanes need still takes the FP64 pipe for all 32)
    msgb::DBuf<int> order;
    // column chunks: each support cut into pieces of at most kColChunk entries
    // (chunk c covers entries [ch_beg[c], min(ch_beg[c] + kColChunk, cptr[j+1]))
    // of column j = ch_col[c]; column j owns chunks [ch_ptr[j], ch_ptr[j+1]));
    // column sums are taken over chunks, then over a column's chunks in order
    std::vector<int> h_cptr;
    int n_chunks = 0;
    msgb::DBuf<int> ch_beg, ch_col, ch_ptr;
    msgb::DBuf<double> ch_part;          // per-chunk partial sums
    msgb::DBuf<unsigned> ch_cnt;         // per-column arrival counters (back to 0 after each use)
};
constexpr int kColChunk = 1024;
constexpr int kOrderWin = 4096;   // window of the smoothing's cell order (1024 threads x 4 cells)

struct ms_coarse {
    int M = 0;
    int precision = 0;
    const ms_basis *basis = nullptr;
    msgb::DBuf<double> Ac;       // M*M row-major, Galerkin operator
    msgb::DBuf<double> inv64;    // M*M inverse (FP64)
    msgb::DBuf<float> inv32;     // M*M inverse (FP32, mixed)
    bool use64 = false;          // mixed stage whose FP32 inverse was too inaccurate: FP64 inverse used
    double inv32_error = 0.0;    // ||inv32 A_c v - v|| / ||v|| on a test vector
    int refine_steps = 2;        // FP64 refinement steps of a mixed stage's coarse solve
    int sp_w = 0;                // ELL copy of A_c for the refinement residuals (0: dense)
    msgb::DBuf<int> sp_col;
    msgb::DBuf<double> sp_val;
    int coop_blocks = 0;         // blocks of the one-launch refinement (0: kernel chain)
    msgb::DBuf<int> refine_err;  // its grid-barrier error word
    msgb::DBuf<double> work64;   // factor workspace
    msgb::DBuf<float> work32;
    // Galerkin column chunks (size gchunk, chosen so the partial rows of split
    // columns fit in memory): chunk beg / column / slot of its partial row (-1:
    // the column is a single chunk)
    int gchunk = 0, n_gchunks = 0;
    msgb::DBuf<int> gch_beg, gch_col, gch_ptr, gch_slot;
    msgb::DBuf<double> gpart;
    msgb::DBuf<unsigned> gcnt;
    // Galerkin scratch: cell-major (A P) lists
    int WAP = 0;
    msgb::DBuf<int> apid;
    msgb::DBuf<double> apval;
    // restriction: MS_RESTRICT_GALERKIN (R = P^T) or MS_RESTRICT_FV (R sums
    // each block's cells: block member lists, ascending cells, with their
    // column chunks; unit weights)
    int restriction = 0;
    bool nonsym = false;        // A_c not symmetric (finite volume, or a non-symmetric A): Gauss-Jordan inverse
    std::vector<int> fv_h_cptr;
    msgb::DBuf<int> fv_cptr, fv_ccell, fv_ch_beg, fv_ch_col, fv_ch_ptr;
    msgb::DBuf<double> fv_ch_part;
    msgb::DBuf<unsigned> fv_ch_cnt;
    int fv_n_chunks = 0;
    // Gauss-Jordan scratch (finite-volume stages)
    msgb::DBuf<unsigned long long> gj_cand_v;   // pivot candidates as integer keys of |a_ik|
    msgb::DBuf<int> gj_cand_i, gj_piv, gj_idx;
    msgb::DBuf<unsigned long long> gj_bar;
};

namespace msgb {
// Column view of a restriction operator (row j of R = entries [cptr[j],
// cptr[j+1]) over cells ccell with weights cval / cval32, or unit weights
// when they are null), cut into column chunks for deterministic sums.
struct RestrictView {
    int M = 0;
    int64_t nnz = 0;
    int n_chunks = 0;
    const int *ch_beg = nullptr, *ch_col = nullptr, *ch_ptr = nullptr, *cptr = nullptr, *ccell = nullptr;
    const double *cval = nullptr;
    const float *cval32 = nullptr;
    double *ch_part = nullptr;
    unsigned *ch_cnt = nullptr;
};
RestrictView restrict_view(const ms_coarse &c);
}  // namespace msgb

namespace msgb {

// ---------------------------------------------------------------- analysis
void analyse_grid(ms_system &s, const ms_grid &g);
// segments of the segment ILU(0) sweeps (host analysis of a row pattern)
struct SegmentPlan {
    std::vector<int> off, sid, ord;   // segment starts (+ n), segment of each row, hand-out orders (fwd, bwd)
    int kg[2] = {0, 0};               // most couplings of one row leaving its segment: lower, higher rows
    int width = 0;                    // most segments on one level
    bool fits = false;                // kg within what the sweeps take
};
void segment_plan(int n, const std::vector<int> &nb, const std::vector<int> &deg, const std::vector<int> &rowlen,
                  int max_len, SegmentPlan &sp);
int partition_cartesian(const ms_system &s, int bx, int by, int bz, std::vector<int> &part);
// Support patterns for a partition; fills per-block sorted cell lists.
void analyse_supports(const ms_system &s, const std::vector<int> &part, int M, int rule, int bx, int by, int bz,
                      std::vector<int> &cptr, std::vector<int> &ccell);
// Cell-major slot layout from the column view.
void slot_layout(const ms_system &s, const std::vector<int> &part, int M, const std::vector<int> &cptr,
                 const std::vector<int> &ccell, int &B, std::vector<int> &pid, std::vector<int> &csrc,
                 std::vector<unsigned char> &is_home);

// ------------------------------------------------------------------ kernels
// assembly
void launch_face_trans(ms_system &s, const double *perm, const double *mob, const double *pprev, cudaStream_t st);
void launch_row_assemble(ms_system &s, cudaStream_t st);
void launch_check_perm(const double *perm, int64_t count, int *flag, cudaStream_t st);
// sparse
void launch_spmv(const ms_system &s, const double *x, double *y, cudaStream_t st);
void launch_residual(const ms_system &s, const double *q, const double *x, double *r, double *red,
                     unsigned int *cnt, double *norm_out, cudaStream_t st, float *r32 = nullptr);
void launch_residual_update(const ms_system &s, double *r, double *x, const double *z, cudaStream_t st);
void launch_residual_update32(const ms_system &s, const double *r, float *r32, double *x, const float *z,
                              cudaStream_t st);
void launch_jacobi(const ms_system &s, const double *r, double *z, double omega, cudaStream_t st);
void launch_jacobi32(const ms_system &s, const double *r, float *z, float omega, cudaStream_t st);
void launch_norm2(const double *v, int n, double *red, unsigned int *cnt, double *out, cudaStream_t st);
int multidot_blocks(int n);
// two-phase transport; fl = (mu_w, mu_o, n_w, n_o, s_wc, s_or)
double frac_flow_max_slope(double mu_w, double mu_o, double n_w, double n_o, double s_wc, double s_or);
void launch_total_mobility(int n, const double fl[6], const double *S, double *lam, cudaStream_t st);
void launch_face_flux(const ms_system &s, const double *p, double *u, cudaStream_t st);
void launch_outflow_limit(const ms_system &s, const double *u, const double *q, double pore_volume,
                          unsigned long long *min_bits, cudaStream_t st);
// one transport step's upstream weights (fluxes u, sources q fixed over its substeps)
void launch_transport_coef(ms_system &s, const double *u, const double *q, cudaStream_t st);
// nsub substeps from S (in place), fractional flows through fwa / fwb; one
// cooperative launch with a grid barrier per substep (MSGB_TRANSPORT_COOP=0:
// one launch per substep)
void launch_transport_run(ms_system &s, const double fl[6], int nsub, double h_over_pv, double *S, double *fwa,
                          double *fwb, cudaStream_t st);
void launch_multidot(int n, int k, const double *V, const double *w, double *red, unsigned int *cnt, double *h,
                     cudaStream_t st);
// the same, then ||y||_2 into norm_out (red: at least ceil(n / 256) partials)
void launch_multiaxpy_norm(int n, int k, const double *V, const double *c, double sign, double *y, double *red,
                           unsigned int *cnt, double *norm_out, cudaStream_t st);
void launch_multiaxpy(int n, int k, const double *V, const double *c, double sign, double *y, cudaStream_t st,
                      const int *kdev = nullptr);
// GMRES state on the device (graph-driven solves): Hessenberg matrix
// (m+1) x m, rotations, rotated right-hand side, solution of the small
// system, 1/norm for the next basis vector, and counters.
// One Arnoldi step's update of the GMRES least-squares problem: column j of
// the Hessenberg matrix H (row stride m) takes the j earlier Givens
// rotations, rotation j is made to zero H(j+1, j), and g takes it.  Every
// product that meets a sum is an explicit fma, so the host-driven loop and
// the device graph round identically.
__host__ __device__ inline void gmres_givens(double *H, int m, int j, double *cs, double *sn, double *g) {
    for (int i = 0; i < j; ++i) {
        const double a = H[(size_t)i * m + j], b = H[(size_t)(i + 1) * m + j];
        H[(size_t)i * m + j] = fma(cs[i], a, sn[i] * b);
        H[(size_t)(i + 1) * m + j] = fma(cs[i], b, -(sn[i] * a));
    }
    const double a = H[(size_t)j * m + j], b = H[(size_t)(j + 1) * m + j];
    const double rho = sqrt(fma(a, a, b * b));
    cs[j] = rho > 0 ? a / rho : 1.0;
    sn[j] = rho > 0 ? b / rho : 0.0;
    H[(size_t)j * m + j] = rho;
    H[(size_t)(j + 1) * m + j] = 0.0;
    g[j + 1] = -(sn[j] * g[j]);
    g[j] = cs[j] * g[j];
}

// H(0:k, 0:k) y = g(0:k), H upper triangular after the rotations
__host__ __device__ inline void gmres_back_solve(const double *H, int m, int k, const double *g, double *y) {
    for (int i = k - 1; i >= 0; --i) {
        double acc = g[i];
        for (int l = i + 1; l < k; ++l) acc = fma(-H[(size_t)i * m + l], y[l], acc);
        y[i] = acc / H[(size_t)i * m + i];
    }
}

struct GmresDev {
    double *H, *cs, *sn, *g, *y, *scal, *res, *hist;
    int *k, *it, *stop, *err, *restarts;   // restarts: bounds the while loop on its own
    int m, max_iter;
    double nq, tol;
};
void launch_scale_dev(int n, const double *x, const double *a, double *y, cudaStream_t st);
// steps: device array of the m conditional handles of the Arnoldi steps (a
// handle steers exactly one conditional node)
void launch_gmres_begin(const GmresDev &G, const double *beta_norm, const cudaGraphConditionalHandle *steps,
                        cudaStream_t st);
void launch_gmres_step(const GmresDev &G, int j, const double *h1, const double *h2, const double *hn,
                       const cudaGraphConditionalHandle *steps, cudaStream_t st);
void launch_gmres_solve(const GmresDev &G, cudaStream_t st);
void launch_gmres_restart(const GmresDev &G, const double *beta_norm, cudaGraphConditionalHandle outer,
                          cudaStream_t st);
void launch_scale(int n, const double *x, double a, double *y, cudaStream_t st);
void launch_cycle_control(const double *norms, double tol, int max_iter, int *ctl_it, double *ctl_res, double *hist,
                          cudaGraphConditionalHandle handle, cudaStream_t st);
void launch_sub(const double *a, const double *b, double *c, int n, cudaStream_t st);
void launch_scatter_zero(double *v, int idx, cudaStream_t st);
void build_column_chunks(const std::vector<int> &cptr, int M, int C, std::vector<int> &beg, std::vector<int> &col,
                         std::vector<int> &ptr, std::vector<int> *slot, int *multi);
void launch_restrict(const RestrictView &v, const double *r, double *d, cudaStream_t st);
void launch_restrict32(const RestrictView &v, const float *r, float *d, cudaStream_t st);
void launch_prolong(const ms_basis &b, int n, const double *xc, double *x, cudaStream_t st);
void launch_prolong32(const ms_basis &b, int n, const float *xc, double *x, cudaStream_t st);
void launch_to_float(const double *a, float *b, int64_t n, cudaStream_t st);
void launch_widen(const float *a, double *b, int64_t n, cudaStream_t st);
void launch_narrow(const double *a, float *b, int64_t n, cudaStream_t st);
// ILU(0)
void launch_ilu_factor(ms_system &s, bool fp32, cudaStream_t st);
void launch_ilu_apply64(ms_system &s, const double *r, double *y, double *z, cudaStream_t st);
void launch_ilu_apply32(ms_system &s, const double *r, float *y, float *z, cudaStream_t st);
void launch_ilu_extract_dirs(ms_system &s, bool fp32, cudaStream_t st);
void launch_ilu_apply64_scratch(const ms_system &s, const double *r, double *y, double *z, int *flags, int *sync,
                                cudaStream_t st);
void launch_ilu_tiled64(ms_system &s, const double *r, double *y, double *z, cudaStream_t st);
void launch_ilu_tiled32(ms_system &s, const double *r, float *y, float *z, cudaStream_t st);
void launch_ilu_tiled32f(ms_system &s, const float *r, float *y, float *z, cudaStream_t st);
void plan_ilu_cluster(ms_system &s);
// segmented line sweeps (k_ilu_seg.cu): layout, FP64 scan tables, the two sweeps
bool plan_ilu_seg(ms_system &s, int p);
size_t seg_table_size(const ms_system &s);
void pack_seg_tables(ms_system &s, const double *coef4, double *table, cudaStream_t st);
template <typename T, typename TR>
void seg_fwd(ms_system &s, int p, const T *coef4, const T *scanm, const TR *rhs, T *out, cudaStream_t st);
template <typename T>
void seg_bwd(ms_system &s, int p, const T *coef4, const T *scanm, const T *rhs, T *out, cudaStream_t st);
bool launch_ilu_factor_cluster(ms_system &s, cudaStream_t st);
void launch_ilu_pack_coef4(ms_system &s, bool fp32, cudaStream_t st);
void launch_ilu_cluster64(ms_system &s, const double *r, double *y, double *z, cudaStream_t st);
void launch_ilu_cluster32(ms_system &s, const double *r, float *y, float *z, cudaStream_t st);
void launch_ilu_cluster32f(ms_system &s, const float *r, float *y, float *z, cudaStream_t st);
void launch_ilu_lines64(ms_system &s, const double *r, double *y, double *z, cudaStream_t st);
bool launch_ilu_level64(ms_system &s, const double *r, double *y, double *z, cudaStream_t st);
bool launch_ilu_level32(ms_system &s, const double *r, float *y, float *z, cudaStream_t st);
void launch_ilu_seg_pack(ms_system &s, bool fp32, cudaStream_t st);
bool launch_ilu_seg64(ms_system &s, const double *r, double *y, double *z, cudaStream_t st);
bool launch_ilu_seg32(ms_system &s, const double *r, float *y, float *z, cudaStream_t st);
void launch_ilu_lines32(ms_system &s, const double *r, float *y, float *z, cudaStream_t st);
void launch_ilu_lines32f(ms_system &s, const float *r, float *y, float *z, cudaStream_t st);
// basis
void launch_basis_init(ms_basis &b, int n, cudaStream_t st);
void launch_basis_maps(const ms_system &s, ms_basis &b, cudaStream_t st);
void launch_basis_scale(const ms_system &s, ms_basis &b, bool fp32, cudaStream_t st);
void launch_msrsb_iter(const ms_system &s, ms_basis &b, bool fp32, unsigned long long *ctl, double tol, int max_iter,
                       cudaStream_t st);
void launch_basis_columns(ms_basis &b, cudaStream_t st);
// Re-smooth the bases of several systems from their block indicators in one
// persistent launch per precision; members it cannot take (no slot maps, more
// than 8 connections per row) get taken[m] = 0 and are left to the caller.
void smooth_batch(ms_ctx *ctx, const std::vector<ms_system *> &sys, const std::vector<ms_basis *> &bases,
                  std::vector<char> &taken);
// Galerkin
int launch_ap_count(const ms_system &s, const ms_basis &b, int *cnt_max, int *host_pinned, cudaStream_t st);
void launch_ap_fill(const ms_system &s, const ms_basis &b, ms_coarse &c, cudaStream_t st);
// A_c = R (A P) from the (A P) lists of c, R given by its column view
// (cval null: unit weights); symmetrise for the Galerkin operator.
void launch_rap(const ms_system &s, const std::vector<int> &h_cptr, const int *cptr, const int *ccell,
                const double *cval, bool symmetrise, ms_coarse &c, cudaStream_t st);
// dense
void dense_factor_inverse64(ms_coarse &c, int *err, cudaStream_t st);
void dense_factor_inverse32(ms_coarse &c, int *err, cudaStream_t st);
// blocked symmetric sweep in one launch (FP64 CUDA cores; FP32 on tcgen05)
void dense_sweep_inverse64(ms_coarse &c, int *err, cudaStream_t st);
void dense_sweep_inverse32(ms_coarse &c, int *err, cudaStream_t st);
void coarse_sparse_copy(ms_coarse &c, int *scratch, int *host, cudaStream_t st);
void dense_gj_inverse64(ms_coarse &c, int *err, cudaStream_t st);
void dense_gj_inverse32(ms_coarse &c, int *err, cudaStream_t st);
void launch_check_diag(const ms_coarse &c, int *err, cudaStream_t st);
void launch_cpr_pressure(ms_system &s, const ms_cpr_fluid &f, double dt, const double *p, const double *sw,
                         const double *p0, const double *s0, const double *qw, const double *qo, double *rhs,
                         double *wout, cudaStream_t st);
double coarse_inverse_check32(const ms_coarse &c, double *host2, cudaStream_t st);
void launch_gemv64(const double *A, int M, const double *x, double *y, cudaStream_t st);
void launch_gemv32(const float *A, int M, const float *x, float *y, cudaStream_t st);
void launch_coarse_refine(const ms_coarse &c, const double *d, double *xc, double *rc, float *t32a, float *t32b,
                          int steps, cudaStream_t st);
// partitions
void launch_components(const ms_system &s, const int *cls, int *label, cudaStream_t st);
void launch_dynamic_classes(const ms_system &s, const double *dp, int n_bins, double eps, int *cls,
                            unsigned long long *maxbuf, cudaStream_t st);
int launch_number_components(const ms_system &s, int *label, int *part, int *scratch, int *host_pinned,
                             cudaStream_t st);

}  // namespace msgb
