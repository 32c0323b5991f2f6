// C ABI (include/ms.h): handle management and host orchestration of the
// kernels.  Every numeric step of the method runs in this library's CUDA
// kernels; the host only sequences launches, moves caller arrays, reads
// convergence scalars and builds integer patterns (ms_analysis.cpp).
#include <algorithm>
#include <thread>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <new>

#include "ms_internal.h"

using namespace msgb;

namespace {

// Make the context's device current for the duration of a call.
struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev && cudaSetDevice(dev) != cudaSuccess) cudaGetLastError();   // later calls report it
    }
    ~DeviceGuard() {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

bool is_device_ptr(const void *p) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Device view of a caller array: the array itself if it is device memory,
// otherwise a copy in `stage`.
template <typename T>
const T *device_in(const T *p, size_t count, DBuf<T> &stage, cudaStream_t st) {
    if (!p) return nullptr;
    if (is_device_ptr(p)) return p;
    stage.alloc(std::max<size_t>(count, 1));
    MS_CUDA(cudaMemcpyAsync(stage.p, p, count * sizeof(T), cudaMemcpyHostToDevice, st));
    return stage.p;
}

template <typename T>
void copy_out(T *dst, const T *src, size_t count, cudaStream_t st) {
    MS_CUDA(cudaMemcpyAsync(dst, src, count * sizeof(T), is_device_ptr(dst) ? cudaMemcpyDeviceToDevice
                                                                           : cudaMemcpyDeviceToHost, st));
}

void sync(cudaStream_t st) { MS_CUDA(cudaStreamSynchronize(st)); }

int read_error_word(ms_ctx *ctx, const int *dev_word) {
    int *h = (int *)ctx->pinned.get(64);
    MS_CUDA(cudaMemcpyAsync(h, dev_word, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    sync(ctx->stream);
    return *h;
}

void check_sweep_errors(ms_ctx *ctx, ms_system *s) {
    const int e = read_error_word(ctx, s->sync.p + 3);
    if (e) {
        MS_CUDA(cudaMemsetAsync(s->sync.p + 3, 0, sizeof(int), ctx->stream));
        // a sweep that gave up left its barrier counter short: start it afresh
        if (s->lev_bar.n) MS_CUDA(cudaMemsetAsync(s->lev_bar.p, 0, 2 * sizeof(unsigned long long), ctx->stream));
        if (e & kErrTimeout) throw Error{MS_ERR_TIMEOUT, "a level-ordered sweep wait ran out"};
        if (e & kErrSingular) throw Error{MS_ERR_INVALID_ARG, "ILU(0) met a zero pivot"};
        throw Error{MS_ERR_CUDA, "device error word " + std::to_string(e)};
    }
}

// A grid-barrier timeout in a stage's one-launch coarse solve: reset its
// barrier and report it.
void check_refine_errors(ms_ctx *ctx, ms_coarse *c) {
    if (!c || !c->refine_err.n) return;
    const int e = read_error_word(ctx, c->refine_err.p);
    if (!e) return;
    MS_CUDA(cudaMemsetAsync(c->refine_err.p, 0, sizeof(int), ctx->stream));
    if (c->gj_bar.n) MS_CUDA(cudaMemsetAsync(c->gj_bar.p, 0, 2 * sizeof(unsigned long long), ctx->stream));
    throw Error{MS_ERR_TIMEOUT, "a coarse-solve grid barrier wait ran out"};
}

ms_status fail(ms_ctx *ctx, ms_status st, const std::string &what) {
    if (ctx) ctx->err = what;
    return st;
}

#define API_TRY try {
#define API_CATCH(ctx)                                                         \
    }                                                                          \
    catch (const Error &e) { return fail((ctx), e.status, e.what); }           \
    catch (const std::bad_alloc &) { return fail((ctx), MS_ERR_OOM, "host allocation failed"); } \
    catch (...) { return fail((ctx), MS_ERR_CUDA, "unexpected exception"); }

// ------------------------------------------------------------ internals
void ensure_fp32_matrix(ms_system &s, cudaStream_t st) {
    const size_t en = std::max<size_t>((size_t)s.W * s.n, 1);
    s.off_p32.alloc(en);
    s.off_u32.alloc(en);
    s.diag32.alloc(s.n);
    launch_to_float(s.off_p.p, s.off_p32.p, (int64_t)en, st);
    launch_to_float(s.off_u.p, s.off_u32.p, (int64_t)en, st);
    launch_to_float(s.diag.p, s.diag32.p, s.n, st);
}

void ensure_ilu(ms_ctx *ctx, ms_system &s, bool fp32) {
    if (s.ilu64_valid && (!fp32 || s.ilu32_valid)) return;
    const bool had64 = s.ilu64_valid;
    launch_ilu_factor(s, fp32, ctx->stream);
    check_sweep_errors(ctx, &s);
    if (s.structured) {
        if (!had64) {
            launch_ilu_extract_dirs(s, false, ctx->stream);
            if (s.cl_ok[0]) launch_ilu_pack_coef4(s, false, ctx->stream);
        }
        if (fp32) {
            launch_ilu_extract_dirs(s, true, ctx->stream);
            if (s.cl_ok[1]) launch_ilu_pack_coef4(s, true, ctx->stream);
        }
    } else if (s.n_seg > 0) {
        if (!had64) launch_ilu_seg_pack(s, false, ctx->stream);
        if (fp32) launch_ilu_seg_pack(s, true, ctx->stream);
    }
    s.ilu64_valid = true;
    if (fp32) s.ilu32_valid = true;
}

// z = (LU)^{-1} r: wavefront sweeps on structured grids (line scan across a
// cluster, line scan over CTA tiles, or pencil tiles, chosen per precision when
// the system is analysed), segment dataflow sweeps otherwise (level-synchronous
// sweeps in one cooperative launch, or flag-ordered sweeps, where those cannot run).
void ilu_apply64(ms_system &s, const double *r, double *y, double *z, cudaStream_t st) {
    switch (s.ilu_kind[0]) {
        case 3: launch_ilu_cluster64(s, r, y, z, st); break;
        case 2: launch_ilu_lines64(s, r, y, z, st); break;
        case 1: launch_ilu_tiled64(s, r, y, z, st); break;
        case 5: if (launch_ilu_seg64(s, r, y, z, st)) break; [[fallthrough]];
        case 4: if (launch_ilu_level64(s, r, y, z, st)) break; [[fallthrough]];
        default: launch_ilu_apply64(s, r, y, z, st);
    }
}

void ilu_apply32(ms_system &s, const double *r, float *y, float *z, cudaStream_t st) {
    switch (s.ilu_kind[1]) {
        case 3: launch_ilu_cluster32(s, r, y, z, st); break;
        case 2: launch_ilu_lines32(s, r, y, z, st); break;
        case 1: launch_ilu_tiled32(s, r, y, z, st); break;
        case 5: if (launch_ilu_seg32(s, r, y, z, st)) break; [[fallthrough]];
        case 4: if (launch_ilu_level32(s, r, y, z, st)) break; [[fallthrough]];
        default: launch_ilu_apply32(s, r, y, z, st);
    }
}

// FP32 right-hand side: structured systems only
void ilu_apply32f(ms_system &s, const float *r, float *y, float *z, cudaStream_t st) {
    switch (s.ilu_kind[1]) {
        case 3: launch_ilu_cluster32f(s, r, y, z, st); break;
        case 2: launch_ilu_lines32f(s, r, y, z, st); break;
        default: launch_ilu_tiled32f(s, r, y, z, st);
    }
}

// Smooth a basis: reset from the indicator (reset) or continue; returns iterations.
int smooth_basis(ms_ctx *ctx, ms_system &s, ms_basis &b, bool reset, double tol, int max_iter) {
    cudaStream_t st = ctx->stream;
    if (reset) launch_basis_init(b, s.n, st);
    int it = 0;
    double inc = 0.0;
    if (b.rule != MS_SUPPORT_BLOCK) {
        const bool fp32 = b.precision == MS_PREC_MIXED;
        // iterations are enqueued in batches; a control kernel after each one
        // counts it and stops the rest on the device once converged, so the host
        // reads the state once per batch instead of once per iteration
        s.w_max.alloc(4);
        unsigned long long *h = (unsigned long long *)ctx->pinned.get(64);
        if (max_iter > 0) {
            launch_basis_scale(s, b, fp32, st);
            MS_CUDA(cudaMemsetAsync(s.w_max.p, 0, 4 * sizeof(unsigned long long), st));
            constexpr int kBatch = 16;
            for (int queued = 0; queued < max_iter;) {
                const int k = std::min(kBatch, max_iter - queued);
                for (int q = 0; q < k; ++q) launch_msrsb_iter(s, b, fp32, s.w_max.p, tol, max_iter, st);
                queued += k;
                MS_CUDA(cudaMemcpyAsync(h, s.w_max.p, 4 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
                sync(st);
                if (h[0]) break;
            }
            it = (int)h[1];
            std::memcpy(&inc, &h[3], sizeof(double));
            if (it & 1) {   // the result is in the other buffer
                if (fp32) std::swap(b.pval32.p, b.pval32_tmp.p);
                else std::swap(b.pval.p, b.pval_tmp.p);
            }
            if (!(inc == inc)) throw Error{MS_ERR_INVALID_ARG, "basis smoothing produced NaN"};
        }
    }
    b.iters = it;
    b.last_inc = inc;
    b.assembly_id = s.assembly_id;
    launch_basis_columns(b, st);
    return it;
}

ms_basis *create_basis(ms_ctx *ctx, ms_system &s, const std::vector<int> &part, int M, int rule, int precision,
                       int bx, int by, int bz) {
    std::vector<int> cptr, ccell, pid, csrc;
    std::vector<unsigned char> home;
    analyse_supports(s, part, M, rule, bx, by, bz, cptr, ccell);
    int B = 0;
    slot_layout(s, part, M, cptr, ccell, B, pid, csrc, home);
    MS_REQUIRE((int64_t)B * s.n < ((int64_t)1 << 31), MS_ERR_INVALID_ARG, "basis slot layout too large");
    std::unique_ptr<ms_basis> b(new ms_basis());
    b->M = M;
    b->B = B;
    b->nnz = (int64_t)ccell.size();
    b->rule = rule;
    b->precision = precision;
    b->h_part = part;
    cudaStream_t st = ctx->stream;
    b->part.upload(part, st);
    b->pid.upload(pid, st);
    b->is_home.upload(home, st);
    b->cptr.upload(cptr, st);
    {
        std::vector<int> cb, cc, cp;
        build_column_chunks(cptr, M, kColChunk, cb, cc, cp, nullptr, nullptr);
        b->n_chunks = (int)cb.size();
        b->ch_beg.upload(cb, st);
        b->ch_col.upload(cc, st);
        b->ch_ptr.upload(cp, st);
        b->ch_part.alloc(std::max<size_t>(cb.size(), 1));
        b->ch_cnt.alloc(std::max(M, 1));
        b->ch_cnt.zero(st);
    }
    b->h_cptr = cptr;
    b->ccell.upload(ccell, st);
    b->csrc.upload(csrc, st);
    if (rule != MS_SUPPORT_BLOCK) launch_basis_maps(s, *b, st);
    const size_t slots = (size_t)B * s.n;
    b->pval.alloc(slots);
    b->cval.alloc(std::max<int64_t>(b->nnz, 1));
    if (precision == MS_PREC_MIXED) {
        b->pval32.alloc(slots);
        b->pval32_tmp.alloc(slots);
        b->cval32.alloc(std::max<int64_t>(b->nnz, 1));
        MS_CUDA(cudaMemsetAsync(b->pval32_tmp.p, 0, slots * sizeof(float), st));
    } else {
        b->pval_tmp.alloc(slots);
        MS_CUDA(cudaMemsetAsync(b->pval_tmp.p, 0, slots * sizeof(double), st));
    }
    return b.release();
}

// Symmetric coarse inverses: the blocked sweep in one launch (default), or
// MSGB_COARSE_INVERSE=chain for the Cholesky factor-and-invert kernel chain.
bool coarse_chain() {
    const char *e = std::getenv("MSGB_COARSE_INVERSE");
    return e && std::string(e) == "chain";
}

// Error word of a coarse factorisation: a timeout of the Gauss-Jordan grid
// barrier resets its counter before the error is raised.
void coarse_error(ms_ctx *ctx, ms_coarse &c, int err) {
    if (!err) return;
    if (err & kErrTimeout) {
        if (c.gj_bar.n) MS_CUDA(cudaMemsetAsync(c.gj_bar.p, 0, 2 * sizeof(unsigned long long), ctx->stream));
        throw Error{MS_ERR_TIMEOUT, "a coarse factorisation wait ran out"};
    }
    throw Error{MS_ERR_COARSE_SINGULAR, c.nonsym
                                            ? "coarse Gauss-Jordan elimination met a zero pivot column"
                                            : "coarse Cholesky met a non-positive pivot"};
}

void galerkin_values(ms_ctx *ctx, ms_system &s, const ms_basis &b, ms_coarse &c) {
    cudaStream_t st = ctx->stream;
    MS_REQUIRE(s.assembled, MS_ERR_STATE, "system not assembled");
    const bool fv = c.restriction == MS_RESTRICT_FV;
    c.nonsym = fv || !s.symmetric;   // Gauss-Jordan inverse instead of Cholesky
    s.w_i0.alloc(4);
    int *h = (int *)ctx->pinned.get(64);
    const int wap = launch_ap_count(s, b, s.w_i0.p, h, st);
    c.WAP = std::max(wap, 1);
    c.apid.alloc((size_t)c.WAP * s.n);
    c.apval.alloc((size_t)c.WAP * s.n);
    launch_ap_fill(s, b, c, st);
    c.Ac.alloc((size_t)c.M * c.M);
    if (fv) launch_rap(s, c.fv_h_cptr, c.fv_cptr.p, c.fv_ccell.p, nullptr, false, c, st);
    else launch_rap(s, b.h_cptr, b.cptr.p, b.ccell.p, b.cval.p, s.symmetric, c, st);
    MS_CUDA(cudaMemsetAsync(s.w_i0.p, 0, sizeof(int), st));
    c.use64 = false;
    c.inv32_error = 0.0;
    const bool gj = c.nonsym;
    const bool chain = coarse_chain();
    auto inverse64 = [&]() {
        if (gj) dense_gj_inverse64(c, s.w_i0.p, st);
        else if (chain) dense_factor_inverse64(c, s.w_i0.p, st);
        else dense_sweep_inverse64(c, s.w_i0.p, st);
    };
    if (c.precision == MS_PREC_MIXED) {
        bool try32 = true;
        if (gj) {   // the FP32 path equilibrates with 1/sqrt(a_jj)
            launch_check_diag(c, s.w_i0.p, st);
            try32 = read_error_word(ctx, s.w_i0.p) == 0;
            MS_CUDA(cudaMemsetAsync(s.w_i0.p, 0, sizeof(int), st));
        }
        if (try32) {
            if (gj) dense_gj_inverse32(c, s.w_i0.p, st);
            else if (chain) dense_factor_inverse32(c, s.w_i0.p, st);
            else dense_sweep_inverse32(c, s.w_i0.p, st);
            const int err32 = read_error_word(ctx, s.w_i0.p);
            if (err32 & kErrTimeout) coarse_error(ctx, c, err32);
            c.inv32_error = err32 ? INFINITY : coarse_inverse_check32(c, (double *)ctx->pinned.get(64), st);
        } else {
            c.inv32_error = INFINITY;
        }
        // each FP64 refinement step contracts the coarse error by about this
        // factor e: take the steps that bring e^(steps+1) to 0.03^3 (2 steps up
        // to e = 0.03, at most 5, up to e = 0.15); fall back to an FP64 inverse
        // beyond that
        const double e = c.inv32_error;
        if (e <= 0.03) {
            c.refine_steps = 2;
        } else if (e <= 0.15) {
            c.refine_steps = std::min(5, (int)std::ceil(std::log(2.7e-5) / std::log(e)) - 1);
        } else {
            c.use64 = true;
            MS_CUDA(cudaMemsetAsync(s.w_i0.p, 0, sizeof(int), st));
            inverse64();
        }
        if (!c.use64) coarse_sparse_copy(c, s.w_i0.p + 1, (int *)ctx->pinned.get(64), st);
    } else {
        inverse64();
    }
    coarse_error(ctx, c, read_error_word(ctx, s.w_i0.p));
    // the apid/apval scratch is only needed while forming A_c
    c.apid.release();
    c.apval.release();
}

// Block member lists of the finite-volume restriction (cells ascending) and
// their column chunks.
void fv_view(ms_ctx *ctx, const ms_basis &b, ms_coarse &c) {
    const int M = b.M;
    const int n = (int)b.h_part.size();
    std::vector<int> cptr(M + 1, 0), cell(n);
    for (int i = 0; i < n; ++i) {
        MS_REQUIRE(b.h_part[i] >= 0 && b.h_part[i] < M, MS_ERR_INVALID_ARG, "partition entry out of range");
        cptr[b.h_part[i] + 1]++;
    }
    for (int j = 0; j < M; ++j) cptr[j + 1] += cptr[j];
    std::vector<int> fill(cptr.begin(), cptr.end() - 1);
    for (int i = 0; i < n; ++i) cell[fill[b.h_part[i]]++] = i;
    cudaStream_t st = ctx->stream;
    std::vector<int> cb, cc, cp;
    build_column_chunks(cptr, M, kColChunk, cb, cc, cp, nullptr, nullptr);
    c.fv_n_chunks = (int)cb.size();
    c.fv_ch_beg.upload(cb, st);
    c.fv_ch_col.upload(cc, st);
    c.fv_ch_ptr.upload(cp, st);
    c.fv_ch_part.alloc(std::max<size_t>(cb.size(), 1));
    c.fv_ch_cnt.alloc(std::max(M, 1));
    c.fv_ch_cnt.zero(st);
    c.fv_cptr.upload(cptr, st);
    c.fv_ccell.upload(cell, st);
    c.fv_h_cptr = std::move(cptr);
}

ms_coarse *create_coarse(ms_ctx *ctx, ms_system &s, const ms_basis &b, int precision, int restriction) {
    std::unique_ptr<ms_coarse> c(new ms_coarse());
    c->M = b.M;
    c->precision = precision;
    c->basis = &b;
    c->restriction = restriction;
    if (restriction == MS_RESTRICT_FV) fv_view(ctx, b, *c);
    galerkin_values(ctx, s, b, *c);
    return c.release();
}

// Dynamic partition of a device dp into device part; returns block count.
int partition_dynamic_dev(ms_ctx *ctx, ms_system &s, const double *dp, int n_bins, double eps, int *part) {
    cudaStream_t st = ctx->stream;
    const int nb = (s.n + 255) / 256;
    s.w_i1.alloc(s.n);                    // classes, then labels
    s.w_i2.alloc((size_t)s.n + nb + 2);   // scan scratch
    s.w_max.alloc(4);
    launch_dynamic_classes(s, dp, n_bins, eps, s.w_i1.p, s.w_max.p, st);
    s.w_i0.alloc(std::max(s.n, 4));
    launch_components(s, s.w_i1.p, s.w_i0.p, st);
    int *h = (int *)ctx->pinned.get(64);
    return launch_number_components(s, s.w_i0.p, part, s.w_i2.p, h, st);
}

ms_basis *adaptive_basis(ms_ctx *ctx, ms_system &s, const double *dp_dev, const ms_adapt_opts &o,
                         int precision) {
    MS_REQUIRE(o.n_bins > 0 && o.eps > 0, MS_ERR_INVALID_ARG, "adaptive options: n_bins > 0 and eps > 0 required");
    DBuf<int> part_d;
    part_d.alloc(s.n);
    const int M = partition_dynamic_dev(ctx, s, dp_dev, o.n_bins, o.eps, part_d.p);
    std::vector<int> part(s.n);
    MS_CUDA(cudaMemcpyAsync(part.data(), part_d.p, s.n * sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    sync(ctx->stream);
    const int rule = o.smoothed ? MS_SUPPORT_HOP : MS_SUPPORT_BLOCK;
    std::unique_ptr<ms_basis> b(create_basis(ctx, s, part, M, rule, precision, 0, 0, 0));
    b->omega = o.omega > 0 ? o.omega : 2.0 / 3.0;
    b->tol = o.tol > 0 ? o.tol : 1e-3;
    b->max_iter = o.max_iter > 0 ? o.max_iter : 500;
    smooth_basis(ctx, s, *b, true, b->tol, b->max_iter);
    return b.release();
}

double read_norm(ms_ctx *ctx, const double *dev) {
    double *h = (double *)ctx->pinned.get(64);
    MS_CUDA(cudaMemcpyAsync(h, dev, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    sync(ctx->stream);
    return *h;
}

}  // namespace

namespace {
thread_local int64_t t_device_bytes = 0;
std::atomic<int64_t> g_device_allocs{0};
}  // namespace

namespace msgb {
void note_device_alloc(size_t bytes) {
    t_device_bytes += (int64_t)bytes;
    g_device_allocs.fetch_add(1, std::memory_order_relaxed);
}
}  // namespace msgb

// =================================================================== ABI
extern "C" {

int32_t ms_abi_version(void) { return MS_ABI_VERSION; }

const char *ms_status_string(ms_status s) {
    switch (s) {
        case MS_OK: return "ok";
        case MS_ERR_INVALID_ARG: return "invalid argument";
        case MS_ERR_OOM: return "out of memory";
        case MS_ERR_CUDA: return "CUDA error";
        case MS_ERR_NOT_CONVERGED: return "not converged";
        case MS_ERR_COARSE_SINGULAR: return "coarse system not positive definite";
        case MS_ERR_TIMEOUT: return "device wait timed out";
        case MS_ERR_STATE: return "invalid state";
    }
    return "unknown status";
}

const char *ms_last_error(const ms_ctx *ctx) { return ctx ? ctx->err.c_str() : ""; }

ms_status ms_create(ms_ctx **out, int32_t device, void *stream) {
    if (!out) return MS_ERR_INVALID_ARG;
    *out = nullptr;
    API_TRY
    int ndev = 0;
    MS_CUDA(cudaGetDeviceCount(&ndev));
    MS_REQUIRE(device >= 0 && device < ndev, MS_ERR_INVALID_ARG, "no such CUDA device");
    std::unique_ptr<ms_ctx> c(new ms_ctx());
    c->device = device;
    c->stream = (cudaStream_t)stream;
    DeviceGuard g(device);
    MS_CUDA(cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device));
    *out = c.release();
    return MS_OK;
    API_CATCH(nullptr)
}

ms_status ms_destroy(ms_ctx *ctx) {
    delete ctx;
    return MS_OK;
}

ms_status ms_set_stream(ms_ctx *ctx, void *stream) {
    if (!ctx) return MS_ERR_INVALID_ARG;
    ctx->stream = (cudaStream_t)stream;
    return MS_OK;
}

ms_status ms_system_create(ms_ctx *ctx, const ms_grid *grid, int32_t ref_cell, ms_system **out) {
    if (!ctx || !grid || !out) return fail(ctx, MS_ERR_INVALID_ARG, "null argument");
    *out = nullptr;
    API_TRY
    DeviceGuard g(ctx->device);
    std::unique_ptr<ms_system> s(new ms_system());
    s->device = ctx->device;
    analyse_grid(*s, *grid);
    MS_REQUIRE(ref_cell >= 0 && ref_cell < s->n, MS_ERR_INVALID_ARG, "reference cell out of range");
    s->ref = ref_cell;
    *out = s.release();
    return MS_OK;
    API_CATCH(ctx)
}

ms_status ms_system_release(ms_system *sys) {
    if (sys) {
        DeviceGuard g(sys->device);
        delete sys;
    }
    return MS_OK;
}

ms_status ms_system_get_info(const ms_system *s, ms_system_info *info) {
    if (!s || !info) return MS_ERR_INVALID_ARG;
    info->n = s->n;
    info->n_faces = s->nf;
    info->ell_width = s->W;
    info->n_levels = s->n_levels;
    info->ref_cell = s->ref;
    return MS_OK;
}

ms_status ms_assemble_tpfa(ms_ctx *ctx, ms_system *s, const double *perm, const double *mobility,
                           const double *p_prev) {
    if (!ctx || !s || !perm) return fail(ctx, MS_ERR_INVALID_ARG, "null argument");
    if (p_prev && !mobility) return fail(ctx, MS_ERR_INVALID_ARG, "p_prev given without mobility");
    API_TRY
    DeviceGuard g(ctx->device);
    cudaStream_t st = ctx->stream;
    const int64_t N = (int64_t)s->nx * s->ny * s->nz;
    DBuf<double> stage_perm, stage_mob, stage_pp;
    const double *kp = device_in(perm, (size_t)(3 * N), stage_perm, st);
    const double *mob = device_in(mobility, (size_t)s->n, stage_mob, st);
    const double *pp = device_in(p_prev, (size_t)s->n, stage_pp, st);
    s->w_i0.alloc(4);
    MS_CUDA(cudaMemsetAsync(s->w_i0.p, 0, sizeof(int), st));
    launch_check_perm(kp, 3 * N, s->w_i0.p, st);
    if (read_error_word(ctx, s->w_i0.p)) throw Error{MS_ERR_INVALID_ARG, "permeability negative, NaN or infinite"};
    launch_face_trans(*s, kp, mob, pp, st);
    launch_row_assemble(*s, st);
    ensure_fp32_matrix(*s, st);
    s->ilu64_valid = s->ilu32_valid = false;
    s->assembled = true;
    s->pinned = s->symmetric = true;
    s->assembly_id++;
    sync(st);
    return MS_OK;
    API_CATCH(ctx)
}

ms_status ms_cpr_pressure_system(ms_ctx *ctx, ms_system *s, const double *perm, const ms_cpr_fluid *f,
                                 const double *p, const double *sw, const double *p0, const double *s0,
                                 const double *q_w, const double *q_o, double dt, double *rhs, double *weights) {
    if (!ctx || !s || !perm || !f || !p || !sw || !p0 || !s0 || !q_w || !q_o || !rhs)
        return fail(ctx, MS_ERR_INVALID_ARG, "null argument");
    API_TRY
    DeviceGuard g(ctx->device);
    MS_REQUIRE(dt > 0 && f->mu_w > 0 && f->mu_o > 0 && f->n_w >= 1 && f->n_o >= 1 && f->s_wc >= 0 && f->s_or >= 0 &&
                   f->s_wc + f->s_or < 1.0 && f->phi0 > 0 && f->rho_w0 > 0 && f->rho_o0 > 0,
               MS_ERR_INVALID_ARG, "bad CPR fluid or time step");
    cudaStream_t st = ctx->stream;
    const int64_t N = (int64_t)s->nx * s->ny * s->nz;
    const size_t n = (size_t)s->n;
    DBuf<double> stage_perm, sp, ss, sp0, ss0, sqw, sqo, out_r, out_w;
    const double *kp = device_in(perm, (size_t)(3 * N), stage_perm, st);
    s->w_i0.alloc(4);
    MS_CUDA(cudaMemsetAsync(s->w_i0.p, 0, sizeof(int), st));
    launch_check_perm(kp, 3 * N, s->w_i0.p, st);
    if (read_error_word(ctx, s->w_i0.p)) throw Error{MS_ERR_INVALID_ARG, "permeability negative, NaN or infinite"};
    launch_face_trans(*s, kp, nullptr, nullptr, st);   // geometric transmissibilities
    const double *pd = device_in(p, n, sp, st), *sd = device_in(sw, n, ss, st);
    const double *p0d = device_in(p0, n, sp0, st), *s0d = device_in(s0, n, ss0, st);
    const double *qwd = device_in(q_w, n, sqw, st), *qod = device_in(q_o, n, sqo, st);
    double *rd = rhs, *wd = weights;
    if (!is_device_ptr(rhs)) { out_r.alloc(n); rd = out_r.p; }
    if (weights && !is_device_ptr(weights)) { out_w.alloc(2 * n); wd = out_w.p; }
    launch_cpr_pressure(*s, *f, dt, pd, sd, p0d, s0d, qwd, qod, rd, wd, st);
    ensure_fp32_matrix(*s, st);
    s->ilu64_valid = s->ilu32_valid = false;
    s->assembled = true;
    s->pinned = s->symmetric = false;
    s->assembly_id++;
    if (rd != rhs) copy_out(rhs, rd, n, st);
    if (weights && wd != weights) copy_out(weights, wd, 2 * n, st);
    sync(st);
    return MS_OK;
    API_CATCH(ctx)
}

ms_status ms_system_get_matrix(ms_ctx *ctx, const ms_system *s, int32_t pinned, int32_t *col, double *val,
                               double *diag) {
    if (!ctx || !s || !col || !val || !diag) return fail(ctx, MS_ERR_INVALID_ARG, "null argument");
    API_TRY
    DeviceGuard g(ctx->device);
    MS_REQUIRE(s->assembled, MS_ERR_STATE, "system not assembled");
    const size_t en = (size_t)s->W * s->n;
    if (en) {
        copy_out(col, s->col.p, en, ctx->stream);
        copy_out(val, pinned ? s->off_p.p : s->off_u.p, en, ctx->stream);
    }
    copy_out(diag, s->diag.p, s->n, ctx->stream);
    sync(ctx->stream);
    return MS_OK;
    API_CATCH(ctx)
}

ms_status ms_spmv(ms_ctx *ctx, const ms_system *s, const double *x, double *y) {
    if (!ctx || !s || !x || !y) return fail(ctx, MS_ERR_INVALID_ARG, "null argument");
    API_TRY
    DeviceGuard g(ctx->device);
    MS_REQUIRE(s->assembled, MS_ERR_STATE, "system not assembled");
    ms_system &m = const_cast<ms_system &>(*s);
    const double *xd = device_in(x, s->n, m.w_q, ctx->stream);
    m.w_r.alloc(s->n);
    launch_spmv(*s, xd, m.w_r.p, ctx->stream);
    copy_out(y, m.w_r.p, s->n, ctx->stream);
    sync(ctx->stream);
    return MS_OK;
    API_CATCH(ctx)
}

ms_status ms_ilu_apply(ms_ctx *ctx, ms_system *s, int32_t precision, const double *r, double *z) {
    if (!ctx || !s || !r || !z) return fail(ctx, MS_ERR_INVALID_ARG, "null argument");
    API_TRY
    DeviceGuard g(ctx->device);
    MS_REQUIRE(s->assembled, MS_ERR_STATE, "system not assembled");
    cudaStream_t st = ctx->stream;
    const bool fp32 = precision == MS_PREC_MIXED;
    ensure_ilu(ctx, *s, fp32);
    const double *rd = device_in(r, s->n, s->w_q, st);
    s->w_z.alloc(s->n);
    if (fp32) {
        s->w_y32.alloc(s->n);
        s->w_z32.alloc(s->n);
        ilu_apply32(*s, rd, s->w_y32.p, s->w_z32.p, st);
        launch_widen(s->w_z32.p, s->w_z.p, s->n, st);
    } else {
        s->w_y.alloc(s->n);
        ilu_apply64(*s, rd, s->w_y.p, s->w_z.p, st);
    }
    check_sweep_errors(ctx, s);
    copy_out(z, s->w_z.p, s->n, st);
    sync(st);
    return MS_OK;
    API_CATCH(ctx)
}

ms_status ms_allocation_stats(int64_t *thread_bytes, int64_t *allocations) {
    if (thread_bytes) *thread_bytes = t_device_bytes;
    if (allocations) *allocations = g_device_allocs.load(std::memory_order_relaxed);
    return MS_OK;
}

ms_status ms_pressure_update(ms_ctx *ctx, const ms_system *s, const double *p, const double *p_prev, double *dp) {
    if (!ctx || !s || !p || !p_prev || !dp) return fail(ctx, MS_ERR_INVALID_ARG, "null argument");
    API_TRY
    DeviceGuard g(ctx->device);
    MS_REQUIRE(is_device_ptr(p) && is_device_ptr(p_prev) && is_device_ptr(dp), MS_ERR_INVALID_ARG,
               "ms_pressure_update takes device arrays");
    launch_sub(p, p_prev, dp, s->n, ctx->stream);
    return MS_OK;
    API_CATCH(ctx)
}

ms_status ms_set_wait_limit(ms_ctx *ctx, ms_system *s, double seconds) {
    if (!ctx || !s) return fail(ctx, MS_ERR_INVALID_ARG, "null argument");
    if (!(seconds >= 0.0 && seconds <= 60.0)) return fail(ctx, MS_ERR_INVALID_ARG, "wait limit must be in [0, 60] s");
    API_TRY
    DeviceGuard g(ctx->device);
    int us = seconds == 0.0 ? 0 : std::max(1, (int)std::lround(seconds * 1e6));
    MS_CUDA(cudaMemcpyAsync(s->sync.p + 4, &us, sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
    sync(ctx->stream);
    return MS_OK;
    API_CATCH(ctx)
}

ms_status ms_debug_withhold_segments(ms_ctx *ctx, ms_system *s, int32_t precision, int32_t count) {
    if (!ctx || !s) return fail(ctx, MS_ERR_INVALID_ARG, "null argument");
    API_TRY
    DeviceGuard g(ctx->device);
    const int p = precision == MS_PREC_MIXED ? 1 : 0;
    MS_REQUIRE(s->assembled && (p ? s->ilu32_valid : s->ilu64_valid), MS_ERR_STATE,
               "needs the ILU(0) factors of that precision (run ms_ilu_apply first)");
    MS_REQUIRE(!s->structured && s->ilu_kind[p] == 5 && s->n_seg > 0 && s->seg_kg[0] <= kSegMaxKG &&
                   s->seg_kg[1] <= kSegMaxKG && (p ? (const void *)s->seg_v32.p : (const void *)s->seg_v64.p),
               MS_ERR_STATE, "the system's ILU(0) sweeps are not the segment sweeps");
    MS_REQUIRE(count >= 1 && count < s->n_seg, MS_ERR_INVALID_ARG, "count must be in [1, number of segments)");
    // the next segment sweep hands out tickets from `count` on; sweep_end
    // resets the ticket for every later sweep
    int v = count;
    MS_CUDA(cudaMemcpyAsync(s->sync.p + 1, &v, sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
    sync(ctx->stream);
    return MS_OK;
    API_CATCH(ctx)
}

ms_status ms_plan_segments(ms_ctx *ctx, int32_t n, const int32_t *rowptr, const int32_t *col, int32_t max_len,
                           int32_t *seg_off, int32_t *n_seg, int32_t *order, int32_t *kg, int32_t *width) {
    if (!rowptr || !col || !seg_off || !n_seg || !order || !kg || !width)
        return fail(ctx, MS_ERR_INVALID_ARG, "null argument");
    if (n < 1) return fail(ctx, MS_ERR_INVALID_ARG, "n must be >= 1");
    if (max_len < 1 || max_len > kSegPlanMax) return fail(ctx, MS_ERR_INVALID_ARG, "max_len must be in 1..256");
    API_TRY
    MS_REQUIRE(rowptr[0] == 0, MS_ERR_INVALID_ARG, "rowptr[0] must be 0");
    std::vector<int> deg(n + 1, 0), nb, rowlen(n);
    for (int i = 0; i < n; ++i) {
        MS_REQUIRE(rowptr[i + 1] >= rowptr[i], MS_ERR_INVALID_ARG, "rowptr must not decrease");
        for (int e = rowptr[i]; e < rowptr[i + 1]; ++e) {
            const int k = col[e];
            MS_REQUIRE(k >= 0 && k < n, MS_ERR_INVALID_ARG, "column out of range");
            if (k != i) nb.push_back(k);
        }
        auto b0 = nb.begin() + deg[i];
        std::sort(b0, nb.end());
        nb.erase(std::unique(b0, nb.end()), nb.end());
        rowlen[i] = (int)(nb.end() - b0);
        deg[i + 1] = (int)nb.size();
    }
    SegmentPlan sp;
    segment_plan(n, nb, deg, rowlen, max_len, sp);
    const int ns = (int)sp.off.size() - 1;
    std::memcpy(seg_off, sp.off.data(), sp.off.size() * sizeof(int));
    std::memcpy(order, sp.ord.data(), sp.ord.size() * sizeof(int));
    *n_seg = ns;
    kg[0] = sp.kg[0];
    kg[1] = sp.kg[1];
    *width = sp.width;
    return MS_OK;
    API_CATCH(ctx)
}

ms_status ms_partition_cartesian(ms_ctx *ctx, const ms_system *s, int32_t bx, int32_t by, int32_t bz,
                                 int32_t *part, int32_t *n_blocks) {
    if (!ctx || !s || !part || !n_blocks) return fail(ctx, MS_ERR_INVALID_ARG, "null argument");
    API_TRY
    std::vector<int> p;
    *n_blocks = partition_cartesian(*s, bx, by, bz, p);
    std::memcpy(part, p.data(), p.size() * sizeof(int));
    return MS_OK;
    API_CATCH(ctx)
}

ms_status ms_partition_wells(ms_ctx *ctx, const ms_system *s, int32_t n_wells, const int32_t *well_ptr,
                             const int32_t *well_cells, int32_t *part, int32_t *n_blocks) {
    if (!ctx || !s || !part || !n_blocks || n_wells < 0 || (n_wells > 0 && (!well_ptr || !well_cells)))
        return fail(ctx, MS_ERR_INVALID_ARG, "null argument");
    API_TRY
    const int n = s->n;
    MS_REQUIRE(well_ptr == nullptr || well_ptr[0] == 0, MS_ERR_INVALID_ARG, "well_ptr[0] must be 0");
    std::vector<int> p(n, -1);
    for (int w = 0; w < n_wells; ++w) {
        MS_REQUIRE(well_ptr[w + 1] >= well_ptr[w], MS_ERR_INVALID_ARG, "well_ptr must not decrease");
        for (int e = well_ptr[w]; e < well_ptr[w + 1]; ++e) {
            const int i = well_cells[e];
            MS_REQUIRE(i >= 0 && i < n, MS_ERR_INVALID_ARG, "well cell out of range");
            MS_REQUIRE(p[i] == -1, MS_ERR_INVALID_ARG, "cell listed in two wells (or twice)");
            p[i] = w;
        }
    }
    for (int &v : p)
        if (v == -1) v = n_wells;
    std::memcpy(part, p.data(), (size_t)n * sizeof(int));
    *n_blocks = n_wells + 1;
    return MS_OK;
    API_CATCH(ctx)
}

ms_status ms_partition_components(ms_ctx *ctx, const ms_system *sc, const int32_t *cls, int32_t *part,
                                  int32_t *n_blocks) {
    if (!ctx || !sc || !cls || !part || !n_blocks) return fail(ctx, MS_ERR_INVALID_ARG, "null argument");
    API_TRY
    DeviceGuard g(ctx->device);
    ms_system &s = const_cast<ms_system &>(*sc);
    cudaStream_t st = ctx->stream;
    DBuf<int> stage;
    const int *cd = device_in(cls, s.n, stage, st);
    const int nb = (s.n + 255) / 256;
    DBuf<int> label, out, scratch;
    label.alloc(s.n);
    out.alloc(s.n);
    scratch.alloc((size_t)s.n + nb + 2);
    launch_components(s, cd, label.p, st);
    int *h = (int *)ctx->pinned.get(64);
    *n_blocks = launch_number_components(s, label.p, out.p, scratch.p, h, st);
    copy_out(part, out.p, s.n, st);
    sync(st);
    return MS_OK;
    API_CATCH(ctx)
}

ms_status ms_partition_dynamic(ms_ctx *ctx, const ms_system *sc, const double *dp, int32_t n_bins, double eps,
                               int32_t *part, int32_t *n_blocks) {
    if (!ctx || !sc || !dp || !part || !n_blocks) return fail(ctx, MS_ERR_INVALID_ARG, "null argument");
    if (n_bins <= 0 || !(eps > 0)) return fail(ctx, MS_ERR_INVALID_ARG, "n_bins > 0 and eps > 0 required");
    API_TRY
    DeviceGuard g(ctx->device);
    ms_system &s = const_cast<ms_system &>(*sc);
    cudaStream_t st = ctx->stream;
    DBuf<double> stage;
    const double *dd = device_in(dp, s.n, stage, st);
    DBuf<int> out;
    out.alloc(s.n);
    *n_blocks = partition_dynamic_dev(ctx, s, dd, n_bins, eps, out.p);
    copy_out(part, out.p, s.n, st);
    sync(st);
    return MS_OK;
    API_CATCH(ctx)
}

ms_status ms_build_basis(ms_ctx *ctx, ms_system *s, const int32_t *partition, int32_t n_blocks,
                         const ms_basis_opts *opts, ms_basis **out, int32_t *iters) {
    if (!ctx || !s || !partition || !opts || !out) return fail(ctx, MS_ERR_INVALID_ARG, "null argument");
    *out = nullptr;
    API_TRY
    DeviceGuard g(ctx->device);
    MS_REQUIRE(s->assembled, MS_ERR_STATE, "system not assembled");
    MS_REQUIRE(n_blocks > 0 && n_blocks <= s->n, MS_ERR_INVALID_ARG, "n_blocks out of range");
    MS_REQUIRE(opts->precision == MS_PREC_FP64 || opts->precision == MS_PREC_MIXED, MS_ERR_INVALID_ARG,
               "unknown precision");
    MS_REQUIRE(opts->support >= 0 && opts->support <= 2, MS_ERR_INVALID_ARG, "unknown support rule");
    MS_REQUIRE(opts->support == MS_SUPPORT_BLOCK || (opts->omega > 0 && opts->omega < 2 && opts->max_iter >= 0),
               MS_ERR_INVALID_ARG, "basis options out of range");
    std::vector<int> part(partition, partition + s->n);
    for (int v : part) MS_REQUIRE(v >= 0 && v < n_blocks, MS_ERR_INVALID_ARG, "partition id out of range");
    std::unique_ptr<ms_basis> b(
        create_basis(ctx, *s, part, n_blocks, opts->support, opts->precision, opts->bx, opts->by, opts->bz));
    b->omega = opts->omega;
    b->tol = opts->tol;
    b->max_iter = opts->max_iter;
    const int it = smooth_basis(ctx, *s, *b, true, b->tol, b->max_iter);
    if (iters) *iters = it;
    sync(ctx->stream);
    *out = b.release();
    return MS_OK;
    API_CATCH(ctx)
}

ms_status ms_basis_rebuild(ms_ctx *ctx, ms_system *s, ms_basis *b, int32_t *iters) {
    if (!ctx || !s || !b) return fail(ctx, MS_ERR_INVALID_ARG, "null argument");
    API_TRY
    DeviceGuard g(ctx->device);
    MS_REQUIRE(s->assembled, MS_ERR_STATE, "system not assembled");
    const int it = smooth_basis(ctx, *s, *b, true, b->tol, b->max_iter);
    if (iters) *iters = it;
    return MS_OK;
    API_CATCH(ctx)
}

ms_status ms_basis_update(ms_ctx *ctx, ms_system *s, ms_basis *b, double tol, int32_t max_iter, int32_t *iters) {
    if (!ctx || !s || !b || max_iter < 0) return fail(ctx, MS_ERR_INVALID_ARG, "bad argument");
    API_TRY
    DeviceGuard g(ctx->device);
    MS_REQUIRE(s->assembled, MS_ERR_STATE, "system not assembled");
    const int it = smooth_basis(ctx, *s, *b, false, tol, max_iter);
    if (iters) *iters = it;
    return MS_OK;
    API_CATCH(ctx)
}

ms_status ms_basis_release(ms_basis *b) {
    delete b;
    return MS_OK;
}

ms_status ms_basis_get_info(const ms_basis *b, ms_basis_info *info) {
    if (!b || !info) return MS_ERR_INVALID_ARG;
    info->M = b->M;
    info->nnz = b->nnz;
    info->max_overlap = b->B;
    info->iters = b->iters;
    info->last_increment = b->last_inc;
    return MS_OK;
}

ms_status ms_basis_get(ms_ctx *ctx, const ms_basis *b, int32_t *cptr, int32_t *cells, double *val) {
    if (!ctx || !b || !cptr || !cells || !val) return fail(ctx, MS_ERR_INVALID_ARG, "null argument");
    API_TRY
    DeviceGuard g(ctx->device);
    copy_out(cptr, b->cptr.p, (size_t)b->M + 1, ctx->stream);
    if (b->nnz) {
        copy_out(cells, b->ccell.p, (size_t)b->nnz, ctx->stream);
        copy_out(val, b->cval.p, (size_t)b->nnz, ctx->stream);
    }
    sync(ctx->stream);
    return MS_OK;
    API_CATCH(ctx)
}

ms_status ms_add_adaptive_basis(ms_ctx *ctx, ms_system *s, const double *dp, const ms_adapt_opts *opts,
                                ms_basis **out) {
    if (!ctx || !s || !dp || !opts || !out) return fail(ctx, MS_ERR_INVALID_ARG, "null argument");
    *out = nullptr;
    API_TRY
    DeviceGuard g(ctx->device);
    MS_REQUIRE(s->assembled, MS_ERR_STATE, "system not assembled");
    DBuf<double> stage;
    const double *dd = device_in(dp, s->n, stage, ctx->stream);
    MS_REQUIRE(opts->precision == MS_PREC_FP64 || opts->precision == MS_PREC_MIXED, MS_ERR_INVALID_ARG,
               "unknown precision");
    *out = adaptive_basis(ctx, *s, dd, *opts, opts->precision);
    return MS_OK;
    API_CATCH(ctx)
}

ms_status ms_galerkin(ms_ctx *ctx, ms_system *s, const ms_basis *b, int32_t precision, ms_coarse **out) {
    if (!ctx || !s || !b || !out) return fail(ctx, MS_ERR_INVALID_ARG, "null argument");
    *out = nullptr;
    API_TRY
    DeviceGuard g(ctx->device);
    MS_REQUIRE(precision == MS_PREC_FP64 || precision == MS_PREC_MIXED, MS_ERR_INVALID_ARG, "unknown precision");
    MS_REQUIRE(precision == MS_PREC_FP64 || b->precision == MS_PREC_MIXED, MS_ERR_INVALID_ARG,
               "a mixed-precision coarse operator needs a mixed-precision basis");
    *out = create_coarse(ctx, *s, *b, precision, MS_RESTRICT_GALERKIN);
    return MS_OK;
    API_CATCH(ctx)
}

ms_status ms_coarse_create(ms_ctx *ctx, ms_system *s, const ms_basis *b, int32_t precision, int32_t restriction,
                           ms_coarse **out) {
    if (!ctx || !s || !b || !out) return fail(ctx, MS_ERR_INVALID_ARG, "null argument");
    *out = nullptr;
    API_TRY
    DeviceGuard g(ctx->device);
    MS_REQUIRE(precision == MS_PREC_FP64 || precision == MS_PREC_MIXED, MS_ERR_INVALID_ARG, "unknown precision");
    MS_REQUIRE(precision == MS_PREC_FP64 || b->precision == MS_PREC_MIXED, MS_ERR_INVALID_ARG,
               "a mixed-precision coarse operator needs a mixed-precision basis");
    MS_REQUIRE(restriction == MS_RESTRICT_GALERKIN || restriction == MS_RESTRICT_FV, MS_ERR_INVALID_ARG,
               "unknown restriction");
    *out = create_coarse(ctx, *s, *b, precision, restriction);
    return MS_OK;
    API_CATCH(ctx)
}

ms_status ms_dense_inverse(ms_ctx *ctx, int32_t M, const double *A, double *X) {
    if (!ctx || !A || !X || M <= 0) return fail(ctx, MS_ERR_INVALID_ARG, "null argument or M <= 0");
    API_TRY
    DeviceGuard g(ctx->device);
    cudaStream_t st = ctx->stream;
    const size_t MM = (size_t)M * M;
    ms_coarse c;
    c.M = M;
    c.restriction = MS_RESTRICT_FV;
    c.Ac.alloc(MM);
    MS_CUDA(cudaMemcpyAsync(c.Ac.p, A, MM * sizeof(double), cudaMemcpyHostToDevice, st));
    DBuf<int> err;
    err.alloc(1);
    err.zero(st);
    dense_gj_inverse64(c, err.p, st);
    coarse_error(ctx, c, read_error_word(ctx, err.p));
    MS_CUDA(cudaMemcpyAsync(X, c.inv64.p, MM * sizeof(double), cudaMemcpyDeviceToHost, st));
    sync(st);
    return MS_OK;
    API_CATCH(ctx)
}

ms_status ms_spd_inverse(ms_ctx *ctx, int32_t M, const double *A, double *X, int32_t precision) {
    if (!ctx || !A || !X || M <= 0) return fail(ctx, MS_ERR_INVALID_ARG, "null argument or M <= 0");
    if (precision != MS_PREC_FP64 && precision != MS_PREC_MIXED) return fail(ctx, MS_ERR_INVALID_ARG, "bad precision");
    API_TRY
    DeviceGuard g(ctx->device);
    cudaStream_t st = ctx->stream;
    const size_t MM = (size_t)M * M;
    ms_coarse c;
    c.M = M;
    c.Ac.alloc(MM);
    MS_CUDA(cudaMemcpyAsync(c.Ac.p, A, MM * sizeof(double), cudaMemcpyHostToDevice, st));
    DBuf<int> err;
    err.alloc(1);
    err.zero(st);
    if (precision == MS_PREC_FP64) {
        dense_sweep_inverse64(c, err.p, st);
        coarse_error(ctx, c, read_error_word(ctx, err.p));
        MS_CUDA(cudaMemcpyAsync(X, c.inv64.p, MM * sizeof(double), cudaMemcpyDeviceToHost, st));
    } else {
        dense_sweep_inverse32(c, err.p, st);
        coarse_error(ctx, c, read_error_word(ctx, err.p));
        c.inv64.alloc(MM);
        launch_widen(c.inv32.p, c.inv64.p, (int64_t)MM, st);
        MS_CUDA(cudaMemcpyAsync(X, c.inv64.p, MM * sizeof(double), cudaMemcpyDeviceToHost, st));
    }
    sync(st);
    return MS_OK;
    API_CATCH(ctx)
}

ms_status ms_coarse_get_inverse(ms_ctx *ctx, const ms_coarse *c, double *X, int32_t *M, int32_t *fp64,
                                double *inv_error, int32_t *refine_steps) {
    if (!ctx || !c) return fail(ctx, MS_ERR_INVALID_ARG, "null argument");
    API_TRY
    DeviceGuard g(ctx->device);
    const bool d64 = c->precision != MS_PREC_MIXED || c->use64;
    if (M) *M = c->M;
    if (fp64) *fp64 = d64 ? 1 : 0;
    if (inv_error) *inv_error = c->precision == MS_PREC_MIXED ? c->inv32_error : 0.0;
    if (refine_steps) *refine_steps = d64 ? 0 : c->refine_steps;
    if (X) {
        const size_t MM = (size_t)c->M * c->M;
        cudaStream_t st = ctx->stream;
        if (d64) {
            MS_CUDA(cudaMemcpyAsync(X, c->inv64.p, MM * sizeof(double), cudaMemcpyDeviceToHost, st));
        } else {
            DBuf<double> w;
            w.alloc(MM);
            launch_widen(c->inv32.p, w.p, (int64_t)MM, st);
            MS_CUDA(cudaMemcpyAsync(X, w.p, MM * sizeof(double), cudaMemcpyDeviceToHost, st));
            sync(st);
        }
        sync(st);
    }
    return MS_OK;
    API_CATCH(ctx)
}

ms_status ms_coarse_refresh(ms_ctx *ctx, ms_system *s, ms_coarse *c) {
    if (!ctx || !s || !c) return fail(ctx, MS_ERR_INVALID_ARG, "null argument");
    API_TRY
    DeviceGuard g(ctx->device);
    galerkin_values(ctx, *s, *c->basis, *c);
    return MS_OK;
    API_CATCH(ctx)
}

ms_status ms_coarse_release(ms_coarse *c) {
    delete c;
    return MS_OK;
}

ms_status ms_coarse_get(ms_ctx *ctx, const ms_coarse *c, double *Ac, int32_t *M) {
    if (!ctx || !c) return fail(ctx, MS_ERR_INVALID_ARG, "null argument");
    API_TRY
    DeviceGuard g(ctx->device);
    if (M) *M = c->M;
    if (Ac) {
        copy_out(Ac, c->Ac.p, (size_t)c->M * c->M, ctx->stream);
        sync(ctx->stream);
    }
    return MS_OK;
    API_CATCH(ctx)
}

ms_status ms_solve(ms_ctx *ctx, ms_system *s, ms_coarse *const *stages, int32_t n_stages, const double *q,
                   double *p, const ms_solve_opts *opts, ms_solve_info *info) {
    if (!ctx || !s || !q || !p || !opts) return fail(ctx, MS_ERR_INVALID_ARG, "null argument");
    if (n_stages < 0 || (n_stages > 0 && !stages)) return fail(ctx, MS_ERR_INVALID_ARG, "bad stage list");
    const auto t0 = std::chrono::steady_clock::now();
    API_TRY
    DeviceGuard g(ctx->device);
    MS_REQUIRE(s->assembled, MS_ERR_STATE, "system not assembled");
    MS_REQUIRE(opts->tol >= 0 && opts->max_iter >= 0, MS_ERR_INVALID_ARG, "tol and max_iter must be >= 0");
    MS_REQUIRE(opts->smoother == MS_SMOOTHER_ILU0 || opts->smoother == MS_SMOOTHER_JACOBI, MS_ERR_INVALID_ARG,
               "unknown smoother");
    MS_REQUIRE(opts->precision == MS_PREC_FP64 || opts->precision == MS_PREC_MIXED, MS_ERR_INVALID_ARG,
               "unknown precision");
    MS_REQUIRE(opts->adapt_schedule >= 0 && opts->adapt_schedule <= 2, MS_ERR_INVALID_ARG, "unknown schedule");
    MS_REQUIRE(opts->outer == MS_OUTER_RICHARDSON || opts->outer == MS_OUTER_GMRES, MS_ERR_INVALID_ARG,
               "unknown outer iteration");
    MS_REQUIRE(opts->outer == MS_OUTER_RICHARDSON || opts->adapt_schedule == 0, MS_ERR_INVALID_ARG,
               "GMRES takes no adaptive schedule");
    const bool mixed = opts->precision == MS_PREC_MIXED;
    for (int l = 0; l < n_stages; ++l) {
        MS_REQUIRE(stages[l] && stages[l]->basis, MS_ERR_INVALID_ARG, "null stage");
        MS_REQUIRE(!mixed || stages[l]->precision == MS_PREC_MIXED, MS_ERR_INVALID_ARG,
                   "mixed solve needs mixed-precision coarse operators");
    }
    cudaStream_t st = ctx->stream;
    const int n = s->n;
    int Mmax = 1;
    for (int l = 0; l < n_stages; ++l) Mmax = std::max(Mmax, stages[l]->M);

    // workspace
    s->w_x.alloc(n); s->w_r.alloc(n); s->w_z.alloc(n); s->w_y.alloc(n); s->w_xprev.alloc(n);
    const int rblocks = (n + 255) / 256;
    s->w_red.alloc(rblocks + 8);
    s->w_cnt.alloc(4);
    s->w_cnt.zero(st);
    DBuf<double> norms;
    norms.alloc(4);
    bool any32 = mixed;
    for (int l = 0; l < n_stages; ++l) any32 = any32 || stages[l]->precision == MS_PREC_MIXED;
    if (mixed) { s->w_y32.alloc(n); s->w_z32.alloc(n); }
    if (any32 || opts->adapt_schedule) s->w_r32.alloc(n);

    // q (pinned: q[ref] = 0) and the initial guess
    s->w_q.alloc(n);
    MS_CUDA(cudaMemcpyAsync(s->w_q.p, q, n * sizeof(double),
                            is_device_ptr(q) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
    if (s->pinned) launch_scatter_zero(s->w_q.p, s->ref, st);
    if (opts->use_x0) {
        MS_CUDA(cudaMemcpyAsync(s->w_x.p, p, n * sizeof(double),
                                is_device_ptr(p) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
    } else {
        s->w_x.zero(st);
    }
    if (opts->smoother == MS_SMOOTHER_ILU0) ensure_ilu(ctx, *s, mixed);

    // mixed form: the residual also provides the FP32 right-hand side of the FP32 sweeps
    float *rin32 = nullptr;
    if (mixed) {
        s->w_rin32.alloc(n);
        rin32 = s->w_rin32.p;
    }
    launch_norm2(s->w_q.p, n, s->w_red.p, s->w_cnt.p, norms.p, st);
    launch_residual(*s, s->w_q.p, s->w_x.p, s->w_r.p, s->w_red.p, s->w_cnt.p, norms.p + 1, st, rin32);
    double hn[2];
    {
        double *h = (double *)ctx->pinned.get(64);
        MS_CUDA(cudaMemcpyAsync(h, norms.p, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
        sync(st);
        hn[0] = h[0]; hn[1] = h[1];
    }
    const double nq = hn[0];
    double res = nq > 0 ? hn[1] / nq : 0.0;
    if (info && info->history) info->history[0] = res;
    if (nq == 0.0) s->w_x.zero(st);

    // dynamic stage (owned by this call)
    std::unique_ptr<ms_basis> dyn_basis;
    std::unique_ptr<ms_coarse> dyn_coarse;
    const double jw = opts->jacobi_omega > 0 ? opts->jacobi_omega : 2.0 / 3.0;

    // one multistage cycle (Sec. 3): per stage, smoother then coarse correction;
    // the last stage's residual also yields ||q - A x|| in norms[1]
    auto enqueue_cycle = [&](cudaStream_t st) {
        const int total = n_stages + (dyn_coarse ? 1 : 0);
        for (int l = 0; l < total; ++l) {
            const ms_coarse &c = l < n_stages ? *stages[l] : *dyn_coarse;
            const ms_basis &b = *c.basis;
            // r holds q - A x here
            if (mixed) {
                if (opts->smoother == MS_SMOOTHER_ILU0) {
                    if (s->structured) ilu_apply32f(*s, s->w_rin32.p, s->w_y32.p, s->w_z32.p, st);
                    else ilu_apply32(*s, s->w_r.p, s->w_y32.p, s->w_z32.p, st);
                }
                else launch_jacobi32(*s, s->w_r.p, s->w_z32.p, (float)jw, st);
                launch_residual_update32(*s, s->w_r.p, s->w_r32.p, s->w_x.p, s->w_z32.p, st);
            } else {
                if (opts->smoother == MS_SMOOTHER_ILU0) ilu_apply64(*s, s->w_r.p, s->w_y.p, s->w_z.p, st);
                else launch_jacobi(*s, s->w_r.p, s->w_z.p, jw, st);
                launch_residual_update(*s, s->w_r.p, s->w_x.p, s->w_z.p, st);
            }
            const int M = c.M;
            if (c.precision == MS_PREC_MIXED) {
                if (!mixed) {   // FP64 residual restricted with the FP32 basis copy
                    launch_to_float(s->w_r.p, s->w_r32.p, n, st);
                }
                launch_restrict32(restrict_view(c), s->w_r32.p, s->w_d32.p, st);
                // coarse solve: FP32 inverse with FP64 refinement against A_c
                // (or the FP64 inverse when FP32 cannot resolve this coarse system)
                launch_widen(s->w_d32.p, s->w_d.p, M, st);
                if (c.use64) launch_gemv64(c.inv64.p, M, s->w_d.p, s->w_xc.p, st);
                else launch_coarse_refine(c, s->w_d.p, s->w_xc.p, s->w_rc.p, s->w_d32.p, s->w_xc32.p, c.refine_steps, st);
                launch_narrow(s->w_xc.p, s->w_xc32.p, M, st);
                launch_prolong32(b, n, s->w_xc32.p, s->w_x.p, st);
            } else {
                launch_restrict(restrict_view(c), s->w_r.p, s->w_d.p, st);
                launch_gemv64(c.inv64.p, M, s->w_d.p, s->w_xc.p, st);
                launch_prolong(b, n, s->w_xc.p, s->w_x.p, st);
            }
            const bool last = (l == total - 1);
            launch_residual(*s, s->w_q.p, s->w_x.p, s->w_r.p, s->w_red.p, s->w_cnt.p, last ? norms.p + 1 : nullptr,
                            st, rin32);
        }
    };
    auto grow_coarse_work = [&]() {
        s->w_d32.alloc(Mmax); s->w_xc32.alloc(Mmax);
        s->w_d.alloc(Mmax); s->w_xc.alloc(Mmax); s->w_rc.alloc(Mmax);
    };
    grow_coarse_work();

    int it = 0;
    if (opts->outer == MS_OUTER_GMRES && res > opts->tol && it < opts->max_iter) {
        // restarted flexible GMRES, right-preconditioned with one multistage
        // cycle from a zero guess (the cycle runs on w_q / w_x / w_r, so the
        // GMRES iterate lives in w_xprev and q is kept in the Krylov block)
        MS_REQUIRE(opts->adapt_schedule == 0, MS_ERR_INVALID_ARG, "GMRES takes no adaptive schedule");
        const int m = opts->restart > 0 ? std::min(opts->restart, 120) : 30;
        s->w_kry.alloc((size_t)(2 * m + 3) * n);
        double *V = s->w_kry.p, *Z = V + (size_t)(m + 1) * n, *w = Z + (size_t)m * n, *qk = w + n;
        s->w_kred.alloc((size_t)multidot_blocks(n) * (m + 8));   // block partials, vectors in groups of 8
        s->w_kh.alloc((size_t)3 * (m + 1) + 2);
        s->w_kcnt.alloc(16);                                     // one arrival counter per group of 8
        s->w_kcnt.zero(st);
        double *h1 = s->w_kh.p, *h2 = h1 + (m + 1), *hn_dev = h2 + (m + 1), *ydev = hn_dev + 1;
        double *xg = s->w_xprev.p;
        MS_CUDA(cudaMemcpyAsync(qk, s->w_q.p, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
        MS_CUDA(cudaMemcpyAsync(xg, s->w_x.p, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
        MS_CUDA(cudaMemcpyAsync(w, s->w_r.p, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
        auto precond = [&](const double *v, double *z) {
            MS_CUDA(cudaMemcpyAsync(s->w_q.p, v, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
            MS_CUDA(cudaMemcpyAsync(s->w_r.p, v, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
            s->w_x.zero(st);
            if (mixed) launch_to_float(v, s->w_rin32.p, n, st);
            enqueue_cycle(st);
            MS_CUDA(cudaMemcpyAsync(z, s->w_x.p, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
        };
        std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), gv(m + 1), y(m);
        double beta = hn[1];   // ||q - A x0||, as stored on the device
        // The whole solve as one CUDA graph: a while node over restarts whose
        // body begins the restart, runs m conditional Arnoldi steps (each step's
        // Hessenberg column, rotations and convergence test computed on the
        // device decide whether the next one runs), then updates x and tests
        // the true residual.  Same arithmetic as the host loop below, which
        // runs instead when the kernels are traced, graphs are switched off
        // (MSGB_SOLVE_GRAPH=0) or the graph cannot be built.
        auto gmres_graph = [&]() -> bool {
            const int H0 = (m + 1) * m;
            const size_t hist_n = (size_t)opts->max_iter + 1;
            s->w_kgd.alloc((size_t)H0 + 2 * m + (m + 1) + m + 2 + hist_n);
            s->w_kgi.alloc(5);
            GmresDev G{};
            G.H = s->w_kgd.p;
            G.cs = G.H + H0;
            G.sn = G.cs + m;
            G.g = G.sn + m;
            G.y = G.g + (m + 1);
            G.scal = G.y + m;
            G.res = G.scal + 1;
            G.hist = G.res + 1;
            G.k = s->w_kgi.p;
            G.it = G.k + 1;
            G.stop = G.k + 2;
            G.err = G.k + 3;
            G.restarts = G.k + 4;
            G.m = m;
            G.max_iter = opts->max_iter;
            G.nq = nq;
            G.tol = opts->tol;
            {
                const int h4[5] = {0, it, 0, 0, 0};
                MS_CUDA(cudaMemcpyAsync(s->w_kgi.p, h4, sizeof(h4), cudaMemcpyHostToDevice, st));
            }
            if (!ctx->capture) MS_CUDA(cudaStreamCreateWithFlags(&ctx->capture, cudaStreamNonBlocking));
            cudaStream_t cs = ctx->capture;
            cudaGraph_t graph = nullptr;
            cudaGraphExec_t exec = nullptr;
            bool ok = false, launched = false;
            std::vector<std::string> step_names, edge_names;
            // capture fn's launches into `into` after the nodes `deps`; returns
            // the captured sink nodes (what the next node must wait for)
            auto capture = [&](cudaGraph_t into, const std::vector<cudaGraphNode_t> &deps, auto &&fn) {
                MS_CUDA(cudaStreamBeginCaptureToGraph(cs, into, deps.empty() ? nullptr : deps.data(), nullptr,
                                                      deps.size(), cudaStreamCaptureModeRelaxed));
                std::vector<cudaGraphNode_t> sinks;
                try {
                    fn();
                    cudaStreamCaptureStatus cst;
                    const cudaGraphNode_t *dn = nullptr;
                    size_t nd = 0;
                    MS_CUDA(cudaStreamGetCaptureInfo(cs, &cst, nullptr, nullptr, &dn, nullptr, &nd));
                    sinks.assign(dn, dn + nd);
                } catch (...) {
                    cudaGraph_t dummy = nullptr;
                    cudaStreamEndCapture(cs, &dummy);
                    throw;
                }
                cudaGraph_t out = into;
                MS_CUDA(cudaStreamEndCapture(cs, &out));
                return sinks;
            };
            try {
                MS_CUDA(cudaGraphCreate(&graph, 0));
                cudaGraphConditionalHandle outer;
                MS_CUDA(cudaGraphConditionalHandleCreate(&outer, graph, 1, cudaGraphCondAssignDefault));
                cudaGraphNodeParams wp = {};
                wp.type = cudaGraphNodeTypeConditional;
                wp.conditional.handle = outer;
                wp.conditional.type = cudaGraphCondTypeWhile;
                wp.conditional.size = 1;
                cudaGraphNode_t wnode;
                MS_CUDA(cudaGraphAddNode(&wnode, graph, nullptr, nullptr, 0, &wp));
                cudaGraph_t body = wp.conditional.phGraph_out[0];
                // one handle per conditional step, kept on the device for the
                // kernels that open the next step
                std::vector<cudaGraphConditionalHandle> hstep(m);
                for (int j = 0; j < m; ++j)
                    MS_CUDA(cudaGraphConditionalHandleCreate(&hstep[j], body, 0, cudaGraphCondAssignDefault));
                static_assert(sizeof(cudaGraphConditionalHandle) == sizeof(unsigned long long), "handle size");
                s->w_kgh.alloc(m);
                MS_CUDA(cudaMemcpyAsync(s->w_kgh.p, hstep.data(), sizeof(unsigned long long) * m,
                                        cudaMemcpyHostToDevice, st));
                const cudaGraphConditionalHandle *hsteps = (const cudaGraphConditionalHandle *)s->w_kgh.p;
                // restart begin: beta = ||r||, g = beta e_0, V_0 = r / beta (the
                // kernels that set a handle sit in the graph of the node they
                // steer or in a body graph below it, never in a child graph)
                profile_record_begin();
                std::vector<cudaGraphNode_t> prevs = capture(body, {}, [&]() {
                    launch_gmres_begin(G, norms.p + 1, hsteps, cs);
                    launch_scale_dev(n, w, G.scal, V, cs);
                });
                edge_names = profile_record_end();
                for (int j = 0; j < m; ++j) {
                    cudaGraphNodeParams ip = {};
                    ip.type = cudaGraphNodeTypeConditional;
                    ip.conditional.handle = hstep[j];
                    ip.conditional.type = cudaGraphCondTypeIf;
                    ip.conditional.size = 1;
                    cudaGraphNode_t inode;
                    MS_CUDA(cudaGraphAddNode(&inode, body, prevs.data(), nullptr, prevs.size(), &ip));
                    if (j == 0) profile_record_begin();
                    capture(ip.conditional.phGraph_out[0], {}, [&]() {
                        const double *vk = V + (size_t)j * n;
                        double *zk = Z + (size_t)j * n;
                        // the cycle launches on the capture stream
                        std::swap(st, cs);
                        try {
                            precond(vk, zk);
                        } catch (...) {
                            std::swap(st, cs);
                            throw;
                        }
                        std::swap(st, cs);
                        launch_spmv(*s, zk, w, cs);
                        launch_multidot(n, j + 1, V, w, s->w_kred.p, s->w_kcnt.p, h1, cs);
                        launch_multiaxpy(n, j + 1, V, h1, -1.0, w, cs);
                        launch_multidot(n, j + 1, V, w, s->w_kred.p, s->w_kcnt.p, h2, cs);
                        launch_multiaxpy_norm(n, j + 1, V, h2, -1.0, w, s->w_red.p, s->w_cnt.p, hn_dev, cs);
                        launch_gmres_step(G, j, h1, h2, hn_dev, hsteps, cs);
                        launch_scale_dev(n, w, G.scal, V + (size_t)(j + 1) * n, cs);
                    });
                    if (j == 0) step_names = profile_record_end();
                    prevs.assign(1, inode);
                }
                // restart end: x += Z y, true residual, continue while above tol
                profile_record_begin();
                capture(body, prevs, [&]() {
                    launch_gmres_solve(G, cs);
                    launch_multiaxpy(n, m, Z, G.y, 1.0, xg, cs, G.k);
                    launch_residual(*s, qk, xg, w, s->w_red.p, s->w_cnt.p, norms.p + 1, cs, nullptr);
                    launch_gmres_restart(G, norms.p + 1, outer, cs);
                });
                {
                    auto e2 = profile_record_end();
                    edge_names.insert(edge_names.end(), e2.begin(), e2.end());
                }
                MS_CUDA(cudaGraphInstantiate(&exec, graph, 0));
                launched = true;
                MS_CUDA(cudaGraphLaunch(exec, st));
                int hi[4];
                double hres = 0.0;
                MS_CUDA(cudaMemcpyAsync(hi, s->w_kgi.p, sizeof(hi), cudaMemcpyDeviceToHost, st));
                MS_CUDA(cudaMemcpyAsync(&hres, G.res, sizeof(double), cudaMemcpyDeviceToHost, st));
                sync(st);
                if (hi[3]) throw Error{MS_ERR_CUDA, "GMRES: Arnoldi vector or residual became NaN"};
                const int it_end = hi[1];
                const int steps = it_end - it;
                // launches were counted once per captured node: count what ran
                // (steps Arnoldi steps, about ceil(steps / m) restarts)
                profile_add_launches(step_names, (int64_t)steps - m);
                profile_add_launches(edge_names, (int64_t)std::max(1, (steps + m - 1) / m) - 1);
                if (info && info->history && steps > 0)
                    copy_out(info->history + it + 1, G.hist + it + 1, (size_t)steps, st);
                it = it_end;
                res = hres;
                ok = true;
            } catch (const Error &) {
                profile_record_end();
                if (launched) {
                    if (exec) cudaGraphExecDestroy(exec);
                    if (graph) cudaGraphDestroy(graph);
                    throw;
                }
                cudaGetLastError();   // the graph could not be built: the host loop runs instead
                ok = false;
            }
            if (exec) cudaGraphExecDestroy(exec);
            if (graph) cudaGraphDestroy(graph);
            return ok;
        };
        // Opt-in (MSGB_GMRES_GRAPH=1): the solve captures a new graph on each
        // call, which must not meet another host thread's device-wide
        // synchronisation or allocator release, so it is kept for callers that
        // drive the device from one thread.
        const char *gmres_env = std::getenv("MSGB_GMRES_GRAPH");
        const char *graph_env = std::getenv("MSGB_SOLVE_GRAPH");
        if (gmres_env && gmres_env[0] == '1' && !(graph_env && graph_env[0] == '0') && !profile_enabled() &&
            gmres_graph()) {
            if (!(res == res)) throw Error{MS_ERR_CUDA, "residual became NaN"};
            beta = res * nq;
            if (opts->smoother == MS_SMOOTHER_ILU0) check_sweep_errors(ctx, s);
        }
        while (res > opts->tol && it < opts->max_iter) {
            launch_scale(n, w, 1.0 / beta, V, st);
            std::fill(gv.begin(), gv.end(), 0.0);
            gv[0] = beta;
            int k = 0;
            while (k < m && it < opts->max_iter) {
                const double *vk = V + (size_t)k * n;
                double *zk = Z + (size_t)k * n;
                precond(vk, zk);
                launch_spmv(*s, zk, w, st);
                // classical Gram-Schmidt, twice
                launch_multidot(n, k + 1, V, w, s->w_kred.p, s->w_kcnt.p, h1, st);
                launch_multiaxpy(n, k + 1, V, h1, -1.0, w, st);
                launch_multidot(n, k + 1, V, w, s->w_kred.p, s->w_kcnt.p, h2, st);
                launch_multiaxpy_norm(n, k + 1, V, h2, -1.0, w, s->w_red.p, s->w_cnt.p, hn_dev, st);
                double *hh = (double *)ctx->pinned.get(sizeof(double) * (2 * (m + 1) + 1));
                MS_CUDA(cudaMemcpyAsync(hh, h1, sizeof(double) * (2 * (m + 1) + 1), cudaMemcpyDeviceToHost, st));
                sync(st);
                for (int i = 0; i <= k; ++i) H[(size_t)i * m + k] = hh[i] + hh[(m + 1) + i];
                const double hn = hh[2 * (m + 1)];
                if (!(hn == hn)) throw Error{MS_ERR_CUDA, "GMRES: Arnoldi vector became NaN"};
                H[(size_t)(k + 1) * m + k] = hn;
                if (hn > 0.0) launch_scale(n, w, 1.0 / hn, V + (size_t)(k + 1) * n, st);
                gmres_givens(H.data(), m, k, cs.data(), sn.data(), gv.data());
                ++k;
                ++it;
                res = std::fabs(gv[k]) / nq;
                if (info && info->history) info->history[it] = res;
                if (res <= opts->tol || hn == 0.0) break;
            }
            gmres_back_solve(H.data(), m, k, gv.data(), y.data());
            MS_CUDA(cudaMemcpyAsync(ydev, y.data(), sizeof(double) * k, cudaMemcpyHostToDevice, st));
            launch_multiaxpy(n, k, Z, ydev, 1.0, xg, st);
            launch_residual(*s, qk, xg, w, s->w_red.p, s->w_cnt.p, norms.p + 1, st, nullptr);
            beta = read_norm(ctx, norms.p + 1);
            res = beta / nq;
            if (!(res == res)) throw Error{MS_ERR_CUDA, "residual became NaN"};
            if (info && info->history) info->history[it] = res;
            if (opts->smoother == MS_SMOOTHER_ILU0) check_sweep_errors(ctx, s);
        }
        if (info && info->dyn_blocks)
            for (int k = 0; k < it; ++k) info->dyn_blocks[k] = 0;
        MS_CUDA(cudaMemcpyAsync(s->w_x.p, xg, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
        MS_CUDA(cudaMemcpyAsync(s->w_q.p, qk, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
    }

    // Cycles that rebuild the dynamic stage (Sec. 5.1 schedules), or run while
    // kernels are traced, are driven from the host with one residual read per
    // cycle; all other cycles run as one CUDA graph with a device-side while
    // loop (MSGB_SOLVE_GRAPH=0 keeps every cycle on the host).
    const char *genv = std::getenv("MSGB_SOLVE_GRAPH");
    const bool graphs = !(genv && genv[0] == '0') && !profile_enabled();
    while (opts->outer != MS_OUTER_GMRES && res > opts->tol && it < opts->max_iter) {
        const bool rebuilds = opts->adapt_schedule == 1 || (opts->adapt_schedule == 2 && it < 2);
        if (graphs && !rebuilds) break;
        if (opts->adapt_schedule) MS_CUDA(cudaMemcpyAsync(s->w_xprev.p, s->w_x.p, n * sizeof(double),
                                                          cudaMemcpyDeviceToDevice, st));
        enqueue_cycle(st);
        if (info && info->dyn_blocks) info->dyn_blocks[it] = dyn_coarse ? dyn_coarse->M : 0;
        ++it;
        res = read_norm(ctx, norms.p + 1) / nq;
        if (!(res == res)) throw Error{MS_ERR_CUDA, "residual became NaN"};
        if (info && info->history) info->history[it] = res;
        if (opts->smoother == MS_SMOOTHER_ILU0) check_sweep_errors(ctx, s);
        if (opts->adapt_schedule && res > opts->tol &&
            (opts->adapt_schedule == 1 || (opts->adapt_schedule == 2 && it <= 2))) {
            s->w_part.alloc(n);
            launch_sub(s->w_x.p, s->w_xprev.p, s->w_part.p, n, st);
            const int dprec = mixed ? MS_PREC_MIXED : MS_PREC_FP64;
            dyn_coarse.reset();
            dyn_basis.reset(adaptive_basis(ctx, *s, s->w_part.p, opts->adapt, dprec));
            dyn_coarse.reset(create_coarse(ctx, *s, *dyn_basis, dprec, MS_RESTRICT_GALERKIN));
            Mmax = std::max(Mmax, dyn_basis->M);
            grow_coarse_work();
        }
    }
    if (opts->outer != MS_OUTER_GMRES && res > opts->tol && it < opts->max_iter) {
        // remaining cycles: while (res > tol && it < max_iter) { cycle } on the device
        DBuf<int> ctl_it;
        DBuf<double> ctl_res, hist;
        ctl_it.alloc(1);
        ctl_res.alloc(1);
        MS_CUDA(cudaMemcpyAsync(ctl_it.p, &it, sizeof(int), cudaMemcpyHostToDevice, st));
        if (info && info->history) hist.alloc((size_t)opts->max_iter + 1);
        cudaGraph_t graph = nullptr, body = nullptr;
        cudaGraphExec_t exec = nullptr;
        std::vector<std::string> captured;
        try {
            MS_CUDA(cudaGraphCreate(&graph, 0));
            cudaGraphConditionalHandle handle;
            MS_CUDA(cudaGraphConditionalHandleCreate(&handle, graph, 1, cudaGraphCondAssignDefault));
            cudaGraphNodeParams cp = {};
            cp.type = cudaGraphNodeTypeConditional;
            cp.conditional.handle = handle;
            cp.conditional.type = cudaGraphCondTypeWhile;
            cp.conditional.size = 1;
            cudaGraphNode_t node;
            MS_CUDA(cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &cp));
            body = cp.conditional.phGraph_out[0];
            // captured on a private stream (the caller's may be the legacy default
            // stream, which cannot be captured); the graph is launched on the caller's
            if (!ctx->capture) MS_CUDA(cudaStreamCreateWithFlags(&ctx->capture, cudaStreamNonBlocking));
            cudaStream_t cs = ctx->capture;
            profile_record_begin();
            MS_CUDA(cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
            try {
                enqueue_cycle(cs);
                launch_cycle_control(norms.p, opts->tol, opts->max_iter, ctl_it.p, ctl_res.p, hist.p, handle, cs);
            } catch (...) {
                cudaGraph_t dummy = nullptr;
                cudaStreamEndCapture(cs, &dummy);
                throw;
            }
            MS_CUDA(cudaStreamEndCapture(cs, &body));
            captured = profile_record_end();
            MS_CUDA(cudaGraphInstantiate(&exec, graph, 0));
            MS_CUDA(cudaGraphLaunch(exec, st));
            int it_end = it;
            double res_end = 0;
            {
                char *h = (char *)ctx->pinned.get(64);
                MS_CUDA(cudaMemcpyAsync(h, ctl_it.p, sizeof(int), cudaMemcpyDeviceToHost, st));
                MS_CUDA(cudaMemcpyAsync(h + 8, ctl_res.p, sizeof(double), cudaMemcpyDeviceToHost, st));
                sync(st);
                std::memcpy(&it_end, h, sizeof(int));
                std::memcpy(&res_end, h + 8, sizeof(double));
            }
            if (it_end - it > 1) profile_add_launches(captured, it_end - it - 1);
            if (info && info->history && it_end > it)
                copy_out(info->history + it + 1, hist.p + it + 1, (size_t)(it_end - it), st);
            if (info && info->dyn_blocks)
                for (int k = it; k < it_end; ++k) info->dyn_blocks[k] = dyn_coarse ? dyn_coarse->M : 0;
            it = it_end;
            res = res_end;
        } catch (...) {
            profile_record_end();
            if (exec) cudaGraphExecDestroy(exec);
            if (graph) cudaGraphDestroy(graph);
            throw;
        }
        cudaGraphExecDestroy(exec);
        cudaGraphDestroy(graph);
        if (!(res == res)) throw Error{MS_ERR_CUDA, "residual became NaN"};
        if (opts->smoother == MS_SMOOTHER_ILU0) check_sweep_errors(ctx, s);
    }
    for (int l = 0; l < n_stages; ++l) check_refine_errors(ctx, stages[l]);
    if (dyn_coarse) check_refine_errors(ctx, dyn_coarse.get());
    copy_out(p, s->w_x.p, n, st);
    sync(st);
    const bool conv = res <= opts->tol;
    if (info) {
        info->iters = it;
        info->converged = conv ? 1 : 0;
        info->rel_residual = res;
        info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
    return conv ? MS_OK : fail(ctx, MS_ERR_NOT_CONVERGED, "iteration cap reached");
    API_CATCH(ctx)
}

// MSGB_BATCH_SMOOTH=0 re-smooths each member's basis on its own worker
// instead of the batched launch (for comparison).
bool batch_smoothing_enabled() {
    const char *e = std::getenv("MSGB_BATCH_SMOOTH");
    return !(e && std::string(e) == "0");
}

ms_status ms_set_batch_tuning(ms_ctx *ctx, int32_t tile_cells, int32_t ctas_per_sm) {
    if (!ctx) return fail(ctx, MS_ERR_INVALID_ARG, "null argument");
    if (tile_cells < 256 || tile_cells > 16384 || tile_cells % 256 != 0 || ctas_per_sm < 1 || ctas_per_sm > 8)
        return fail(ctx, MS_ERR_INVALID_ARG, "tile_cells must be a multiple of 256 in [256, 16384], ctas_per_sm in [1, 8]");
    ctx->batch_tile = tile_cells;
    ctx->batch_ctas_per_sm = ctas_per_sm;
    return MS_OK;
}

ms_status ms_basis_rebuild_batch(ms_ctx *ctx, ms_system *const *sys, ms_basis *const *bases, int32_t n,
                                 int32_t *iters) {
    if (!ctx || n < 0 || (n > 0 && (!sys || !bases))) return fail(ctx, MS_ERR_INVALID_ARG, "null argument");
    if (n == 0) return MS_OK;
    API_TRY
    DeviceGuard g(ctx->device);
    std::vector<ms_system *> vs(sys, sys + n);
    std::vector<ms_basis *> vb(bases, bases + n);
    for (int m = 0; m < n; ++m) {
        MS_REQUIRE(vs[m] && vb[m], MS_ERR_INVALID_ARG, "null member");
        MS_REQUIRE(vs[m]->assembled, MS_ERR_STATE, "system not assembled");
        for (int k = 0; k < m; ++k)
            MS_REQUIRE(vs[k] != vs[m] && vb[k] != vb[m], MS_ERR_INVALID_ARG, "members must be distinct");
    }
    std::vector<char> tk;
    smooth_batch(ctx, vs, vb, tk);
    for (int m = 0; m < n; ++m) {
        if (!tk[m]) smooth_basis(ctx, *vs[m], *vb[m], true, vb[m]->tol, vb[m]->max_iter);
        if (iters) iters[m] = vb[m]->iters;
    }
    sync(ctx->stream);
    return MS_OK;
    API_CATCH(ctx)
}

ms_status ms_solve_batch(ms_ctx *ctx, ms_batch_member *members, int32_t n_members, const ms_solve_opts *opts,
                         int32_t n_workers) {
    if (!ctx || !opts || n_members < 0 || (n_members > 0 && !members))
        return fail(ctx, MS_ERR_INVALID_ARG, "null argument");
    if (n_members == 0) return MS_OK;
    API_TRY
    DeviceGuard g(ctx->device);
    for (int m = 0; m < n_members; ++m) {
        MS_REQUIRE(members[m].sys && members[m].q && members[m].p, MS_ERR_INVALID_ARG, "incomplete member");
        members[m].status = MS_ERR_STATE;
        members[m].basis_iters = 0;
    }
    const int W = std::max(1, std::min(n_members, n_workers > 0 ? n_workers : 16));
    while ((int)ctx->workers.size() < W) {
        std::unique_ptr<ms_ctx> w(new ms_ctx());
        w->device = ctx->device;
        w->sm_count = ctx->sm_count;
        MS_CUDA(cudaStreamCreateWithFlags(&w->stream, cudaStreamNonBlocking));
        w->owns_stream = true;
        ctx->workers.push_back(std::move(w));
    }
    // every member's basis re-smoothing in one persistent launch on the
    // caller's stream (members it cannot take re-smooth on their worker)
    std::vector<char> taken(n_members, 0);
    {
        std::vector<ms_system *> bs;
        std::vector<ms_basis *> bb;
        std::vector<int> at;
        for (int m = 0; m < n_members; ++m)
            if (members[m].rebuild) {
                MS_REQUIRE(members[m].sys->assembled, MS_ERR_STATE, "member system not assembled");
                bs.push_back(members[m].sys);
                bb.push_back(members[m].rebuild);
                at.push_back(m);
            }
        if (!bs.empty() && batch_smoothing_enabled()) {
            std::vector<char> tk;
            smooth_batch(ctx, bs, bb, tk);
            for (size_t k = 0; k < at.size(); ++k)
                if (tk[k]) {
                    taken[at[k]] = 1;
                    members[at[k]].basis_iters = bb[k]->iters;
                }
        }
    }
    // order: earlier work on the caller's stream -> all workers -> later work on it
    cudaEvent_t ev;
    MS_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    MS_CUDA(cudaEventRecord(ev, ctx->stream));
    for (int w = 0; w < W; ++w) MS_CUDA(cudaStreamWaitEvent(ctx->workers[w]->stream, ev, 0));
    // largest members first
    std::vector<int> order(n_members);
    for (int m = 0; m < n_members; ++m) order[m] = m;
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int b) { return members[a].sys->n > members[b].sys->n; });
    std::atomic<int> next{0};
    auto work = [&](ms_ctx *wc) {
        cudaSetDevice(wc->device);
        for (int k = next++; k < n_members; k = next++) {
            ms_batch_member &mb = members[order[k]];
            ms_status st = MS_OK;
            if (mb.rebuild) {
                if (!taken[order[k]]) st = ms_basis_rebuild(wc, mb.sys, mb.rebuild, &mb.basis_iters);
                for (int l = 0; st == MS_OK && l < mb.n_stages; ++l)
                    if (mb.stages[l] && mb.stages[l]->basis == mb.rebuild) st = ms_coarse_refresh(wc, mb.sys, mb.stages[l]);
            }
            if (st == MS_OK) st = ms_solve(wc, mb.sys, mb.stages, mb.n_stages, mb.q, mb.p, opts, mb.info);
            mb.status = st;
        }
    };
    std::vector<std::thread> pool;
    for (int w = 1; w < W; ++w) pool.emplace_back(work, ctx->workers[w].get());
    work(ctx->workers[0].get());
    for (auto &t : pool) t.join();
    for (int w = 0; w < W; ++w) {
        MS_CUDA(cudaEventRecord(ev, ctx->workers[w]->stream));
        MS_CUDA(cudaStreamWaitEvent(ctx->stream, ev, 0));
    }
    cudaEventDestroy(ev);
    ms_status worst = MS_OK;
    for (int m = 0; m < n_members; ++m) {
        const ms_status st = members[m].status;
        if (st != MS_OK && st != MS_ERR_NOT_CONVERGED) {
            ctx->err = "member " + std::to_string(m) + ": " + ms_status_string(st);
            return st;
        }
        if (st == MS_ERR_NOT_CONVERGED) worst = st;
    }
    return worst;
    API_CATCH(ctx)
}

ms_status ms_total_mobility(ms_ctx *ctx, const ms_system *s, const ms_fluid *fl, const double *S, double *lam) {
    if (!ctx || !s || !fl || !S || !lam) return fail(ctx, MS_ERR_INVALID_ARG, "null argument");
    API_TRY
    DeviceGuard g(ctx->device);
    MS_REQUIRE(fl->mu_w > 0 && fl->mu_o > 0 && fl->s_wc + fl->s_or < 1.0, MS_ERR_INVALID_ARG, "bad fluid");
    cudaStream_t st = ctx->stream;
    const double par[6] = {fl->mu_w, fl->mu_o, fl->n_w, fl->n_o, fl->s_wc, fl->s_or};
    DBuf<double> stage, out;
    const double *Sd = device_in(S, s->n, stage, st);
    double *ld = lam;
    if (!is_device_ptr(lam)) {
        out.alloc(s->n);
        ld = out.p;
    }
    launch_total_mobility(s->n, par, Sd, ld, st);
    if (ld != lam) copy_out(lam, ld, s->n, st);
    sync(st);
    return MS_OK;
    API_CATCH(ctx)
}

ms_status ms_transport_step(ms_ctx *ctx, ms_system *s, const ms_fluid *fl, const double *p, const double *q,
                            double dt, double *S, int32_t *substeps) {
    if (!ctx || !s || !fl || !p || !q || !S) return fail(ctx, MS_ERR_INVALID_ARG, "null argument");
    API_TRY
    DeviceGuard g(ctx->device);
    MS_REQUIRE(s->assembled, MS_ERR_STATE, "system not assembled");
    MS_REQUIRE(fl->mu_w > 0 && fl->mu_o > 0 && fl->s_wc + fl->s_or < 1.0 && fl->porosity > 0 && fl->cfl > 0 &&
                   dt >= 0,
               MS_ERR_INVALID_ARG, "bad fluid or time step");
    cudaStream_t st = ctx->stream;
    const int n = s->n;
    const double par[6] = {fl->mu_w, fl->mu_o, fl->n_w, fl->n_o, fl->s_wc, fl->s_or};
    DBuf<double> sp, sq;
    const double *pd = device_in(p, n, sp, st);
    const double *qd = device_in(q, n, sq, st);
    s->w_tu.alloc(std::max(s->nf, 1));
    s->w_ts.alloc((size_t)3 * n);
    double *S0 = s->w_ts.p, *S1 = S0 + n, *fw = S1 + n;
    MS_CUDA(cudaMemcpyAsync(S0, S, n * sizeof(double), is_device_ptr(S) ? cudaMemcpyDeviceToDevice
                                                                         : cudaMemcpyHostToDevice, st));
    launch_face_flux(*s, pd, s->w_tu.p, st);
    const double pv = fl->porosity * s->dx * s->dy * s->dz;
    s->w_max.alloc(1);
    const unsigned long long inf_bits = 0x7FF0000000000000ull;   // +infinity
    MS_CUDA(cudaMemcpyAsync(s->w_max.p, &inf_bits, sizeof(inf_bits), cudaMemcpyHostToDevice, st));
    launch_outflow_limit(*s, s->w_tu.p, qd, pv, s->w_max.p, st);
    unsigned long long *h = (unsigned long long *)ctx->pinned.get(64);
    MS_CUDA(cudaMemcpyAsync(h, s->w_max.p, sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
    sync(st);
    double tmin;
    std::memcpy(&tmin, h, sizeof(double));
    const double slope = frac_flow_max_slope(fl->mu_w, fl->mu_o, fl->n_w, fl->n_o, fl->s_wc, fl->s_or);
    const double hmax = slope > 0 ? fl->cfl * tmin / slope : INFINITY;
    int nsub = 1;
    if (dt > 0 && std::isfinite(hmax)) {
        const double k = std::ceil(dt / hmax);
        MS_REQUIRE(k < 1e7, MS_ERR_INVALID_ARG, "time step needs more than 1e7 transport substeps");
        nsub = std::max(1, (int)k);
    }
    const double hs = dt / nsub;
    // the upstream weights once, then every substep (one launch where the
    // grid can be resident at once)
    launch_transport_coef(*s, s->w_tu.p, qd, st);
    launch_transport_run(*s, par, nsub, hs / pv, S0, S1, fw, st);
    MS_CUDA(cudaMemcpyAsync(S, S0, n * sizeof(double), is_device_ptr(S) ? cudaMemcpyDeviceToDevice
                                                                         : cudaMemcpyDeviceToHost, st));
    sync(st);
    if (const int e = read_error_word(ctx, s->sync.p + 3)) {
        MS_CUDA(cudaMemsetAsync(s->sync.p + 3, 0, sizeof(int), st));
        s->tbar_ready = false;   // a barrier that gave up: the counters start afresh next time
        throw Error{(e & kErrTimeout) ? MS_ERR_TIMEOUT : MS_ERR_CUDA, "a transport substep barrier wait ran out"};
    }
    if (substeps) *substeps = nsub;
    return MS_OK;
    API_CATCH(ctx)
}

ms_status ms_profile_enable(int32_t on) {
    profile_enable(on != 0);
    return MS_OK;
}

ms_status ms_profile_reset(void) {
    profile_reset();
    return MS_OK;
}

ms_status ms_profile_read(ms_kernel_stat *out, int32_t capacity, int32_t *count, int64_t *total_launches) {
    if (capacity < 0 || (capacity > 0 && !out)) return MS_ERR_INVALID_ARG;
    const int k = profile_read(out, capacity, total_launches);
    if (count) *count = k;
    return MS_OK;
}

}  // extern "C"
