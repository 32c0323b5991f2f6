// Allocation-free ILU(0) application: ms_ilu_apply_noalloc (include/ms.h).
//
// All scratch of the call -- the sweep words, the per-row completion flags
// and the intermediate vector of the forward sweep -- lives in one
// file-scope device array of fixed size, so the call performs no device or
// host allocation.  In host code the array's name is only a host-side
// stand-in: its device address is looked up once per device with
// cudaGetSymbolAddress (with that device current) and passed to the kernels.
#include <mutex>

#include "ms_internal.h"

namespace {

constexpr int64_t kMaxRows = 1 << 20;                            // largest system served
constexpr size_t kSyncBytes = 256;                               // sweep words (8 ints), padded
constexpr size_t kFlagBytes = (size_t)kMaxRows * sizeof(int);    // per-row completion flags
constexpr size_t kVecBytes = (size_t)kMaxRows * sizeof(double);  // forward-sweep vector
constexpr size_t kScratchBytes = kSyncBytes + kFlagBytes + kVecBytes;

static __device__ __align__(256) unsigned char g_ilu_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void *g_scratch_addr[kMaxDevices] = {};

// Device address of g_ilu_scratch on `dev` (current); first call per device does the lookup.
void *scratch_address(int dev) {
    if (dev < 0 || dev >= kMaxDevices) throw msgb::Error{MS_ERR_INVALID_ARG, "device index out of range"};
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_ilu_scratch);
        if (e != cudaSuccess || !p)
            throw msgb::Error{MS_ERR_CUDA, std::string("cudaGetSymbolAddress of the static scratch failed: ") +
                                               cudaGetErrorString(e)};
        g_scratch_addr[dev] = p;
    }
    return g_scratch_addr[dev];
}

bool on_device(const void *p, int dev) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) && a.device == dev;
}

}  // namespace

extern "C" ms_status ms_ilu_apply_noalloc(ms_ctx *ctx, const ms_system *sys, const double *r, double *z) {
    if (!ctx || !sys || !r || !z) {
        if (ctx) ctx->err = "null argument";
        return MS_ERR_INVALID_ARG;
    }
    try {
        int prev = -1;
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        struct Restore {
            int d;
            ~Restore() {
                if (d >= 0) cudaSetDevice(d);
            }
        } restore{prev != ctx->device ? prev : -1};
        if (prev != ctx->device) MS_CUDA(cudaSetDevice(ctx->device));
        MS_REQUIRE((int64_t)sys->n <= kMaxRows, MS_ERR_INVALID_ARG,
                   "ms_ilu_apply_noalloc serves at most 1048576 unknowns; this system has " + std::to_string(sys->n));
        MS_REQUIRE(on_device(r, ctx->device) && on_device(z, ctx->device), MS_ERR_INVALID_ARG,
                   "ms_ilu_apply_noalloc needs r and z in device memory of the context's device");
        MS_REQUIRE(sys->assembled && sys->ilu64_valid, MS_ERR_STATE,
                   "ms_ilu_apply_noalloc needs the FP64 ILU(0) factors of the current assembly (run ms_ilu_apply or "
                   "ms_solve first)");
        unsigned char *base = static_cast<unsigned char *>(scratch_address(ctx->device));
        int *sync = reinterpret_cast<int *>(base);
        int *flags = reinterpret_cast<int *>(base + kSyncBytes);
        double *y = reinterpret_cast<double *>(base + kSyncBytes + kFlagBytes);
        cudaStream_t st = ctx->stream;
        // ticket, done counter and error word start at zero; the sweep counter
        // sync[0] keeps growing across calls so stale flags never match
        MS_CUDA(cudaMemsetAsync(sync + 1, 0, 3 * sizeof(int), st));
        msgb::launch_ilu_apply64_scratch(*sys, r, y, z, flags, sync, st);
        int err = 0;
        MS_CUDA(cudaMemcpyAsync(&err, sync + 3, sizeof(int), cudaMemcpyDeviceToHost, st));
        MS_CUDA(cudaStreamSynchronize(st));
        if (err & msgb::kErrTimeout) throw msgb::Error{MS_ERR_TIMEOUT, "a level-ordered sweep wait ran out"};
        if (err) throw msgb::Error{MS_ERR_CUDA, "device error word " + std::to_string(err)};
        return MS_OK;
    } catch (const msgb::Error &e) {
        ctx->err = e.what;
        return e.status;
    } catch (...) {
        ctx->err = "unexpected exception";
        return MS_ERR_CUDA;
    }
}
