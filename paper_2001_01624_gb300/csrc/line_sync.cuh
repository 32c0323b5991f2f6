// Device helpers shared by the structured ILU(0) line sweeps: shared-memory
// addresses, mbarriers, bulk copies into shared memory, cluster barriers and
// ranks, device time, tagged words, and bounded waits.
#pragma once

#include "ms_internal.h"

namespace msgb {
namespace {

// levels of the shuffle scan over L lanes, and the per-line table of the
// scan's multipliers (one per level and lane)
__host__ __device__ constexpr int scan_levels(int L) { return L >= 32 ? 5 : L >= 16 ? 4 : L >= 8 ? 3 : L >= 4 ? 2 : 1; }
__host__ __device__ constexpr int scan_table(int L) { return L * scan_levels(L); }

__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mb_init(unsigned bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mb_expect(unsigned bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mb_try(unsigned bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ bool mb_test(unsigned bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{ .reg .pred p; mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ unsigned map_cta(unsigned addr, unsigned rank) {
    unsigned r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
    return r;
}
// relaxed arrivals: no ordering of earlier memory operations is needed (the
// data they guard travels with transaction bytes, or was consumed already)
__device__ __forceinline__ void mb_arrive_relaxed(unsigned bar) {
    asm volatile("mbarrier.arrive.relaxed.cta.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void mb_arrive_relaxed_remote(unsigned cbar) {
    asm volatile("mbarrier.arrive.relaxed.cluster.shared::cluster.b64 _, [%0];" ::"r"(cbar) : "memory");
}
__device__ __forceinline__ void mb_expect_relaxed(unsigned bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.relaxed.cta.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
// asynchronous store into the shared memory of a CTA of the cluster (this one
// included), counted as transaction bytes on that CTA's barrier
__device__ __forceinline__ void st_async2(unsigned addr, float a, float b, unsigned cbar) {
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v2.f32 [%0], {%1, %2}, [%3];" ::"r"(addr), "f"(a),
                 "f"(b), "r"(cbar)
                 : "memory");
}
__device__ __forceinline__ void st_async2(unsigned addr, double a, double b, unsigned cbar) {
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v2.f64 [%0], {%1, %2}, [%3];" ::"r"(addr), "d"(a),
                 "d"(b), "r"(cbar)
                 : "memory");
}
// Rows handed across a cluster boundary go through global memory: each value
// as 8-byte words that carry the launch's tag in their upper half (FP32: the
// value's bits; FP64: its low and high halves), one slot per line, written once
// per launch, so no slot is reused within a launch and a reader (the relay
// warp) knows a value is there when its tag is.
__device__ __forceinline__ void ring_put(unsigned long long *w, float v, unsigned tag) {
    *(volatile unsigned long long *)w = (unsigned long long)__float_as_uint(v) | ((unsigned long long)tag << 32);
}
__device__ __forceinline__ void ring_put(unsigned long long *w, double v, unsigned tag) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    *(volatile unsigned long long *)w = (b & 0xffffffffull) | ((unsigned long long)tag << 32);
    *(volatile unsigned long long *)(w + 1) = (b >> 32) | ((unsigned long long)tag << 32);
}
template <typename T>
__host__ __device__ constexpr int ring_words() { return sizeof(T) == 8 ? 2 : 1; }

__device__ __forceinline__ void bulk_g2s(unsigned dst, const void *src, unsigned bytes, unsigned bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}
__device__ __forceinline__ void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ unsigned cluster_rank() {
    unsigned r;
    asm volatile("mov.u32 %0, %cluster_ctarank;" : "=r"(r));
    return r;
}

template <typename T>
__device__ __forceinline__ T shfl_up(T v, int d) {
    return __shfl_up_sync(0xffffffffu, v, d);
}

// the four packed coefficients of one cell
template <typename T>
struct Coef4 {
    T a, b, c, d;
};
__device__ __forceinline__ Coef4<float> load_coef(const float *p) {
    const float4 v = *reinterpret_cast<const float4 *>(p);
    return {v.x, v.y, v.z, v.w};
}
__device__ __forceinline__ Coef4<double> load_coef(const double *p) {
    const double2 u = reinterpret_cast<const double2 *>(p)[0], v = reinterpret_cast<const double2 *>(p)[1];
    return {u.x, u.y, v.x, v.y};
}

// rhs window: the line plus 16 bytes of alignment slack on each side, a multiple of 16 bytes
__host__ __device__ constexpr int rhs_win(int nx, int esz) {
    return (nx + 3 * (16 / esz) + 16 / esz - 1) / (16 / esz) * (16 / esz);
}

// wait for a barrier phase, bounded; per lane (no warp vote)
__device__ __forceinline__ bool wait_lane(unsigned bar, unsigned parity, int *err) {
    unsigned long long t0 = 0;
    int spins = 0;
    while (!mb_try(bar, parity)) {
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

}  // namespace
}  // namespace msgb
