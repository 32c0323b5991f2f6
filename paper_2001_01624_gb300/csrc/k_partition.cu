// Coarse partitions built on the GPU (Sec. 5.1):
//  * face-connected components of cells with equal class (static partitions:
//    class = general block x facies; dynamic partitions: class = bin of the
//    pressure update), numbered by their lowest cell index;
//  * the dynamic classes: bins of log10(max(|dp|, eps max|dp|)).
//
// Components use lock-free union-find: every edge joins the two roots by
// hooking the larger root under the smaller one with compare-and-swap, so a
// component's final root is its lowest cell whatever the schedule; then
// roots are ranked by an exclusive scan, which numbers blocks in order of
// their lowest cell.
#include "ms_internal.h"

namespace msgb {

namespace {

constexpr int kThreads = 256;
inline int blocks_for(int64_t n) { return (int)((n + kThreads - 1) / kThreads); }

__device__ __forceinline__ int find_root(int *parent, int x) {
    int p = __ldcg(&parent[x]);
    while (p != x) {
        const int gp = __ldcg(&parent[p]);
        if (gp != p) atomicCAS(&parent[x], p, gp);   // path halving; only ever moves toward a smaller root
        x = p;
        p = __ldcg(&parent[x]);
    }
    return x;
}

__global__ void k_cc_init(int n, int *parent) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) parent[i] = i;
}

__global__ void k_cc_hook(int n, int W, const int *__restrict__ col, const int *__restrict__ cls, int *parent) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int ci = cls[i];
    for (int w = 0; w < W; ++w) {
        const int k = col[(int64_t)w * n + i];
        if (k <= i || cls[k] != ci) continue;   // each edge once, from its lower end
        int a = i, b = k;
        for (int guard = 0; guard < 1 << 20; ++guard) {
            int ra = find_root(parent, a), rb = find_root(parent, b);
            if (ra == rb) break;
            if (ra > rb) { const int t = ra; ra = rb; rb = t; }
            const int old = atomicCAS(&parent[rb], rb, ra);
            if (old == rb) break;
            a = ra;
            b = old;
        }
    }
}

__global__ void k_cc_compress(int n, int *parent) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) parent[i] = find_root(parent, i);
}

// exclusive scan of root flags: per-block sums, then one CTA scans the sums
__global__ void k_root_blocksum(int n, const int *__restrict__ label, int *__restrict__ bsum) {
    __shared__ int s[kThreads];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    s[threadIdx.x] = (i < n && label[i] == i) ? 1 : 0;
    __syncthreads();
    for (int o = kThreads / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) bsum[blockIdx.x] = s[0];
}

__global__ void k_scan_sums(int nb, int *bsum, int *total) {
    __shared__ int carry;
    __shared__ int s[1024];
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < nb; base += 1024) {
        const int i = base + threadIdx.x;
        const int v = i < nb ? bsum[i] : 0;
        s[threadIdx.x] = v;
        __syncthreads();
        for (int o = 1; o < 1024; o <<= 1) {   // Hillis-Steele inclusive scan
            const int t = threadIdx.x >= (unsigned)o ? s[threadIdx.x - o] : 0;
            __syncthreads();
            s[threadIdx.x] += t;
            __syncthreads();
        }
        if (i < nb) bsum[i] = carry + s[threadIdx.x] - v;
        __syncthreads();
        if (threadIdx.x == 1023) carry += s[1023];
        __syncthreads();
    }
    if (threadIdx.x == 0) *total = carry;
}

__global__ void k_root_rank(int n, const int *__restrict__ label, const int *__restrict__ bsum, int *__restrict__ rank) {
    __shared__ int s[kThreads];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int f = (i < n && label[i] == i) ? 1 : 0;
    s[threadIdx.x] = f;
    __syncthreads();
    for (int o = 1; o < kThreads; o <<= 1) {
        const int t = threadIdx.x >= (unsigned)o ? s[threadIdx.x - o] : 0;
        __syncthreads();
        s[threadIdx.x] += t;
        __syncthreads();
    }
    if (i < n) rank[i] = bsum[blockIdx.x] + s[threadIdx.x] - f;
}

__global__ void k_assign(int n, const int *__restrict__ label, const int *__restrict__ rank, int *__restrict__ part) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) part[i] = rank[label[i]];
}

// ------------------------------------------------------------ dynamic bins
__device__ __forceinline__ unsigned long long ord_bits(double v) {   // order-preserving map
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
__device__ __forceinline__ double from_ord(unsigned long long o) {
    const unsigned long long b = (o >> 63) ? (o & 0x7fffffffffffffffull) : ~o;
    return __longlong_as_double((long long)b);
}

// buf[0] = max |dp| (ordered bits), buf[1] = min v, buf[2] = max v
__global__ void k_dyn_absmax(int n, const double *__restrict__ dp, unsigned long long *buf) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double a = i < n ? fabs(dp[i]) : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a = fmax(a, __shfl_down_sync(0xffffffffu, a, o));
    if ((threadIdx.x & 31) == 0) atomicMax(&buf[0], ord_bits(a));
}

__device__ __forceinline__ double dyn_value(double dpi, double amax, double eps) {
    double a = fabs(dpi);
    const double fl = eps * amax;
    if (a < fl) a = fl;
    return log10(a);
}

__global__ void k_dyn_range(int n, const double *__restrict__ dp, double eps, unsigned long long *buf) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const double amax = from_ord(buf[0]);
    if (!(amax > 0.0)) return;
    double lo = INFINITY, hi = -INFINITY;
    if (i < n) lo = hi = dyn_value(dp[i], amax, eps);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        lo = fmin(lo, __shfl_down_sync(0xffffffffu, lo, o));
        hi = fmax(hi, __shfl_down_sync(0xffffffffu, hi, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMin(&buf[1], ord_bits(lo));
        atomicMax(&buf[2], ord_bits(hi));
    }
}

__global__ void k_dyn_class(int n, const double *__restrict__ dp, double eps, int n_bins,
                            const unsigned long long *buf, int *__restrict__ cls) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double amax = from_ord(buf[0]);
    int b = 0;
    if (amax > 0.0) {
        const double vmin = from_ord(buf[1]), vmax = from_ord(buf[2]);
        if (vmax > vmin) {
            const double width = (vmax - vmin) / n_bins;
            const double v = dyn_value(dp[i], amax, eps);
            b = (int)floor((v - vmin) / width);
            b = b > n_bins - 1 ? n_bins - 1 : (b < 0 ? 0 : b);
        }
    }
    cls[i] = b;
}

__global__ void k_dyn_buf_init(unsigned long long *buf) {
    if (threadIdx.x == 0) {
        buf[0] = 0ull;
        buf[1] = ~0ull;
        buf[2] = 0ull;
    }
}

}  // namespace

void launch_components(const ms_system &s, const int *cls, int *label, cudaStream_t st) {
    KernelScope ks_(st, "components", 0.0);
    k_cc_init<<<blocks_for(s.n), kThreads, 0, st>>>(s.n, label);
    k_cc_hook<<<blocks_for(s.n), kThreads, 0, st>>>(s.n, s.W, s.col.p, cls, label);
    k_cc_compress<<<blocks_for(s.n), kThreads, 0, st>>>(s.n, label);
    MS_CHECK_LAUNCH();
}

// label: component roots; part: output block ids; scratch: >= n + blocks + 1 ints
int launch_number_components(const ms_system &s, int *label, int *part, int *scratch, int *host_pinned,
                             cudaStream_t st) {
    const int nb = blocks_for(s.n);
    KernelScope ks_(st, "number_components", 0.0);
    int *bsum = scratch, *total = scratch + nb, *rank = scratch + nb + 1;
    k_root_blocksum<<<nb, kThreads, 0, st>>>(s.n, label, bsum);
    k_scan_sums<<<1, 1024, 0, st>>>(nb, bsum, total);
    k_root_rank<<<nb, kThreads, 0, st>>>(s.n, label, bsum, rank);
    k_assign<<<nb, kThreads, 0, st>>>(s.n, label, rank, part);
    MS_CHECK_LAUNCH();
    MS_CUDA(cudaMemcpyAsync(host_pinned, total, sizeof(int), cudaMemcpyDeviceToHost, st));
    MS_CUDA(cudaStreamSynchronize(st));
    return *host_pinned;
}

void launch_dynamic_classes(const ms_system &s, const double *dp, int n_bins, double eps, int *cls,
                            unsigned long long *buf, cudaStream_t st) {
    KernelScope ks_(st, "dynamic_classes", (double)s.n * 8 * 3);
    k_dyn_buf_init<<<1, 32, 0, st>>>(buf);
    k_dyn_absmax<<<blocks_for(s.n), kThreads, 0, st>>>(s.n, dp, buf);
    k_dyn_range<<<blocks_for(s.n), kThreads, 0, st>>>(s.n, dp, eps, buf);
    k_dyn_class<<<blocks_for(s.n), kThreads, 0, st>>>(s.n, dp, eps, n_bins, buf, cls);
    MS_CHECK_LAUNCH();
}

}  // namespace msgb
