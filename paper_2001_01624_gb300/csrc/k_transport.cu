// Two-phase (water / oil) incompressible transport for sequential-implicit
// time steps: Corey relative permeabilities, total mobility for the pressure
// equation, and explicit single-point-upstream saturation updates with CFL
// substeps.  The paper's two-phase setting (Sec. 2): total mobility
// lambda_t = krw/mu_w + kro/mu_o weights the pressure equation; the water
// saturation follows phi dS/dt + div(f_w u) = q_w with fractional flow
// f_w = (krw/mu_w) / lambda_t.
#include <algorithm>
#include <cmath>

#include <cstdlib>

#include "ms_internal.h"
#include "grid_sync.cuh"

namespace msgb {

namespace {

constexpr int kThreads = 256;
inline int blocks_for(int64_t n) { return (int)((n + kThreads - 1) / kThreads); }

struct Fluid {
    double mu_w, mu_o, n_w, n_o, s_wc, s_or;
};

// x^e: repeated products for small integer exponents (exact to one rounding
// per product), the library power otherwise
__host__ __device__ inline double power(double x, double e) {
    if (e == (double)(int)e && e >= 0.0 && e <= 8.0) {
        double r = 1.0;
        for (int k = 0; k < (int)e; ++k) r *= x;
        return r;
    }
    return pow(x, e);
}

__host__ __device__ inline void phase_mobilities(const Fluid &f, double S, double &lw, double &lo) {
    double se = (S - f.s_wc) / (1.0 - f.s_wc - f.s_or);
    se = se < 0.0 ? 0.0 : (se > 1.0 ? 1.0 : se);
    lw = power(se, f.n_w) / f.mu_w;
    lo = power(1.0 - se, f.n_o) / f.mu_o;
}

__host__ __device__ inline double frac_flow(const Fluid &f, double S) {
    double lw, lo;
    phase_mobilities(f, S, lw, lo);
    const double lt = lw + lo;
    return lt > 0.0 ? lw / lt : 0.0;
}

__global__ void k_total_mobility(int n, Fluid f, const double *__restrict__ S, double *__restrict__ lam) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double lw, lo;
    phase_mobilities(f, S[i], lw, lo);
    lam[i] = lw + lo;
}

// total flux across each connection, a -> b positive
__global__ void k_face_flux(int nf, const int *__restrict__ fa, const int *__restrict__ fb,
                            const double *__restrict__ T, const double *__restrict__ p, double *__restrict__ u) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nf) return;
    u[k] = T[k] * (p[fa[k]] - p[fb[k]]);
}

__device__ inline void atomic_min_pos(unsigned long long *m, double v) {
    // positive doubles order like their bit patterns
    atomicMin(m, (unsigned long long)__double_as_longlong(v));
}

// stable explicit step of each cell: pore volume over its total outflow
// (outgoing connection fluxes and production); the minimum over cells
__global__ void k_outflow_limit(int n, const int *__restrict__ rf_ptr, const int *__restrict__ rf_face,
                                const int *__restrict__ fa, const double *__restrict__ u, const double *__restrict__ q,
                                double pore_volume, unsigned long long *min_bits) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double out = q[i] < 0.0 ? -q[i] : 0.0;
    for (int e = rf_ptr[i]; e < rf_ptr[i + 1]; ++e) {
        const int k = rf_face[e];
        const double uo = fa[k] == i ? u[k] : -u[k];   // flux leaving i
        if (uo > 0.0) out += uo;
    }
    if (out > 0.0) atomic_min_pos(min_bits, pore_volume / out);
}

// The fractional flow with the fluid's divisions done once per transport step:
// se = (S - s_wc) / (1 - s_wc - s_or) and the phase mobilities' 1 / mu as
// multipliers, one division per cell (within a few roundings of frac_flow)
struct FluidFast {
    double s_wc, inv_range, inv_mw, inv_mo, n_w, n_o;
    int iw, io;   // the exponents when they are small integers (0..8), else -1
};
// x^e with the exponent's kind decided once per step (repeated products for a
// small integer exponent, the library power otherwise), so a cell spends no
// FP64 comparisons on it
__device__ __forceinline__ double power_k(double x, int ie, double e) {
    if (ie >= 0) {
        double r = 1.0;
        for (int k = 0; k < ie; ++k) r *= x;
        return r;
    }
    return pow(x, e);
}
__device__ __forceinline__ double frac_flow_fast(const FluidFast &f, double S) {
    const double se = fmin(fmax((S - f.s_wc) * f.inv_range, 0.0), 1.0);
    const double lw = power_k(se, f.iw, f.n_w) * f.inv_mw, lo = power_k(1.0 - se, f.io, f.n_o) * f.inv_mo;
    const double lt = lw + lo;
    return lt > 0.0 ? lw / lt : 0.0;
}

// Upstream weights of one transport step (the fluxes u and the sources q do
// not change over its substeps): a cell's water balance is
//     src_i + dg_i fw_i + sum over its inflow faces of |u| fw_upstream
// with src_i the injection (q_i > 0), dg_i the production (q_i < 0) minus the
// fluxes leaving the cell (the cell is their upstream end), and the inflow
// faces' upstream cells and fluxes in an ELL layout [W][n] with a count per
// cell (zero fluxes dropped): the terms of one explicit upstream substep,
// S_new = S + h / (phi V) (q_w - net water outflow), grouped by upstream cell.
__global__ void k_transport_coef(int n, int W, const int *__restrict__ rf_ptr, const int *__restrict__ rf_face,
                                 const int *__restrict__ fa, const int *__restrict__ fb,
                                 const double *__restrict__ u, const double *__restrict__ q,
                                 double *__restrict__ src, double *__restrict__ dg, int *__restrict__ cnt,
                                 int *__restrict__ icol, double *__restrict__ ival) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double qi = q[i];
    double d = qi < 0.0 ? qi : 0.0;
    int c = 0;
    for (int e = rf_ptr[i]; e < rf_ptr[i + 1]; ++e) {
        const int k = rf_face[e];
        const double uk = u[k];   // flux fa -> fb; the upstream end is fa when uk >= 0
        if (fa[k] == i) {
            if (uk >= 0.0) d -= uk;
            else if (c < W) { icol[(int64_t)c * n + i] = fb[k]; ival[(int64_t)c * n + i] = -uk; ++c; }
        } else {
            if (uk < 0.0) d += uk;
            else if (uk > 0.0 && c < W) { icol[(int64_t)c * n + i] = fa[k]; ival[(int64_t)c * n + i] = uk; ++c; }
        }
    }
    src[i] = qi > 0.0 ? qi : 0.0;
    dg[i] = d;
    cnt[i] = c;
}

// One substep in the grouped form: S += h / (phi V) * balance(fw), then the
// new fractional flow.
__device__ __forceinline__ void transport_cell(int i, int n, const double *__restrict__ src,
                                               const double *__restrict__ dg, const int *__restrict__ cnt,
                                               const int *__restrict__ icol, const double *__restrict__ ival,
                                               const FluidFast &f, double h_over_pv, const double *fc, double *fn,
                                               double *S) {
    double acc = src[i] + dg[i] * __ldcg(fc + i);
    const int c = cnt[i];
    for (int w = 0; w < c; ++w) acc += ival[(int64_t)w * n + i] * __ldcg(fc + icol[(int64_t)w * n + i]);
    const double Sn = S[i] + h_over_pv * acc;
    S[i] = Sn;
    fn[i] = frac_flow_fast(f, Sn);
}

// Every substep of a transport step in one cooperative launch: the cells'
// fractional flows of the current substep are read through L2 by their
// neighbours, so a grid barrier (bounded) separates the substeps; the two
// fractional-flow buffers alternate.  nsub barriers in all.
__global__ void __launch_bounds__(256) k_transport_run(int n, int nsub, FluidFast f, double h_over_pv,
                                                       const double *__restrict__ src, const double *__restrict__ dg,
                                                       const int *__restrict__ cnt, const int *__restrict__ icol,
                                                       const double *__restrict__ ival, double *S, double *fwa,
                                                       double *fwb, unsigned long long *bar, int *err) {
    GridSync gs;
    gs.begin(bar, err);
    const int G = gridDim.x * blockDim.x;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += G) fwa[i] = frac_flow_fast(f, S[i]);
    if (!gs.sync(nsub)) return;
    for (int k = 0; k < nsub; ++k) {
        const double *fc = (k & 1) ? fwb : fwa;
        double *fn = (k & 1) ? fwa : fwb;
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += G)
            transport_cell(i, n, src, dg, cnt, icol, ival, f, h_over_pv, fc, fn, S);
        if (k + 1 < nsub && !gs.sync(nsub)) return;
    }
}

// the same, one substep per launch (where a cooperative launch cannot run)
__global__ void k_transport_one(int n, FluidFast f, double h_over_pv, const double *__restrict__ src,
                                const double *__restrict__ dg, const int *__restrict__ cnt,
                                const int *__restrict__ icol, const double *__restrict__ ival, const double *fc,
                                double *fn, double *S) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) transport_cell(i, n, src, dg, cnt, icol, ival, f, h_over_pv, fc, fn, S);
}

__global__ void k_frac_flow_fast(int n, FluidFast f, const double *__restrict__ S, double *__restrict__ fw) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) fw[i] = frac_flow_fast(f, S[i]);
}

constexpr int kTransportBlocksPerSm = 8;

FluidFast fast_fluid(const double fl[6]) {
    auto ik = [](double e) { return (e == (double)(int)e && e >= 0.0 && e <= 8.0) ? (int)e : -1; };
    return FluidFast{fl[4], 1.0 / (1.0 - fl[4] - fl[5]), 1.0 / fl[0], 1.0 / fl[1], fl[2], fl[3], ik(fl[2]), ik(fl[3])};
}

}  // namespace

// Largest derivative of the fractional-flow curve, from central differences
// on 2000 equal intervals of S in [0, 1].
double frac_flow_max_slope(double mu_w, double mu_o, double n_w, double n_o, double s_wc, double s_or) {
    const Fluid f{mu_w, mu_o, n_w, n_o, s_wc, s_or};
    const int K = 2000;
    double m = 0.0;
    for (int k = 1; k < K; ++k) {
        const double s0 = (double)(k - 1) / K, s1 = (double)(k + 1) / K;
        m = std::max(m, (frac_flow(f, s1) - frac_flow(f, s0)) / (s1 - s0));
    }
    return m;
}

void launch_total_mobility(int n, const double fl[6], const double *S, double *lam, cudaStream_t st) {
    const Fluid f{fl[0], fl[1], fl[2], fl[3], fl[4], fl[5]};
    KernelScope ks_(st, "total_mobility", (double)n * 16);
    k_total_mobility<<<blocks_for(n), kThreads, 0, st>>>(n, f, S, lam);
    MS_CHECK_LAUNCH();
}

void launch_face_flux(const ms_system &s, const double *p, double *u, cudaStream_t st) {
    if (s.nf == 0) return;
    KernelScope ks_(st, "face_flux", (double)s.nf * (4 + 4 + 8 + 16 + 8));
    k_face_flux<<<blocks_for(s.nf), kThreads, 0, st>>>(s.nf, s.f_a.p, s.f_b.p, s.f_T.p, p, u);
    MS_CHECK_LAUNCH();
}

void launch_outflow_limit(const ms_system &s, const double *u, const double *q, double pore_volume,
                          unsigned long long *min_bits, cudaStream_t st) {
    KernelScope ks_(st, "outflow_limit", (double)s.n * 16 + (double)s.nf * 2 * (4 + 4 + 8));
    k_outflow_limit<<<blocks_for(s.n), kThreads, 0, st>>>(s.n, s.rf_ptr.p, s.rf_face.p, s.f_a.p, u, q, pore_volume,
                                                          min_bits);
    MS_CHECK_LAUNCH();
}

void launch_transport_coef(ms_system &s, const double *u, const double *q, cudaStream_t st) {
    const int n = s.n, W = std::max(1, s.rf_max);
    s.w_tc.alloc((size_t)(2 + W) * n);
    s.w_tci.alloc((size_t)(1 + W) * n);
    KernelScope ks_(st, "transport_coef", (double)n * (4 + 8 + 8 + 8 + 4) + (double)s.nf * 2 * (4 + 4 + 4 + 8 + 12));
    k_transport_coef<<<blocks_for(n), kThreads, 0, st>>>(n, W, s.rf_ptr.p, s.rf_face.p, s.f_a.p, s.f_b.p, u, q,
                                                         s.w_tc.p, s.w_tc.p + n, s.w_tci.p, s.w_tci.p + n,
                                                         s.w_tc.p + 2 * (size_t)n);
    MS_CHECK_LAUNCH();
}

void launch_transport_run(ms_system &s, const double fl[6], int nsub, double h_over_pv, double *S, double *fwa,
                          double *fwb, cudaStream_t st) {
    const int n = s.n, W = std::max(1, s.rf_max);
    const FluidFast f = fast_fluid(fl);
    const double *src = s.w_tc.p, *dg = src + n, *ival = src + 2 * (size_t)n;
    const int *cnt = s.w_tci.p, *icol = cnt + n;
    (void)W;
    // algorithmic bytes per substep: the cell's weights, S read and written,
    // its fractional flow written, the upstream flows gathered
    const double per_sub = (double)n * (8 + 8 + 4 + 16 + 8 + 8) + (double)s.nf * (4 + 8 + 8);
    static int per_sm = -1;
    if (per_sm < 0) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_transport_run, 256, 0) != cudaSuccess) {
            cudaGetLastError();
            per_sm = 0;
        }
    }
    int sms = 0;
    MS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, s.device));
    const char *env = std::getenv("MSGB_TRANSPORT_COOP");
    const bool coop = per_sm > 0 && !(env && env[0] == '0');
    // blocks per SM of the one-launch form: each block arrives once on the
    // grid barrier per substep, so fewer, fuller blocks shorten the barrier
    int bps = kTransportBlocksPerSm;
    if (const char *b = std::getenv("MSGB_TRANSPORT_BPS")) bps = std::max(1, std::atoi(b));
    bps = std::min(bps, std::max(per_sm, 1));
    if (coop) {
        s.w_tbar.alloc(2);
        if (!s.tbar_ready) {
            s.w_tbar.zero(st);
            s.tbar_ready = true;
        }
        KernelScope ks_(st, "transport", per_sub * nsub + (double)n * 16);
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(std::max(1, std::min(sms * bps, blocks_for(n))));
        cfg.blockDim = dim3(256);
        cfg.stream = st;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeCooperative;   // grid barriers: every block resident
        at[0].val.cooperative = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        MS_CUDA(cudaLaunchKernelEx(&cfg, k_transport_run, n, nsub, f, h_over_pv, src, dg, cnt, icol, ival, S, fwa,
                                   fwb, s.w_tbar.p, s.sync.p + 3));
        return;
    }
    {
        KernelScope ks_(st, "transport", (double)n * 16);
        k_frac_flow_fast<<<blocks_for(n), kThreads, 0, st>>>(n, f, S, fwa);
        MS_CHECK_LAUNCH();
    }
    for (int k = 0; k < nsub; ++k) {
        KernelScope ks_(st, "transport", per_sub);
        k_transport_one<<<blocks_for(n), kThreads, 0, st>>>(n, f, h_over_pv, src, dg, cnt, icol, ival,
                                                           (k & 1) ? fwb : fwa, (k & 1) ? fwa : fwb, S);
        MS_CHECK_LAUNCH();
    }
}

}  // namespace msgb
