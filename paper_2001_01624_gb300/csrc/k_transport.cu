// Two-phase (water / oil) incompressible transport for sequential-implicit
// time steps: Corey relative permeabilities, total mobility for the pressure
// equation, and explicit single-point-upstream saturation updates with CFL
// substeps.  The paper's two-phase setting (Sec. 2): total mobility
// lambda_t = krw/mu_w + kro/mu_o weights the pressure equation; the water
// saturation follows phi dS/dt + div(f_w u) = q_w with fractional flow
// f_w = (krw/mu_w) / lambda_t.
#include <algorithm>
#include <cmath>

#include "ms_internal.h"

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

__global__ void k_frac_flow(int n, Fluid f, const double *__restrict__ S, double *__restrict__ fw) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) fw[i] = frac_flow(f, S[i]);
}

// one explicit upwind substep: S_new = S + h / (phi V) (q_w - net water outflow),
// with the cells' fractional flows fw of the current S
__global__ void k_transport_substep(int n, const int *__restrict__ rf_ptr, const int *__restrict__ rf_face,
                                    const int *__restrict__ fa, const int *__restrict__ fb,
                                    const double *__restrict__ u, const double *__restrict__ q,
                                    const double *__restrict__ fw, const double *__restrict__ S,
                                    double *__restrict__ Snew, double h_over_pv) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double qi = q[i];
    double acc = qi > 0.0 ? qi : qi * fw[i];   // injected water / produced water
    for (int e = rf_ptr[i]; e < rf_ptr[i + 1]; ++e) {
        const int k = rf_face[e];
        const double uk = u[k];
        const int up = uk >= 0.0 ? fa[k] : fb[k];
        const double w = uk * fw[up];   // water flux a -> b
        acc += fa[k] == i ? -w : w;
    }
    Snew[i] = S[i] + h_over_pv * acc;
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

void launch_transport_substep(const ms_system &s, const double fl[6], const double *u, const double *q,
                              const double *S, double *fw, double *Snew, double h_over_pv, cudaStream_t st) {
    const Fluid f{fl[0], fl[1], fl[2], fl[3], fl[4], fl[5]};
    KernelScope ks_(st, "transport", (double)s.n * 40 + (double)s.nf * 2 * (4 + 4 + 4 + 8 + 8));
    k_frac_flow<<<blocks_for(s.n), kThreads, 0, st>>>(s.n, f, S, fw);
    k_transport_substep<<<blocks_for(s.n), kThreads, 0, st>>>(s.n, s.rf_ptr.p, s.rf_face.p, s.f_a.p, s.f_b.p, u, q,
                                                              fw, S, Snew, h_over_pv);
    MS_CHECK_LAUNCH();
}

}  // namespace msgb
