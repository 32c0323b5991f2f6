// CPR pressure stage (Sec. 4, quasi-IMPES decoupling; the predictor of the
// paper's Fig. 3) for a compressible two-phase (water / oil) step, fully
// implicit, primary variables p and s = s_w per cell:
//   R_a,i = V/dt [phi rho_a s_a - (phi rho_a s_a)^0] + sum_j F_a,ij - q_a,i,
//   F_a,ij = T_ij (lambda_a rho_a)(up) (p_i - p_j), up = the cell with the
//   higher pressure (the lower index on a tie),
// rho_a(p) = rho_a0 exp(c_a (p - p_ref)), phi(p) = phi0 exp(c_r (p - p_ref)),
// lambda_a = kr_a(s) / mu_a (Corey).  Quasi-IMPES weights per cell solve
// w_w dR_w/ds_i + w_o dR_o/ds_i = 0, w_w + w_o = 1 (diagonal saturation
// derivatives), and the pressure system is J* = W_w dR_w/dp + W_o dR_o/dp,
// right-hand side -(W_w R_w + W_o R_o).
//
// k_cpr_cell evaluates the per-cell state functions once (mobilities and
// their saturation derivatives, densities, accumulation terms); k_cpr_rows
// walks each row's faces (upstream values from the cell arrays), forms the
// row of both pressure blocks and the saturation diagonals in registers,
// applies the weights and writes the row of J* into the system's matrix.
#include <cmath>

#include "ms_internal.h"

namespace msgb {

namespace {

constexpr int kThreads = 256;
inline int blocks_for(int64_t n) { return (int)((n + kThreads - 1) / kThreads); }

// per cell: lambda_w, lambda_o, dlambda_w/ds, dlambda_o/ds, rho_w, rho_o
constexpr int kCellProps = 6;

// x^e: repeated multiplication for the usual integer Corey exponents (1..8),
// pow otherwise
__device__ __forceinline__ double cpr_pow(double x, double e) {
    const int k = (int)e;
    if ((double)k == e && k >= 0 && k <= 8) {
        double r = 1.0;
        for (int q = 0; q < k; ++q) r *= x;
        return r;
    }
    return pow(x, e);
}

__global__ void k_cpr_cell(int n, ms_cpr_fluid f, double vol_dt, const double *__restrict__ p,
                           const double *__restrict__ s, const double *__restrict__ p0,
                           const double *__restrict__ s0, double *__restrict__ props, double *__restrict__ acc) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double d = 1.0 - f.s_wc - f.s_or;
    const double x = (s[i] - f.s_wc) / d;
    double se = x, dse = 1.0 / d;
    if (x < 0.0) { se = 0.0; dse = 0.0; }
    else if (x > 1.0) { se = 1.0; dse = 0.0; }
    const double pi = p[i], pi0 = p0[i];
    double *pr = props + (int64_t)i * kCellProps;
    pr[0] = cpr_pow(se, f.n_w) / f.mu_w;
    pr[1] = cpr_pow(1.0 - se, f.n_o) / f.mu_o;
    pr[2] = f.n_w * cpr_pow(se, f.n_w - 1.0) * dse / f.mu_w;
    pr[3] = -f.n_o * cpr_pow(1.0 - se, f.n_o - 1.0) * dse / f.mu_o;
    const double rw = f.rho_w0 * exp(f.c_w * (pi - f.p_ref)), ro = f.rho_o0 * exp(f.c_o * (pi - f.p_ref));
    pr[4] = rw;
    pr[5] = ro;
    const double ph = f.phi0 * exp(f.c_r * (pi - f.p_ref)), ph0 = f.phi0 * exp(f.c_r * (pi0 - f.p_ref));
    const double rw0 = f.rho_w0 * exp(f.c_w * (pi0 - f.p_ref)), ro0 = f.rho_o0 * exp(f.c_o * (pi0 - f.p_ref));
    double *a = acc + (int64_t)i * 6;
    a[0] = vol_dt * (ph * rw * s[i] - ph0 * rw0 * s0[i]);                    // water accumulation
    a[1] = vol_dt * (ph * ro * (1.0 - s[i]) - ph0 * ro0 * (1.0 - s0[i]));    // oil accumulation
    a[2] = vol_dt * ph * rw * (f.c_r + f.c_w) * s[i];                         // d/dp
    a[3] = vol_dt * ph * ro * (f.c_r + f.c_o) * (1.0 - s[i]);
    a[4] = vol_dt * ph * rw;                                                   // d/ds
    a[5] = -vol_dt * ph * ro;
}

template <int MW>
__global__ void k_cpr_rows(int n, int W, double c_w, double c_o, const int *__restrict__ rf_ptr,
                           const int *__restrict__ rf_face, const uint8_t *__restrict__ rf_slot,
                           const int *__restrict__ fa, const int *__restrict__ fb, const double *__restrict__ T,
                           const double *__restrict__ p, const double *__restrict__ props,
                           const double *__restrict__ acc, const double *__restrict__ qw,
                           const double *__restrict__ qo, double *__restrict__ off_u, double *__restrict__ off_p,
                           double *__restrict__ diag, double *__restrict__ rhs, double *__restrict__ wout) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double *a = acc + (int64_t)i * 6;
    double Rw = a[0] - qw[i], Ro = a[1] - qo[i];
    double Jw = a[2], Jo = a[3], Dw = a[4], Do = a[5];
    double jw[MW], jo[MW];
#pragma unroll
    for (int w = 0; w < MW; ++w) { jw[w] = 0.0; jo[w] = 0.0; }
    const double pi = p[i];
    for (int e = rf_ptr[i]; e < rf_ptr[i + 1]; ++e) {
        const int f = rf_face[e];
        const int slot = rf_slot[e];
        const int j = fa[f] == i ? fb[f] : fa[f];
        const double pj = p[j];
        const int up = pi > pj ? i : (pj > pi ? j : min(i, j));
        const double *u = props + (int64_t)up * kCellProps;
        const double lw = u[0], lo = u[1], rw = u[4], ro = u[5];
        const double t = T[f], dp = pi - pj;
        const double gw = t * lw * rw, go = t * lo * ro;
        Rw += gw * dp;
        Ro += go * dp;
        // density of the upstream cell moves with its pressure
        const double hw = dp * t * lw * c_w * rw, ho = dp * t * lo * c_o * ro;
        double dwj = -gw, doj = -go;
        if (up == i) {
            Jw += gw + hw;
            Jo += go + ho;
            Dw += dp * t * u[2] * rw;
            Do += dp * t * u[3] * ro;
        } else {
            Jw += gw;
            Jo += go;
            dwj += hw;
            doj += ho;
        }
#pragma unroll
        for (int w = 0; w < MW; ++w)
            if (w == slot) { jw[w] += dwj; jo[w] += doj; }
    }
    const double den = Do - Dw;
    const double ww = den != 0.0 ? Do / den : 0.5, wo = den != 0.0 ? -Dw / den : 0.5;
    diag[i] = ww * Jw + wo * Jo;
#pragma unroll
    for (int w = 0; w < MW; ++w)
        if (w < W) {
            const double v = ww * jw[w] + wo * jo[w];
            off_u[(int64_t)w * n + i] = v;
            off_p[(int64_t)w * n + i] = v;
        }
    rhs[i] = -(ww * Rw + wo * Ro);
    if (wout) {
        wout[i] = ww;
        wout[n + i] = wo;
    }
}

}  // namespace

void launch_cpr_pressure(ms_system &s, const ms_cpr_fluid &f, double dt, const double *p, const double *sw,
                         const double *p0, const double *s0, const double *qw, const double *qo, double *rhs,
                         double *wout, cudaStream_t st) {
    s.w_cpr.alloc((size_t)s.n * (kCellProps + 6));
    double *props = s.w_cpr.p, *acc = s.w_cpr.p + (size_t)s.n * kCellProps;
    const double vol_dt = s.dx * s.dy * s.dz / dt;
    {
        KernelScope ks_(st, "cpr_cell", (double)s.n * (4 * 8 + 12 * 8));
        k_cpr_cell<<<blocks_for(s.n), kThreads, 0, st>>>(s.n, f, vol_dt, p, sw, p0, s0, props, acc);
        MS_CHECK_LAUNCH();
    }
    // per face side: face id, slot, both ends, T, the neighbour's pressure and state; per row: own state,
    // sources, the row of J* (twice: unpinned and pinned copies), diagonal, right-hand side
    KernelScope ks_(st, "cpr_rows",
                    (double)s.nf * 2 * (4 + 1 + 8 + 8 + 8 + kCellProps * 8) +
                        (double)s.n * (4 + 8 + 6 * 8 + 16 + 2 * 8 * s.W + 16 + (wout ? 16 : 0)));
    if (s.W <= 8)
        k_cpr_rows<8><<<blocks_for(s.n), kThreads, 0, st>>>(s.n, s.W, f.c_w, f.c_o, s.rf_ptr.p, s.rf_face.p,
                                                            s.rf_slot.p, s.f_a.p, s.f_b.p, s.f_T.p, p, props, acc,
                                                            qw, qo, s.off_u.p, s.off_p.p, s.diag.p, rhs, wout);
    else if (s.W <= 16)
        k_cpr_rows<16><<<blocks_for(s.n), kThreads, 0, st>>>(s.n, s.W, f.c_w, f.c_o, s.rf_ptr.p, s.rf_face.p,
                                                             s.rf_slot.p, s.f_a.p, s.f_b.p, s.f_T.p, p, props, acc,
                                                             qw, qo, s.off_u.p, s.off_p.p, s.diag.p, rhs, wout);
    else
        throw Error{MS_ERR_INVALID_ARG, "more than 16 connections per cell in the CPR pressure kernel"};
    MS_CHECK_LAUNCH();
}

}  // namespace msgb
