// The cell update of MsRSB basis smoothing (Sec. 5.1), shared by the
// per-system smoothing kernel and the batched persistent kernel, so both
// compute bitwise the same values.
#pragma once

#include "ms_internal.h"

namespace msgb {

// |x| as an integer key that orders like the value (IEEE bit patterns of
// non-negative numbers; NaN above infinity), so the running maximum of the
// basis increments stays off the FP64 pipe; key_value turns the key back.
__device__ __forceinline__ unsigned long long abs_key(double x) {
    return (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull;
}
__device__ __forceinline__ unsigned long long abs_key(float x) {
    return (unsigned long long)(__float_as_uint(x) & 0x7fffffffu);
}
template <typename T>
__device__ __forceinline__ double key_value(unsigned long long k);
template <>
__device__ __forceinline__ double key_value<double>(unsigned long long k) { return __longlong_as_double((long long)k); }
template <>
__device__ __forceinline__ double key_value<float>(unsigned long long k) { return (double)__uint_as_float((unsigned)k); }

// Slot-value loads: LD 0 as the compiler chooses (values constant during the
// launch), 1 through L2 only, 2 weak loads cached in L1 -- values another
// block wrote in the same launch, read after an acquire that synchronises
// with their release (the acquire invalidates the SM's L1, so a later weak
// load cannot return an older value; PTX memory model, causality order).
__device__ __forceinline__ double ld_ca(const double *p) {
    double v;
    asm volatile("ld.global.ca.f64 %0, [%1];" : "=d"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ float ld_ca(const float *p) {
    float v;
    asm volatile("ld.global.ca.f32 %0, [%1];" : "=f"(v) : "l"(p));
    return v;
}

template <typename T, int LD>
__device__ __forceinline__ T ldp(const T *p) {
    if constexpr (LD == 1) return __ldcg(p);
    else if constexpr (LD == 2) return ld_ca(p);
    else return *p;
}

// 1 / x for a normal x of magnitude below 2^1021: a seed from the FP32
// reciprocal of x's mantissa (exponent and sign set by integer arithmetic, so
// no conversion runs on the FP64 pipe), then one third-order step of the
// series 1 / x = r0 / (1 - e) = r0 (1 + e + e^2 + ...), e = 1 - x r0: with
// |e| below 2^-21 the truncation error e^3 is below 2^-63 relative.  Other
// x take the division.
__device__ __forceinline__ double recip_series(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned hi = (unsigned)(b >> 32);
    const int ex = (int)((hi >> 20) & 0x7ffu);
    if (ex == 0 || ex >= 0x7fd) return 1.0 / x;
    const float m = __uint_as_float(0x3f800000u | ((hi & 0xfffffu) << 3) | (unsigned)((b >> 29) & 7u));
    float rm;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rm) : "f"(m));   // 1 / m in (0.5, 1]
    const unsigned rb = __float_as_uint(rm);
    const long long de = (long long)(((int)((rb >> 23) & 0xffu) - 127) - (ex - 1023) + 1023);   // in [1, 2045]
    const double r0 = __longlong_as_double((long long)((b & 0x8000000000000000ull) | ((unsigned long long)de << 52) |
                                                       ((unsigned long long)(rb & 0x7fffffu) << 29)));
    const double e = fma(-x, r0, 1.0);
    return fma(r0, fma(e, e, e), r0);
}

// One cell of the MsRSB iteration with precomputed neighbour slot maps,
// slots below SB (at least the cell's count); returns the key of its largest
// |increment|.
// CG: the slot-value load policy of ldp (k_msrsb_batch reads values other
// blocks of the same launch wrote).
// PRE: the rows come prescaled (diag = 1 - (omega / A_ii) A_ii, off = -(omega / A_ii) A_ij), so the
// Jacobi update is already in the accumulated sum.
template <typename T, int WM, int SB, bool PRE, int CG = 0>
__device__ __forceinline__ unsigned long long msrsb_cell(int i, int cnt, int n, int W, const int *__restrict__ col,
                                                         const T *__restrict__ off, const T *__restrict__ diag,
                                                         const unsigned *__restrict__ nmap,
                                                         const T *__restrict__ pin, T *__restrict__ pout,
                                                         const T *__restrict__ odiag) {
    unsigned long long inck = 0ull;
    T v[SB], acc[SB];
    const T d = diag[i];
#pragma unroll
    for (int s = 0; s < SB; ++s) {
        v[s] = s < cnt ? ldp<T, CG>(pin + (int64_t)s * n + i) : T(0);
        acc[s] = d * v[s];
    }
    if (WM > 0) {
        // at most WM connections: every connection's column, coefficient and
        // slot map are loaded first, then all the gathers, so the loads of
        // different neighbours overlap (same order of the sums as below)
        int kk[WM > 0 ? WM : 1];
        T aw[WM > 0 ? WM : 1];
        unsigned mw[WM > 0 ? WM : 1];
#pragma unroll
        for (int w = 0; w < WM; ++w) {
            const int64_t at = (int64_t)w * n + i;
            kk[w] = w < W ? col[at] : i;
            aw[w] = w < W ? off[at] : T(0);
            mw[w] = w < W ? nmap[at] : 0xffffffffu;
        }
#pragma unroll
        for (int w = 0; w < WM; ++w) {
            if (kk[w] == i) continue;
#pragma unroll
            for (int s = 0; s < SB; ++s) {
                const unsigned t = (mw[w] >> (4 * s)) & 15u;
                if (s < cnt && t != 15u) acc[s] += aw[w] * ldp<T, CG>(pin + (int64_t)t * n + kk[w]);
            }
        }
    } else {
        for (int w = 0; w < W; ++w) {
            const int64_t at = (int64_t)w * n + i;
            const int k = col[at];
            if (k == i) continue;
            const T a = off[at];
            const unsigned m = nmap[at];
#pragma unroll
            for (int s = 0; s < SB; ++s) {
                const unsigned t = (m >> (4 * s)) & 15u;
                if (s < cnt && t != 15u) acc[s] += a * ldp<T, CG>(pin + (int64_t)t * n + k);
            }
        }
    }
    // omega / A_ii precomputed per smoothing run; one reciprocal for the
    // partition-of-unity scale
    T sum = 0;
    if (PRE) {
#pragma unroll
        for (int s = 0; s < SB; ++s)
            if (s < cnt) sum += acc[s];
    } else {
        const T od = odiag[i];
#pragma unroll
        for (int s = 0; s < SB; ++s)
            if (s < cnt) {
                acc[s] = v[s] - od * acc[s];
                sum += acc[s];
            }
    }
    T rs;
    if constexpr (sizeof(T) == 8) rs = recip_series(sum);
    else rs = T(1) / sum;
#pragma unroll
    for (int s = 0; s < SB; ++s)
        if (s < cnt) {
            const T nv = acc[s] * rs;
            inck = max(inck, abs_key(nv - v[s]));
            pout[(int64_t)s * n + i] = nv;
        }
    return inck;
}

}  // namespace msgb
