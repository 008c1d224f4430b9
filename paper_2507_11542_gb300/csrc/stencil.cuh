// stencil.cuh -- device building blocks of the fused level-set stage kernel:
// ghost-aware 7-point line gathers (Sec. 2.1), upwind derivatives ENO1/2/3
// and WENO5 (Sec. 3.1-3.3), Hamiltonians with Lax-Friedrichs dissipation
// (Sec. 4) for each supported dynamics.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/hj.h"
#include "hj_internal.h"

namespace hj {

template <typename T> __device__ __forceinline__ T ld(const T* p) { return __ldg(p); }

__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }

// |x|, and the maximum of two non-negative values, for FP64 as integer
// operations on the bit patterns (non-negative doubles order like their bits):
// exact, and off the FP64 pipe that bounds the FP64 kernels. FP32 as usual.
__device__ __forceinline__ double absv(double a) {
    return __longlong_as_double(__double_as_longlong(a) & 0x7fffffffffffffffLL);
}
__device__ __forceinline__ float absv(float a) { return fabsf(a); }
__device__ __forceinline__ double max_nonneg(double a, double b) {
    const long long ia = __double_as_longlong(a), ib = __double_as_longlong(b);
    return __longlong_as_double(ia > ib ? ia : ib);
}
__device__ __forceinline__ float max_nonneg(float a, float b) { return fmaxf(a, b); }

template <typename T> __device__ __forceinline__ T sgn(T v) {
    return (v > T(0)) ? T(1) : ((v < T(0)) ? T(-1) : T(0));
}

// Values at nodes i-3 .. i+3 along one grid line (stride s, n nodes, node i
// at flat index idx). Off-grid nodes come from the ghost rule of the
// dimension: periodic wrap, or the outermost slope continued outward
// (away from the zero level set by default).
template <typename T>
__device__ __forceinline__ void gather7(const T* __restrict__ u, long long idx, int i, int n, long long s,
                                        bool periodic, int extrap, T v[7]) {
    if (i >= 3 && i + 3 < n) {
#pragma unroll
        for (int k = 0; k < 7; ++k) v[k] = ld(u + idx + (long long)(k - 3) * s);
        return;
    }
    const long long base = idx - (long long)i * s;
    if (periodic) {
#pragma unroll
        for (int k = 0; k < 7; ++k) {
            int j = (i + k - 3) % n;
            if (j < 0) j += n;
            v[k] = ld(u + base + (long long)j * s);
        }
        return;
    }
    const T e0 = ld(u + base), e1 = ld(u + base + s);
    const T f0 = ld(u + base + (long long)(n - 1) * s), f1 = ld(u + base + (long long)(n - 2) * s);
    const T slo = (extrap == HJ_EXTRAP_LINEAR) ? (e0 - e1) : fabs(e0 - e1) * sgn(e0);
    const T shi = (extrap == HJ_EXTRAP_LINEAR) ? (f0 - f1) : fabs(f0 - f1) * sgn(f0);
#pragma unroll
    for (int k = 0; k < 7; ++k) {
        const int j = i + k - 3;
        // product and sum rounded separately (no contraction), as in edge + m * slope
        if (j < 0) v[k] = add_rn(e0, mul_rn(T(-j), slo));
        else if (j >= n) v[k] = add_rn(f0, mul_rn(T(j - n + 1), shi));
        else v[k] = ld(u + base + (long long)j * s);
    }
}

// ---------------------------------------------------------------------------
// WENO5 (Sec. 3.3; Jiang & Peng 2000). Inputs are raw one-sided differences
// r_j = v_{j+1} - v_j (not yet divided by dx) around node i:
//   r0 = v_{i-2}-v_{i-3}, ..., r5 = v_{i+3}-v_{i+2}.
// p- uses (r0, r1, r2, r3, r4); p+ the mirrored (r5, r4, r3, r2, r1). The
// weights are homogeneous of degree zero in the differences, so working on
// raw differences and dividing by dx once at the end is the same scheme when
// the epsilon floor is scaled by dx^2 (weno_floor).
// The two sides share the second differences of windows (r1,r2,r3) and
// (r2,r3,r4) and two of their candidate stencils.
// ---------------------------------------------------------------------------
// FP64: weights c_k/(S_k+eps)^2 normalised with one division,
//   p = sum_k c_k q_k prod_{j!=k} d_j / sum_k c_k prod_{j!=k} d_j,  d_k = (S_k+eps)^2.
// On exactly flat data every d_k underflows and every q_k is zero: return q2.
__device__ __forceinline__ double weno_combine(double q1, double q2, double q3, double s1, double s2, double s3,
                                               double eps, double scale) {
    const double d1 = (s1 + eps) * (s1 + eps);
    const double d2 = (s2 + eps) * (s2 + eps);
    const double d3 = (s3 + eps) * (s3 + eps);
    const double w1 = 0.1 * (d2 * d3);
    const double w2 = 0.6 * (d1 * d3);
    const double w3 = 0.3 * (d1 * d2);
    const double num = w1 * q1 + w2 * q2 + w3 * q3;
    const double den = w1 + w2 + w3;
    return (den > 0.0) ? num / (den * scale) : q2 / scale;
}

// FP32: the epsilon floor keeps (S+eps)^2 >= 1e-36 (normal), so the direct
// form with fast reciprocals cannot overflow or divide by zero.
__device__ __forceinline__ float weno_combine(float q1, float q2, float q3, float s1, float s2, float s3,
                                              float eps, float scale) {
    const float a1 = 0.1f * __fdividef(1.0f, (s1 + eps) * (s1 + eps));
    const float a2 = 0.6f * __fdividef(1.0f, (s2 + eps) * (s2 + eps));
    const float a3 = 0.3f * __fdividef(1.0f, (s3 + eps) * (s3 + eps));
    const float num = a1 * q1 + a2 * q2 + a3 * q3;
    return num * __fdividef(1.0f, (a1 + a2 + a3) * scale);
}

template <typename T>
__device__ __forceinline__ void weno5_pair(const T v[7], T dx, T floor_raw, T& pm, T& pp) {
    const T r0 = v[1] - v[0], r1 = v[2] - v[1], r2 = v[3] - v[2];
    const T r3 = v[4] - v[3], r4 = v[5] - v[4], r5 = v[6] - v[5];
    const T c13 = T(13) / T(12);
    // second differences of the four windows
    const T tA = r0 - T(2) * r1 + r2;  // (r0, r1, r2)
    const T tB = r1 - T(2) * r2 + r3;  // (r1, r2, r3)
    const T tC = r2 - T(2) * r3 + r4;  // (r2, r3, r4)
    const T tD = r3 - T(2) * r4 + r5;  // (r3, r4, r5)
    // left side: v1..v5 = r0..r4
    const T uL1 = r0 - T(4) * r1 + T(3) * r2;
    const T uL2 = r1 - r3;
    const T uL3 = T(3) * r2 - T(4) * r3 + r4;
    const T sL1 = c13 * tA * tA + T(0.25) * uL1 * uL1;
    const T sL2 = c13 * tB * tB + T(0.25) * uL2 * uL2;
    const T sL3 = c13 * tC * tC + T(0.25) * uL3 * uL3;
    // right side: v1..v5 = r5..r1
    const T uR1 = r5 - T(4) * r4 + T(3) * r3;
    const T uR2 = r4 - r2;
    const T uR3 = T(3) * r3 - T(4) * r2 + r1;
    const T sR1 = c13 * tD * tD + T(0.25) * uR1 * uR1;
    const T sR2 = c13 * tC * tC + T(0.25) * uR2 * uR2;
    const T sR3 = c13 * tB * tB + T(0.25) * uR3 * uR3;
    // candidates, times 6
    const T qL1 = T(2) * r0 - T(7) * r1 + T(11) * r2;
    const T qL2 = -r1 + T(5) * r2 + T(2) * r3;   // = qR3
    const T qL3 = T(2) * r2 + T(5) * r3 - r4;    // = qR2
    const T qR1 = T(2) * r5 - T(7) * r4 + T(11) * r3;
    // epsilon = 1e-6 max(v_k^2) + floor
    const T m14 = fmax(fmax(r1 * r1, r2 * r2), fmax(r3 * r3, r4 * r4));
    const T epsL = T(1e-6) * fmax(m14, r0 * r0) + floor_raw;
    const T epsR = T(1e-6) * fmax(m14, r5 * r5) + floor_raw;
    const T scale = T(6) * dx;  // undo the candidates' factor 6 and divide by dx
    pm = weno_combine(qL1, qL2, qL3, sL1, sL2, sL3, epsL, scale);
    pp = weno_combine(qR1, qL3, qL2, sR1, sR2, sR3, epsR, scale);
}

// ---------------------------------------------------------------------------
// ENO1/2/3 (Sec. 3.1-3.2; Osher & Fedkiw Sec. 3.3) from the divided
// differences D1_{j+1/2} = (v_{j+1}-v_j)/dx, D2_j = (D1_{j+1/2}-D1_{j-1/2})/(2dx),
// D3_{j+1/2} = (D2_{j+1}-D2_j)/(3dx). Divisions (not reciprocal products)
// keep the stencil choices identical to the plain definition; a tie picks
// the left candidate.
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void eno_pair(const T v[7], T dx, int order, T& pm, T& pp) {
    T D1[6];  // D1[k] = D^1_{i-5/2+k}
#pragma unroll
    for (int k = 0; k < 6; ++k) D1[k] = (v[k + 1] - v[k]) / dx;
    if (order == 1) { pm = D1[2]; pp = D1[3]; return; }
    T D2[5];  // D2[k] = D^2_{i-2+k}
#pragma unroll
    for (int k = 0; k < 5; ++k) D2[k] = (D1[k + 1] - D1[k]) / (T(2) * dx);
    T D3[4];  // D3[k] = D^3_{i-3/2+k}
#pragma unroll
    for (int k = 0; k < 4; ++k) D3[k] = (D2[k + 1] - D2[k]) / (T(3) * dx);
    // left: stencil start k = i-1, so D2_k = D2[1], D2_{k+1} = D2[2]
    {
        const bool left = fabs(D2[1]) <= fabs(D2[2]);
        const T c = left ? D2[1] : D2[2];
        T p = D1[2] + c * dx;
        if (order == 3) {
            // k* = i-2 (left) or i-1; D3_{k*+1/2} = D3[k*-(i-2)], coefficient 3r^2-6r+2 at r = i-k*
            const T a = left ? D3[0] : D3[1];
            const T b = left ? D3[1] : D3[2];
            const T cs = (fabs(a) <= fabs(b)) ? a : b;
            const T coef = left ? T(2) : T(-1);
            p += cs * coef * dx * dx;
        }
        pm = p;
    }
    // right: stencil start k = i, D2_k = D2[2], D2_{k+1} = D2[3]
    {
        const bool left = fabs(D2[2]) <= fabs(D2[3]);
        const T c = left ? D2[2] : D2[3];
        T p = D1[3] - c * dx;
        if (order == 3) {
            // k* = i-1 (left) or i
            const T a = left ? D3[1] : D3[2];
            const T b = left ? D3[2] : D3[3];
            const T cs = (fabs(a) <= fabs(b)) ? a : b;
            const T coef = left ? T(-1) : T(2);
            p += cs * coef * dx * dx;
        }
        pp = p;
    }
}

template <typename T, int SCHEME>
__device__ __forceinline__ void upwind_pair(const T v[7], double dx, double inv_dx, T floor_raw, T& pm, T& pp) {
    if constexpr (SCHEME == HJ_WENO5) {
        weno5_pair<T>(v, T(dx), floor_raw, pm, pp);
    } else {
        eno_pair<T>(v, T(dx), SCHEME, pm, pp);
    }
}

// Node coordinate lo + i dx (Sec. 2.1), the product and the sum rounded
// separately, as the host and the oracle compute it: a fused multiply-add
// would move coordinates near 0 by a rounding step, and the dissipation local
// in p takes sign decisions on products with them.
template <typename T>
__device__ __forceinline__ T coord(T lo, int i, T dx) { return add_rn(lo, mul_rn(T(i), dx)); }

// Scalars of a stage launch in the kernel's precision.
template <typename T> struct SP;
template <> struct SP<double> {
    static __device__ __forceinline__ double lo(const StageParams& P, int d) { return P.g.lo[d]; }
    static __device__ __forceinline__ double dx(const StageParams& P, int d) { return P.g.dx[d]; }
    static __device__ __forceinline__ double inv_dx(const StageParams& P, int d) { return P.g.inv_dx[d]; }
    static __device__ __forceinline__ double half_inv_dx(const StageParams& P, int d) { return P.half_inv_dx[d]; }
    static __device__ __forceinline__ double half_inv_dx6(const StageParams& P, int d) { return P.half_inv_dx6[d]; }
    static __device__ __forceinline__ double alpha_g(const StageParams& P, int d) { return P.alpha_g[d]; }
    static __device__ __forceinline__ double param(const StageParams& P, int k) { return P.params[k]; }
    static __device__ __forceinline__ double dt(const StageParams& P) { return P.dt; }
    static __device__ __forceinline__ double cv(const StageParams& P) { return P.cv; }
    static __device__ __forceinline__ double cu(const StageParams& P) { return P.cu; }
    static __device__ __forceinline__ double floor(const StageParams& P, int d) { return P.weno_floor[d]; }
};
template <> struct SP<float> {
    static __device__ __forceinline__ float lo(const StageParams& P, int d) { return P.lo_f[d]; }
    static __device__ __forceinline__ float dx(const StageParams& P, int d) { return P.dx_f[d]; }
    static __device__ __forceinline__ float inv_dx(const StageParams& P, int d) { return P.inv_dx_f[d]; }
    static __device__ __forceinline__ float half_inv_dx(const StageParams& P, int d) { return P.half_inv_dx_f[d]; }
    static __device__ __forceinline__ float half_inv_dx6(const StageParams& P, int d) { return P.half_inv_dx6_f[d]; }
    static __device__ __forceinline__ float alpha_g(const StageParams& P, int d) { return P.alpha_g_f[d]; }
    static __device__ __forceinline__ float param(const StageParams& P, int k) { return P.params_f[k]; }
    static __device__ __forceinline__ float dt(const StageParams& P) { return P.dt_f; }
    static __device__ __forceinline__ float cv(const StageParams& P) { return P.cv_f; }
    static __device__ __forceinline__ float cu(const StageParams& P) { return P.cu_f; }
    // the FP32 floor is one constant for every dimension (no parameter load)
    static __device__ __forceinline__ float floor(const StageParams&, int) { return kWenoFloorF32; }
};

// ---------------------------------------------------------------------------
// Hamiltonian + Lax-Friedrichs dissipation (Sec. 4):
//   ydot = Hg(x, (p- + p+)/2) + sum_d alpha_d(x) (p+_d - p-_d)/2
// ---------------------------------------------------------------------------
template <typename T> struct Trig;
template <> struct Trig<double> { static __device__ __forceinline__ const double* get(const StageParams& P) { return P.trig_d; } };
template <> struct Trig<float>  { static __device__ __forceinline__ const float*  get(const StageParams& P) { return P.trig_f; } };

// Whether a dynamics takes cos/sin of the dimension-2 coordinate (from the
// angle table of the launch).
template <int D, int DYN>
__host__ __device__ constexpr bool uses_angle() {
    constexpr int B = dyn_base(DYN);
    return (B == HJ_DYN_AIR3D && D == 3) || (B == HJ_DYN_DUBINS4D && D == 4) || (B == HJ_DYN_ROCKETS && D == 3);
}

// max |d + k sigma| over the signs sigma a box of gradients allows (plus: +1,
// minus: -1).
template <typename T>
__device__ __forceinline__ T max_over_signs(T d, T k, bool plus, bool minus) {
    T best = T(0);
    if (plus) best = max_nonneg(best, absv(d + k));
    if (minus) best = max_nonneg(best, absv(d - k));
    return best;
}

// Lax-Friedrichs dissipation local in p (HJ_ALPHA_BOX; Sec. 4, alpha_d =
// max |dHg/dp_d|): the maximum over the node's box of gradients, p_j from
// pb_j - |dd_j| to pb_j + |dd_j| (the node's p- and p+). A linear part of Hg
// has a constant slope; a term k |l . p| has slope k sign(l . p) l_d, where
// the box allows sign +1 if the maximum of l . p over the box is >= 0 and -1
// if its minimum is <= 0. A slope made of two such terms is largest where
// both signs can be equal at one point of the box, which is checked on the
// box. The norm Hamiltonian -c|p| has |dHg/dp_d| = c |p_d| / |p|, largest at
// the largest |p_d| and the smallest |p_j| (j != d) the box holds; at p = 0
// its generalized gradient is the ball of radius c.
template <typename T, int D, int B>
__device__ __forceinline__ void box_alpha(const StageParams& P, const T* xc, T c, T s, const T* pb, const T* dd,
                                          T* a) {
    const auto q = [&P](int k) { return SP<T>::param(P, k); };
    T lo[D], hi[D];
#pragma unroll
    for (int d = 0; d < D; ++d) {
        const T w = absv(dd[d]);
        lo[d] = pb[d] - w;
        hi[d] = pb[d] + w;
    }
    if constexpr (B == HJ_DYN_NORM) {
        const T cn = q(0);
        T small2[D];
#pragma unroll
        for (int j = 0; j < D; ++j) {
            const T m = (lo[j] <= T(0) && hi[j] >= T(0)) ? T(0) : fmin(absv(lo[j]), absv(hi[j]));
            small2[j] = m * m;
        }
#pragma unroll
        for (int d = 0; d < D; ++d) {
            const T big = max_nonneg(absv(lo[d]), absv(hi[d]));
            T others = T(0);
#pragma unroll
            for (int j = 0; j < D; ++j)
                if (j != d) others += small2[j];
            a[d] = (big == T(0)) ? ((others == T(0)) ? cn : T(0)) : cn * big / sqrt(big * big + others);
        }
    } else if constexpr (B == HJ_DYN_AIR3D && D == 3) {
        const T va = q(0), vb = q(1), amax = q(2), bmax = q(3);
        const T f0 = -va + vb * c, f1 = vb * s;
        const T y0 = lo[0] * xc[1], y1 = hi[0] * xc[1];  // range of p0 y
        const T x0 = lo[1] * xc[0], x1 = hi[1] * xc[0];  // range of p1 x
        const T a0 = fmin(y0, y1), b0 = fmax(y0, y1), a1 = fmin(x0, x1), b1 = fmax(x0, x1);
        const bool plus = b0 - a1 - lo[2] >= T(0), minus = a0 - b1 - hi[2] <= T(0);
        a[0] = max_over_signs(f0, amax * xc[1], plus, minus);
        a[1] = max_over_signs(f1, -amax * xc[0], plus, minus);
        const T top = fmax(lo[2], T(0)), bot = fmin(hi[2], T(0));
        const bool same = (top <= hi[2] && b0 - a1 - top >= T(0)) || (lo[2] <= bot && a0 - b1 - bot <= T(0));
        a[2] = same ? amax + bmax : absv(amax - bmax);
    } else if constexpr (B == HJ_DYN_ROCKETS && D == 3) {
        const T ac = q(0), g = q(1), ue = q(2), up = q(3);
        const T f0 = ac * c, f1 = ac * s + ac - g;
        const T u0 = lo[0] * xc[0], u1 = hi[0] * xc[0];  // range of p0 x
        const T w0 = lo[1] * xc[0], w1 = hi[1] * xc[0];  // range of p1 x
        const T a0 = fmin(u0, u1), b0 = fmax(u0, u1), a1 = fmin(w0, w1), b1 = fmax(w0, w1);
        a[0] = max_over_signs(f0, ue * xc[0], b0 - lo[2] >= T(0), a0 - hi[2] <= T(0));
        a[1] = max_over_signs(f1, -up * xc[0], b1 + hi[2] >= T(0), a1 + lo[2] <= T(0));
        const bool same = fmax(lo[2], -b1) <= fmin(hi[2], b0) || fmax(lo[2], a0) <= fmin(hi[2], -a1);
        a[2] = same ? ue + up : absv(ue - up);
    }
}

// ydot from node coordinates xc, cos/sin (c, s) of the dimension-2
// coordinate (dynamics with uses_angle), the mean derivatives
// pb = (p- + p+)/2 and the half differences dd = (p+ - p-)/2:
// Hg(x, pb) + sum_d alpha_d dd_d, with alpha_d = alpha_d(x) (the maximum of
// |f_d| over the controls at the node) or, for global LF, the launch's
// alpha_g (its maximum over the grid).
//
// DYN may carry kDynBox: alpha_d is then the maximum over the node's box of
// gradients (box_alpha) instead of alpha_d(x).
template <typename T, int D, int DYN>
__device__ __forceinline__ T lf_combine(const StageParams& P, const T* xc, T c, T s, const T* pb, const T* dd,
                                        bool alpha_global) {
    const auto q = [&P](int k) { return SP<T>::param(P, k); };
    constexpr int B = dyn_base(DYN);
    T h = T(0);
    T a[D];
#pragma unroll
    for (int d = 0; d < D; ++d) a[d] = T(0);
    if constexpr (B == HJ_DYN_DOUBLE_INTEGRATOR && D == 2) {
        const T umax = q(0);
        h = pb[0] * xc[1] - umax * absv(pb[1]);
        a[0] = absv(xc[1]);
        a[1] = umax;
    } else if constexpr (B == HJ_DYN_AIR3D && D == 3) {
        const T va = q(0), vb = q(1), amax = q(2), bmax = q(3);
        const T f0 = -va + vb * c, f1 = vb * s;
        h = pb[0] * f0 + pb[1] * f1 + amax * absv(pb[0] * xc[1] - pb[1] * xc[0] - pb[2]) - bmax * absv(pb[2]);
        a[0] = absv(f0) + amax * absv(xc[1]);
        a[1] = absv(f1) + amax * absv(xc[0]);
        a[2] = amax + bmax;
    } else if constexpr (B == HJ_DYN_ROCKETS && D == 3) {
        const T ac = q(0), g = q(1), ue = q(2), up = q(3);
        const T f0 = ac * c, f1 = ac * s + ac - g;
        h = pb[0] * f0 + pb[1] * f1 + ue * absv(pb[0] * xc[0] - pb[2]) - up * absv(pb[1] * xc[0] + pb[2]);
        a[0] = absv(f0) + ue * absv(xc[0]);
        a[1] = absv(f1) + up * absv(xc[0]);
        a[2] = ue + up;
    } else if constexpr (B == HJ_DYN_DUBINS4D && D == 4) {
        const T wmax = q(0), accmax = q(1);
        const T f0 = xc[3] * c, f1 = xc[3] * s;
        h = pb[0] * f0 + pb[1] * f1 - wmax * absv(pb[2]) - accmax * absv(pb[3]);
        a[0] = absv(f0);
        a[1] = absv(f1);
        a[2] = wmax;
        a[3] = accmax;
    } else if constexpr (B == HJ_DYN_NORM) {
        const T cn = q(0);
        T s2 = T(0);
#pragma unroll
        for (int d = 0; d < D; ++d) { s2 += pb[d] * pb[d]; a[d] = cn; }
        h = -cn * sqrt(s2);
    } else if constexpr (B == HJ_DYN_ADVECT) {
#pragma unroll
        for (int d = 0; d < D; ++d) { const T cd = q(d); h += -cd * pb[d]; a[d] = absv(cd); }
    } else if constexpr (B == HJ_DYN_ROTATE && D >= 2) {
        const T w = q(0);
        const T f0 = -w * xc[1], f1 = w * xc[0];
        h = -(pb[0] * f0 + pb[1] * f1);
        a[0] = absv(f0);
        a[1] = absv(f1);
    }
    if constexpr (dyn_is_box(DYN)) box_alpha<T, D, B>(P, xc, c, s, pb, dd, a);
    if (alpha_global) {
#pragma unroll
        for (int d = 0; d < D; ++d) a[d] = SP<T>::alpha_g(P, d);
    }
    T y = h;
#pragma unroll
    for (int d = 0; d < D; ++d) y += a[d] * dd[d];
    return y;
}

// The Lax-Friedrichs term from the raw (undivided) one-sided derivatives:
// sums S_d = p-_d + p+_d and differences Q_d = p+_d - p-_d, with h_d =
// 1/(2 dx_d), so that the mean is h_d S_d and the half difference h_d Q_d.
// (Folding h_d into the air3D coefficients instead was measured slower.)
template <typename T, int D, int DYN>
__device__ __forceinline__ T lf_combine_raw(const StageParams& P, const T* xc, T c, T s, const T* S, const T* Q,
                                            const T* h, bool alpha_global) {
    T pb[D], dd[D];
#pragma unroll
    for (int d = 0; d < D; ++d) {
        pb[d] = S[d] * h[d];
        dd[d] = Q[d] * h[d];
    }
    return lf_combine<T, D, DYN>(P, xc, c, s, pb, dd, alpha_global);
}

// Whether a dynamics reads the coordinate of dimension d (the others are not computed).
template <int D, int DYN>
__host__ __device__ constexpr bool uses_coord(int d) {
    constexpr int B = dyn_base(DYN);
    return (B == HJ_DYN_DOUBLE_INTEGRATOR && d == 1) || (B == HJ_DYN_AIR3D && d <= 1) ||
           (B == HJ_DYN_DUBINS4D && d == 3) || (B == HJ_DYN_ROTATE && d <= 1) || (B == HJ_DYN_ROCKETS && d == 0);
}

// ydot at grid index idx from the one-sided derivatives (already divided by dx).
template <typename T, int D, int DYN>
__device__ __forceinline__ T lf_term_dyn(const StageParams& P, const int* idx, const T* pm, const T* pp) {
    T pb[D], dd[D], x[D];
#pragma unroll
    for (int d = 0; d < D; ++d) {
        pb[d] = T(0.5) * (pm[d] + pp[d]);
        dd[d] = T(0.5) * (pp[d] - pm[d]);
        x[d] = coord(SP<T>::lo(P, d), idx[d], SP<T>::dx(P, d));
    }
    T c = T(0), s = T(0);
    if constexpr (uses_angle<D, DYN>()) {
        const T* tr = Trig<T>::get(P);
        c = tr[idx[2]];
        s = tr[P.g.n[2] + idx[2]];
    }
    return lf_combine<T, D, DYN>(P, x, c, s, pb, dd, P.alpha_global);
}

template <typename T, int D>
__device__ __forceinline__ T lf_term(const StageParams& P, const int* idx, const T* pm, const T* pp) {
    switch (P.dynamics) {
    case HJ_DYN_DOUBLE_INTEGRATOR: return lf_term_dyn<T, D, HJ_DYN_DOUBLE_INTEGRATOR>(P, idx, pm, pp);
    case HJ_DYN_AIR3D:
        return P.alpha_box ? lf_term_dyn<T, D, HJ_DYN_AIR3D + kDynBox>(P, idx, pm, pp)
                           : lf_term_dyn<T, D, HJ_DYN_AIR3D>(P, idx, pm, pp);
    case HJ_DYN_DUBINS4D: return lf_term_dyn<T, D, HJ_DYN_DUBINS4D>(P, idx, pm, pp);
    case HJ_DYN_ROCKETS:
        return P.alpha_box ? lf_term_dyn<T, D, HJ_DYN_ROCKETS + kDynBox>(P, idx, pm, pp)
                           : lf_term_dyn<T, D, HJ_DYN_ROCKETS>(P, idx, pm, pp);
    case HJ_DYN_NORM:
        return P.alpha_box ? lf_term_dyn<T, D, HJ_DYN_NORM + kDynBox>(P, idx, pm, pp)
                           : lf_term_dyn<T, D, HJ_DYN_NORM>(P, idx, pm, pp);
    case HJ_DYN_ADVECT: return lf_term_dyn<T, D, HJ_DYN_ADVECT>(P, idx, pm, pp);
    case HJ_DYN_ROTATE: return lf_term_dyn<T, D, HJ_DYN_ROTATE>(P, idx, pm, pp);
    default: return T(0);
    }
}

}  // namespace hj
