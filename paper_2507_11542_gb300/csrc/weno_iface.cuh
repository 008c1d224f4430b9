// weno_iface.cuh -- WENO5 (Sec. 3.3; Jiang & Peng 2000) evaluated per grid
// interface. The right derivative p+ at node j and the left derivative p- at
// node j+1 use the same five differences
//   e1..e5 = v_{j-1}-v_{j-2}, v_j-v_{j-1}, v_{j+1}-v_j, v_{j+2}-v_{j+1}, v_{j+3}-v_{j+2}
// (mirrored), hence the same three smoothness indicators and epsilon; only
// the candidate stencils and the order of the ideal weights differ:
//
//   windows A = (e1,e2,e3), B = (e2,e3,e4), C = (e3,e4,e5)
//   SA = 13/12 (e1-2e2+e3)^2 + 1/4 (e1-4e2+3e3)^2
//   SB = 13/12 (e2-2e3+e4)^2 + 1/4 (e2-e4)^2
//   SC = 13/12 (e3-2e4+e5)^2 + 1/4 (3e3-4e4+e5)^2
//   eps = 1e-6 max(e_k^2) + floor
//   p-_{j+1} = sum_k w_k phi_k, phi = (2e1-7e2+11e3, -e2+5e3+2e4, 2e3+5e4-e5)/6,
//              w ~ (0.1, 0.6, 0.3) / (S+eps)^2 over (SA, SB, SC)
//   p+_j     = sum_k w_k psi_k, psi = (2e5-7e4+11e3, -e4+5e3+2e2, 2e3+5e2-e1)/6,
//              w ~ (0.1, 0.6, 0.3) / (S+eps)^2 over (SC, SB, SA)
//
// Evaluated here in an equivalent form (the weights sum to one):
//   p- = phi2 + (w1 T1/3 + w3 T2/6),   p+ = psi2 - (w1' T2/3 + w3' T1/6)
// with the third differences T1 = e1-3e2+3e3-e4 = tA-tB and T2 = e2-3e3+3e4-e5
// = tB-tC shared by both sides. The smoothness indicators are scaled by 4
// (S' = 13/3 t^2 + u^2), eps alike, and the ideal weights by 10, which leaves
// every weight unchanged; both results come out times 6. All differences and
// both results are raw (not divided by dx): the caller scales them once per
// node and dimension, by 1/(12 dx) (iface_times6).
#pragma once

#include <cuda_runtime.h>

#include <type_traits>

#include "../../include/hj.h"

namespace hj {

__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// FP32, in the rescaled form of the FP64 interface below (smoothness values
// and epsilon times 4, ideal weights times 10, results times 6; the caller
// divides the 6 out with 1/(2 dx)), with one reciprocal per weight and per
// side: (S' + eps')^2 >= (4e-18)^2 stays a normal number, so the approximate
// reciprocals neither overflow nor divide by zero. No a*b + c is left for the
// compiler to contract, so every inlined copy rounds alike.
__device__ __forceinline__ void weno_iface(float e1, float e2, float e3, float e4, float e5, float floor_raw,
                                           float& pp_j, float& pm_j1) {
    const float tA = fmaf(-2.0f, e2, e1) + e3;
    const float tB = fmaf(-2.0f, e3, e2) + e4;
    const float tC = fmaf(-2.0f, e4, e3) + e5;
    const float uA = fmaf(2.0f, e3 - e2, tA);  // e1 - 4e2 + 3e3
    const float uB = e2 - e4;
    const float uC = fmaf(2.0f, e3 - e4, tC);  // 3e3 - 4e4 + e5
    const float SA = fmaf(uA, uA, (13.0f / 3.0f * tA) * tA);
    const float SB = fmaf(uB, uB, (13.0f / 3.0f * tB) * tB);
    const float SC = fmaf(uC, uC, (13.0f / 3.0f * tC) * tC);
    const float amax = fmaxf(fmaxf(fmaxf(fabsf(e1), fabsf(e2)), fmaxf(fabsf(e3), fabsf(e4))), fabsf(e5));
    const float eps = fmaf(4e-6f, amax * amax, 4.0f * floor_raw);
    const float sA = SA + eps, sB = SB + eps, sC = SC + eps;
    const float rA = rcp_approx(sA * sA);
    const float rB = rcp_approx(sB * sB);
    const float rC = rcp_approx(sC * sC);
    const float T1 = tA - tB, T2 = tB - tC;
    const float X = rA * T1, Y = rC * T2;
    const float XY = __fadd_rn(X, Y);
    const float numL = fmaf(2.0f, XY, Y);  // 2X + 3Y
    const float numR = fmaf(2.0f, XY, X);  // 3X + 2Y
    const float DL = fmaf(3.0f, rC, fmaf(6.0f, rB, rA));
    const float DR = fmaf(3.0f, rA, fmaf(6.0f, rB, rC));
    const float phi6 = fmaf(5.0f, e3, fmaf(2.0f, e4, -e2));  // 6 phi2
    const float psi6 = fmaf(3.0f, uB, phi6);                 // 6 psi2
    pm_j1 = fmaf(numL, rcp_approx(DL), phi6);
    pp_j = fmaf(-numR, rcp_approx(DR), psi6);
}

// Integer maximum of non-negative doubles (their bit patterns order alike):
// keeps the epsilon's max off the FP64 pipe.
__device__ __forceinline__ double nonneg_max(double a, double b) {
    const long long ia = __double_as_longlong(a), ib = __double_as_longlong(b);
    return __longlong_as_double(ia > ib ? ia : ib);
}

__device__ __forceinline__ double abs_bits(double a) {
    return __longlong_as_double(__double_as_longlong(a) & 0x7fffffffffffffffLL);
}

// 1/x for a positive normal double: the hardware estimate refined by two
// Newton-Raphson steps r <- r + r (1 - x r) (each squares the relative error).
__device__ __forceinline__ double rcp_newton(double x) {
    double r;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
    double e = fma(-x, r, 1.0);
    r = fma(r, e, r);
    e = fma(-x, r, 1.0);
    return fma(r, e, r);
}

// FP64. Weights normalised by products of the d_k = (S'_k + eps')^2:
//   w_k = c_k prod_{i!=k} d_i / sum_m c_m prod_{i!=m} d_i,
// and both sides share one reciprocal 1/(DL DR). Three rescalings that leave
// every weight unchanged save FP64 operations (the FP64 pipe bounds this
// kernel):
//   * the smoothness indicators and epsilon times 4: S' = 13/3 t^2 + u^2,
//     eps' = 4e-6 max(e_k^2) + 4 floor;
//   * the ideal weights times 10: DL = PA + 6 PB + 3 PC, DR = 3 PA + 6 PB + PC;
//   * both results times 6: 6 p- = (-e2 + 5e3 + 2e4) + (2X + 3Y)/DL and
//     6 p+ = 6 phi2 + 3 (e2 - e4) - (3X + 2Y)/DR, X = PA T1, Y = PC T2
//     (2X + 3Y = 2(X+Y) + Y, 3X + 2Y = 2(X+Y) + X).
// The caller divides the factor 6 out with its 1/(2 dx) (iface_times6).
// The core takes what consecutive interfaces along a line share (Weno5Line):
// tA, tB, tC (the second differences of the windows' first differences), q =
// 13/3 t^2 for each, the differences d23 = e3 - e2 and d34 = e4 - e3 of the
// first differences, and the third differences T1 = tA - tB, T2 = tB - tC.
__device__ __forceinline__ void weno_core(double e1, double e2, double e3, double e4, double e5, double tA, double tB,
                                          double tC, double qA, double qB, double qC, double d23, double d34,
                                          double T1, double T2, double floor_raw, double& pp_j, double& pm_j1) {
    const double uA = fma(2.0, d23, tA);   // e1 - 4e2 + 3e3
    const double uB = e2 - e4;
    const double uC = fma(-2.0, d34, tC);  // 3e3 - 4e4 + e5
    const double SA = fma(uA, uA, qA);
    const double SB = fma(uB, uB, qB);
    const double SC = fma(uC, uC, qC);
    const double amax = nonneg_max(nonneg_max(nonneg_max(abs_bits(e1), abs_bits(e2)),
                                              nonneg_max(abs_bits(e3), abs_bits(e4))), abs_bits(e5));
    const double eps = fma(4e-6, amax * amax, 4.0 * floor_raw);
    // sA, sB, sC scaled by the power of two that brings the largest into
    // [1, 2): an exact integer subtraction on the bit patterns of these
    // positive normal numbers. eps bounds their ratios (s_min >= 3e-8 s_max:
    // S' <= 133.4 max(e_k^2)), so DL and DR stay within [9e-16, 160] and one
    // shared reciprocal serves every window, flat and tiny ones included.
    // The weights do not change.
    const long long bA = __double_as_longlong(SA + eps), bB = __double_as_longlong(SB + eps),
                    bC = __double_as_longlong(SC + eps);
    const long long bm = bA > bB ? (bA > bC ? bA : bC) : (bB > bC ? bB : bC);
    const long long shift = (bm & 0x7ff0000000000000LL) - 0x3ff0000000000000LL;
    const double sA = __longlong_as_double(bA - shift), sB = __longlong_as_double(bB - shift),
                 sC = __longlong_as_double(bC - shift);
    const double dA = sA * sA, dB = sB * sB, dC = sC * sC;
    const double PA = dB * dC, PB = dA * dC, PC = dA * dB;
    const double X = PA * T1, Y = PC * T2;
    // no a*b + c is left for the compiler to contract: every inlined copy of
    // this function rounds alike, so results do not depend on which thread
    // role evaluates an interface
    const double XY = __dadd_rn(X, Y);
    const double numL = fma(2.0, XY, Y);  // 2X + 3Y
    const double numR = fma(2.0, XY, X);  // 3X + 2Y
    const double DL = fma(3.0, PC, fma(6.0, PB, PA));
    const double DR = fma(3.0, PA, fma(6.0, PB, PC));
    const double phi6 = fma(5.0, e3, fma(2.0, e4, -e2));  // 6 phi2
    const double psi6 = fma(3.0, uB, phi6);               // 6 psi2
    const double r = rcp_newton(DL * DR);
    pm_j1 = fma(numL * DR, r, phi6);
    pp_j = fma(-numR * DL, r, psi6);
}

// 13/3 t^2, the share of t in the rescaled smoothness indicator
__device__ __forceinline__ double curv_sq(double t) { return (13.0 / 3.0 * t) * t; }

// Six times the FP64 one-sided derivatives (weno_core), from the five first
// differences: t as differences of the d = e_{k+1} - e_k.
__device__ __forceinline__ void weno_iface(double e1, double e2, double e3, double e4, double e5, double floor_raw,
                                           double& pp_j, double& pm_j1) {
    const double d12 = e2 - e1, d23 = e3 - e2, d34 = e4 - e3, d45 = e5 - e4;
    const double tA = d23 - d12, tB = d34 - d23, tC = d45 - d34;
    weno_core(e1, e2, e3, e4, e5, tA, tB, tC, curv_sq(tA), curv_sq(tB), curv_sq(tC), d23, d34, tA - tB, tB - tC,
              floor_raw, pp_j, pm_j1);
}

// Whether an interface evaluation returns six times the derivatives (WENO5,
// both precisions; the caller scales by 1/(12 dx) instead of 1/(2 dx)) or the
// derivatives themselves (the ENO schemes).
template <typename T, int SCHEME>
__host__ __device__ constexpr bool iface_times6() {
    return SCHEME == HJ_WENO5;
}

// FP64 WENO5 along a grid line, one interface after the other: the interface
// between nodes j and j+1 reuses four of the five first differences, two of
// the three differences d, two of the three values tA, tB, tC and their
// squares, and one of the two third differences of the interface before it,
// so each step computes one of each. The results are those of weno_iface,
// bit for bit (the same operations on the same operands).
struct Weno5Line {
    double e[5];   // first differences of the current window
    double d[3];   // d23, d34, d45: differences of consecutive e
    double t[3];   // tA, tB, tC
    double sq[3];  // 13/3 of their squares
    double T[2];   // T1, T2
    // the window of the values v0..v5 at nodes j-2 .. j+3
    __device__ __forceinline__ void start(double v0, double v1, double v2, double v3, double v4, double v5) {
        e[0] = v1 - v0; e[1] = v2 - v1; e[2] = v3 - v2; e[3] = v4 - v3; e[4] = v5 - v4;
        const double d12 = e[1] - e[0];
        d[0] = e[2] - e[1]; d[1] = e[3] - e[2]; d[2] = e[4] - e[3];
        t[0] = d[0] - d12; t[1] = d[1] - d[0]; t[2] = d[2] - d[1];
        sq[0] = curv_sq(t[0]); sq[1] = curv_sq(t[1]); sq[2] = curv_sq(t[2]);
        T[0] = t[0] - t[1]; T[1] = t[1] - t[2];
    }
    // slide by one node: v4, v5 are the values at the new window's last two nodes
    __device__ __forceinline__ void slide(double v4, double v5) {
        e[0] = e[1]; e[1] = e[2]; e[2] = e[3]; e[3] = e[4]; e[4] = v5 - v4;
        d[0] = d[1]; d[1] = d[2]; d[2] = e[4] - e[3];
        t[0] = t[1]; t[1] = t[2]; t[2] = d[2] - d[1];
        sq[0] = sq[1]; sq[1] = sq[2]; sq[2] = curv_sq(t[2]);
        T[0] = T[1]; T[1] = t[1] - t[2];
    }
    __device__ __forceinline__ void eval(double floor_raw, double& pp_j, double& pm_j1) const {
        weno_core(e[0], e[1], e[2], e[3], e[4], t[0], t[1], t[2], sq[0], sq[1], sq[2], d[0], d[1], T[0], T[1],
                  floor_raw, pp_j, pm_j1);
    }
};

// Second-order ENO (Sec. 3.2; Osher & Fedkiw 2003 Sec. 3.3) per interface.
// Both one-sided derivatives at the interface between nodes j and j+1 (p+ of
// j and p- of j+1) take the stencil that starts at j: the first difference
// across the interface plus or minus half the smaller (in magnitude; ties to
// the left) of the second differences centred at j and j+1. In raw
// (undivided) units, from the values v0..v3 at nodes j-1 .. j+2:
//   e = v2 - v1, dL = e - (v1 - v0), dR = (v3 - v2) - e,
//   c = |dL| <= |dR| ? dL : dR,  p+_j = e - c/2,  p-_{j+1} = e + c/2.
// |a| <= |b|: for FP64 on the bit patterns (an integer comparison, exact for
// finite values).
__device__ __forceinline__ bool abs_le(double a, double b) {
    return (__double_as_longlong(a) & 0x7fffffffffffffffLL) <= (__double_as_longlong(b) & 0x7fffffffffffffffLL);
}
__device__ __forceinline__ bool abs_le(float a, float b) { return fabsf(a) <= fabsf(b); }

template <typename T>
__device__ __forceinline__ void eno2_iface(T v0, T v1, T v2, T v3, T& pp_j, T& pm_j1) {
    const T e = v2 - v1;
    const T dL = e - (v1 - v0);
    const T dR = (v3 - v2) - e;
    const T c = abs_le(dL, dR) ? dL : dR;
    pp_j = e - T(0.5) * c;
    pm_j1 = e + T(0.5) * c;
}

// Third-order ENO (Sec. 3.2; Osher & Fedkiw 2003 Sec. 3.3) per interface.
// p+ of node j and p- of node j+1 both start from k = j, so they take the
// same second-difference choice (c; k* = j-1 on the left, else j) and the
// same third-difference choice (c*, the smaller of the two differences next
// to k*; ties to the left); only the polynomial coefficients differ. In raw
// units, from e_m = v_{m+1} - v_m, second differences d2_m = e_m - e_{m-1}
// and third differences d3 = d2_{m+1} - d2_m (the divided differences are
// e/dx, d2/(2 dx^2), d3/(6 dx^3)):
//   p+_j     = e_j - c/2 + c* (left ? -1 : 2)/6
//   p-_{j+1} = e_j + c/2 + c* (left ? 2 : -1)/6
// from the values v0..v5 at nodes j-2 .. j+3.
template <typename T>
__device__ __forceinline__ void eno3_iface(T v0, T v1, T v2, T v3, T v4, T v5, T& pp_j, T& pm_j1) {
    const T e0 = v1 - v0, e1 = v2 - v1, e2 = v3 - v2, e3 = v4 - v3, e4 = v5 - v4;
    const T dm = e1 - e0, d0 = e2 - e1, d1 = e3 - e2, d2 = e4 - e3;  // second differences at j-1, j, j+1, j+2
    const bool left = abs_le(d0, d1);
    const T c = left ? d0 : d1;
    const T a = left ? d0 - dm : d1 - d0;  // third differences next to k*
    const T b = left ? d1 - d0 : d2 - d1;
    const T cs = abs_le(a, b) ? a : b;
    const T third = cs * T(1.0 / 6.0);
    pp_j = e2 - T(0.5) * c + (left ? -third : T(2) * third);
    pm_j1 = e2 + T(0.5) * c + (left ? T(2) * third : -third);
}

// The interface between nodes j and j+1 from the values at nodes j-2 .. j+3
// (WENO5 and ENO3 read all six, ENO2 the middle four, ENO1 the middle two:
// first order takes the difference across the interface for both sides).
template <int SCHEME, typename T>
__device__ __forceinline__ void iface_at(T v0, T v1, T v2, T v3, T v4, T v5, T floor_raw, T& pp_j, T& pm_j1) {
    if constexpr (SCHEME == HJ_ENO1) {
        pp_j = pm_j1 = v3 - v2;
    } else if constexpr (SCHEME == HJ_ENO2) {
        eno2_iface(v1, v2, v3, v4, pp_j, pm_j1);
    } else if constexpr (SCHEME == HJ_ENO3) {
        eno3_iface(v0, v1, v2, v3, v4, v5, pp_j, pm_j1);
    } else {
        weno_iface(v1 - v0, v2 - v1, v3 - v2, v4 - v3, v5 - v4, floor_raw, pp_j, pm_j1);
    }
}

}  // namespace hj
