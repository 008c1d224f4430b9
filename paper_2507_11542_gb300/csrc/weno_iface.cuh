// weno_iface.cuh -- WENO5 (Sec. 3.3; Jiang & Peng 2000) evaluated per grid
// interface. The right derivative p+ at node j and the left derivative p- at
// node j+1 use the same five differences
//   e1..e5 = v_{j-1}-v_{j-2}, v_j-v_{j-1}, v_{j+1}-v_j, v_{j+2}-v_{j+1}, v_{j+3}-v_{j+2}
// (mirrored), hence the same three smoothness indicators and epsilon; only
// the candidate stencils and the ideal weights' order differ. Computing both
// from one interface halves the smoothness work per node along a dimension.
//
//   windows A = (e1,e2,e3), B = (e2,e3,e4), C = (e3,e4,e5)
//   SA = 13/12 (e1-2e2+e3)^2 + 1/4 (e1-4e2+3e3)^2
//   SB = 13/12 (e2-2e3+e4)^2 + 1/4 (e2-e4)^2
//   SC = 13/12 (e3-2e4+e5)^2 + 1/4 (3e3-4e4+e5)^2
//   p-_{j+1}: candidates (2e1-7e2+11e3, -e2+5e3+2e4, 2e3+5e4-e5)/6, weights 0.1, 0.6, 0.3 on SA, SB, SC
//   p+_j    : candidates (2e5-7e4+11e3, -e4+5e3+2e2, 2e3+5e2-e1)/6, weights 0.1, 0.6, 0.3 on SC, SB, SA
//   eps = 1e-6 max(e_k^2) + floor (raw differences; the result is divided by dx)
#pragma once

#include <cuda_runtime.h>

namespace hj {

// Smoothness indicators and epsilon of one interface.
template <typename T>
__device__ __forceinline__ void weno_smooth(T e1, T e2, T e3, T e4, T e5, T floor_raw, T& SA, T& SB, T& SC, T& eps) {
    const T c13 = T(13) / T(12);
    const T tA = e1 - T(2) * e2 + e3;
    const T tB = e2 - T(2) * e3 + e4;
    const T tC = e3 - T(2) * e4 + e5;
    const T uA = e1 - T(4) * e2 + T(3) * e3;
    const T uB = e2 - e4;
    const T uC = T(3) * e3 - T(4) * e4 + e5;
    SA = c13 * tA * tA + T(0.25) * uA * uA;
    SB = c13 * tB * tB + T(0.25) * uB * uB;
    SC = c13 * tC * tC + T(0.25) * uC * uC;
    const T m = fmax(fmax(fmax(e1 * e1, e2 * e2), fmax(e3 * e3, e4 * e4)), e5 * e5);
    eps = T(1e-6) * m + floor_raw;
}

// FP32: fast reciprocals of (S+eps)^2 >= 1e-36 (normal) and of each side's
// weight sum; candidates carry their ideal weight and the 1/6.
__device__ __forceinline__ void weno_iface(float e1, float e2, float e3, float e4, float e5, float floor_raw,
                                           float inv_dx, float& pp_j, float& pm_j1) {
    float SA, SB, SC, eps;
    weno_smooth<float>(e1, e2, e3, e4, e5, floor_raw, SA, SB, SC, eps);
    const float rA = __fdividef(1.0f, (SA + eps) * (SA + eps));
    const float rB = __fdividef(1.0f, (SB + eps) * (SB + eps));
    const float rC = __fdividef(1.0f, (SC + eps) * (SC + eps));
    // left of j+1
    const float l1 = (0.1f / 6.0f) * (2.0f * e1 - 7.0f * e2 + 11.0f * e3);
    const float l2 = (0.6f / 6.0f) * (-e2 + 5.0f * e3 + 2.0f * e4);
    const float l3 = (0.3f / 6.0f) * (2.0f * e3 + 5.0f * e4 - e5);
    const float numL = rA * l1 + rB * l2 + rC * l3;
    const float denL = 0.1f * rA + 0.6f * rB + 0.3f * rC;
    // right of j
    const float q1 = (0.1f / 6.0f) * (2.0f * e5 - 7.0f * e4 + 11.0f * e3);
    const float q2 = (0.6f / 6.0f) * (-e4 + 5.0f * e3 + 2.0f * e2);
    const float q3 = (0.3f / 6.0f) * (2.0f * e3 + 5.0f * e2 - e1);
    const float numR = rC * q1 + rB * q2 + rA * q3;
    const float denR = 0.1f * rC + 0.6f * rB + 0.3f * rA;
    pm_j1 = numL * __fdividef(inv_dx, denL);
    pp_j = numR * __fdividef(inv_dx, denR);
}

// Integer maximum of non-negative doubles (their bit patterns order alike):
// keeps the epsilon's max off the FP64 pipe.
__device__ __forceinline__ double nonneg_max(double a, double b) {
    const long long ia = __double_as_longlong(a), ib = __double_as_longlong(b);
    return __longlong_as_double(ia > ib ? ia : ib);
}

// FP64: weights normalised by products of the d_k = (S_k+eps)^2,
//   p = sum_k c_k q_k prod_{i!=k} d_i / sum_k c_k prod_{i!=k} d_i,
// and both sides share one reciprocal 1/(denL denR). When that product
// leaves [1e-290, 1e290] (nearly flat or huge data) each side divides alone,
// and an exactly flat window (den = 0) returns its zero candidate.
__device__ __forceinline__ void weno_iface(double e1, double e2, double e3, double e4, double e5, double floor_raw,
                                           double inv_dx, double& pp_j, double& pm_j1) {
    const double c13 = 13.0 / 12.0;
    const double tA = e1 - 2.0 * e2 + e3;
    const double tB = e2 - 2.0 * e3 + e4;
    const double tC = e3 - 2.0 * e4 + e5;
    const double uA = e1 - 4.0 * e2 + 3.0 * e3;
    const double uB = e2 - e4;
    const double uC = 3.0 * e3 - 4.0 * e4 + e5;
    const double SA = c13 * tA * tA + 0.25 * uA * uA;
    const double SB = c13 * tB * tB + 0.25 * uB * uB;
    const double SC = c13 * tC * tC + 0.25 * uC * uC;
    const double m = nonneg_max(nonneg_max(nonneg_max(e1 * e1, e2 * e2), nonneg_max(e3 * e3, e4 * e4)), e5 * e5);
    const double eps = 1e-6 * m + floor_raw;
    const double dA = (SA + eps) * (SA + eps);
    const double dB = (SB + eps) * (SB + eps);
    const double dC = (SC + eps) * (SC + eps);
    const double PA = dB * dC, PB = dA * dC, PC = dA * dB;
    const double l1 = (0.1 / 6.0) * (2.0 * e1 - 7.0 * e2 + 11.0 * e3);
    const double l2 = (0.6 / 6.0) * (-e2 + 5.0 * e3 + 2.0 * e4);
    const double l3 = (0.3 / 6.0) * (2.0 * e3 + 5.0 * e4 - e5);
    const double q1 = (0.1 / 6.0) * (2.0 * e5 - 7.0 * e4 + 11.0 * e3);
    const double q2 = (0.6 / 6.0) * (-e4 + 5.0 * e3 + 2.0 * e2);
    const double q3 = (0.3 / 6.0) * (2.0 * e3 + 5.0 * e2 - e1);
    const double numL = PA * l1 + PB * l2 + PC * l3;
    const double denL = 0.1 * PA + 0.6 * PB + 0.3 * PC;
    const double numR = PC * q1 + PB * q2 + PA * q3;
    const double denR = 0.1 * PC + 0.6 * PB + 0.3 * PA;
    const double den2 = denL * denR;
    // range test on the exponent field (integer pipe): 1e-290 < den2 < 1e290
    const long long bits = __double_as_longlong(den2);
    const int expo = (int)((bits >> 52) & 0x7ff);
    if (expo > 60 && expo < 1986) {
        const double r = inv_dx / den2;
        pm_j1 = numL * denR * r;
        pp_j = numR * denL * r;
    } else {
        // l2 / 0.6 and q2 / 0.6 are the unweighted central candidates
        pm_j1 = denL > 0.0 ? numL * inv_dx / denL : l2 / 0.6 * inv_dx;
        pp_j = denR > 0.0 ? numR * inv_dx / denR : q2 / 0.6 * inv_dx;
    }
}

}  // namespace hj
