/*
 * hj_oracle.c -- plain FP64 CPU oracle of the LevelSetPy level-set step
 * (arXiv 2507.11542, Sections 2-6). Written for reading, not for speed:
 * every quantity is computed the way the paper (and the textbook it cites,
 * Osher & Fedkiw 2003, Sec. 3.3-3.4) defines it, with no fusion or blocking.
 *
 * TEST INFRASTRUCTURE ONLY: the CUDA library never links or calls this file.
 *
 * Readings of passages where the paper is silent, garbled or inconsistent:
 *  R1 (Sec. 3, forward/backward differences): the paper prints D- and D+ with
 *     swapped labels; p- is the backward difference (v_i - v_{i-1})/dx and p+
 *     the forward difference (v_{i+1} - v_i)/dx, as its upwinding rule needs.
 *  R2 (Sec. 3.2, Listing 4): a tie |D2_k| == |D2_{k+1}| picks the left
 *     candidate, as the ENO3 selector of Sec. 3.2 does for D3.
 *  R3 (Sec. 2.1 boundary values): extrapolated ghosts continue the outermost
 *     slope away from the zero level set, g_m = v_0 + m*|v_0 - v_1|*sign(v_0);
 *     ORC_EXTRAP_LINEAR instead uses the signed slope v_0 - v_1.
 *  R4 (Sec. 3.3): WENO5 follows Jiang & Peng with
 *     eps = 1e-6 * max(v_k^2) + 1e-99.
 *  R5 (Sec. 4): alpha_d is evaluated per node (x-dependent, bounded over all
 *     p); the CFL bound is max over nodes of sum_d alpha_d/dx_d, as printed.
 *  R6 (Sec. 5, Listing 6): dt = min(t_slice - t, max_step, cfl * stepBound)
 *     with stepBound = 1/stepBoundInv, computed before the first substep and
 *     reused by the other two; t advances by dt.
 *  R7 (Sec. 6.1): the backward reachable tube inequality is applied as
 *     V_tau = min(0, Hg_LF) at every stage (ORC_BRT_MIN0), or as
 *     V <- min(V_new, V_old) after each full step (ORC_BRT_MINV).
 *  R12 (Sec. 4, alpha = max |H_p| "over" an unstated set of gradients; the
 *     rockets listing passes dL, dR to its dissipation routine): with
 *     alpha_box, alpha_d at a node is the maximum of |dHg/dp_d| over the box
 *     of gradients spanned by that node's p- and p+ (local in x and p). The
 *     CFL bound keeps the R5 value, the maximum over every p, which bounds
 *     the box maximum from above.
 */
#include "hj_oracle.h"

#include <float.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORC_EINVAL (-1)
#define ORC_ENOMEM (-2)

static int grid_ok(const orc_grid* g) {
    if (!g || g->ndim < 1 || g->ndim > 4) return 0;
    for (int d = 0; d < g->ndim; ++d) {
        int periodic = (g->periodic_mask >> d) & 1u;
        if (g->n[d] < (periodic ? 1 : 2)) return 0;
        if (!(g->hi[d] > g->lo[d])) return 0;
    }
    return 1;
}

int64_t orc_num_nodes(const orc_grid* g) {
    int64_t total = 1;
    for (int d = 0; d < g->ndim; ++d) total *= g->n[d];
    return total;
}

/* Sec. 2.1: uniform cell size; a periodic dimension has n cells on [lo, hi). */
double orc_spacing(const orc_grid* g, int d) {
    int periodic = (g->periodic_mask >> d) & 1u;
    double cells = periodic ? (double)g->n[d] : (double)(g->n[d] - 1);
    return (g->hi[d] - g->lo[d]) / cells;
}

double orc_coord(const orc_grid* g, int d, int64_t i) {
    return g->lo[d] + (double)i * orc_spacing(g, d);
}

static double sgn(double v) { return (v > 0.0) ? 1.0 : ((v < 0.0) ? -1.0 : 0.0); }

/* ------------------------------------------------------------------------
 * Ghost cells (Sec. 2.1; Listings 3-4 "patch data according to grid.bdry").
 * out[k] = value at node k-3 for k = 0 .. n+5.
 * ---------------------------------------------------------------------- */
int orc_pad_line(const double* line, int64_t n, int periodic, int extrap, double* out) {
    if (!line || !out || n < 1) return ORC_EINVAL;
    if (!periodic && n < 2) return ORC_EINVAL;
    for (int64_t k = 0; k < n + 6; ++k) {
        int64_t i = k - 3;
        if (i >= 0 && i < n) {
            out[k] = line[i];
        } else if (periodic) {
            int64_t j = i % n;
            if (j < 0) j += n;
            out[k] = line[j];
        } else {
            /* R3: linear continuation of the outermost slope. */
            double edge, inner;
            int64_t m; /* how many cells beyond the edge node */
            if (i < 0) { edge = line[0]; inner = line[1]; m = -i; }
            else       { edge = line[n - 1]; inner = line[n - 2]; m = i - (n - 1); }
            double slope = (extrap == ORC_EXTRAP_LINEAR) ? (edge - inner)
                                                         : fabs(edge - inner) * sgn(edge);
            out[k] = edge + (double)m * slope;
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------
 * Divided differences on a padded line (Sec. 3.2, Listing 4). With
 * v(j) = padded[j+3]:
 *   D1(j) = D^1_{j+1/2} = (v(j+1) - v(j)) / dx
 *   D2(j) = D^2_j       = (D^1_{j+1/2} - D^1_{j-1/2}) / (2 dx)
 *   D3(j) = D^3_{j+1/2} = (D^2_{j+1} - D^2_j) / (3 dx)
 * ---------------------------------------------------------------------- */
typedef struct { const double* p; double dx; } line_t;
static double V_(const line_t* L, int64_t j) { return L->p[j + 3]; }
static double D1(const line_t* L, int64_t j) { return (V_(L, j + 1) - V_(L, j)) / L->dx; }
static double D2(const line_t* L, int64_t j) { return (D1(L, j) - D1(L, j - 1)) / (2.0 * L->dx); }
static double D3(const line_t* L, int64_t j) { return (D2(L, j + 1) - D2(L, j)) / (3.0 * L->dx); }

/* ENO polynomial derivative at node i built from the stencil that starts at
 * k (k = i-1 for p-, k = i for p+), Osher & Fedkiw Sec. 3.3:
 *   Q1' = D^1_{k+1/2}
 *   c   = D^2_k if |D^2_k| <= |D^2_{k+1}| else D^2_{k+1};  k* = k-1 or k
 *   Q2' = c (2(i-k) - 1) dx
 *   c*  = D^3_{k*+1/2} if |D^3_{k*+1/2}| <= |D^3_{k*+3/2}| else D^3_{k*+3/2}
 *   Q3' = c* (3(i-k*)^2 - 6(i-k*) + 2) dx^2                                   */
static double eno_derivative(const line_t* L, int order, int64_t i, int64_t k) {
    double q1 = D1(L, k);
    if (order == 1) return q1;
    double c;
    int64_t kstar;
    if (fabs(D2(L, k)) <= fabs(D2(L, k + 1))) { c = D2(L, k); kstar = k - 1; }   /* R2 */
    else                                     { c = D2(L, k + 1); kstar = k; }
    double q2 = c * (double)(2 * (i - k) - 1) * L->dx;
    if (order == 2) return q1 + q2;
    double cs;
    if (fabs(D3(L, kstar)) <= fabs(D3(L, kstar + 1))) cs = D3(L, kstar);
    else                                              cs = D3(L, kstar + 1);
    double r = (double)(i - kstar);
    double q3 = cs * (3.0 * r * r - 6.0 * r + 2.0) * L->dx * L->dx;
    return q1 + q2 + q3;
}

/* WENO5 (Sec. 3.3; Jiang & Peng 2000; Osher & Fedkiw Sec. 3.4), R4. */
double orc_weno5(const double v[5], int ideal) {
    const double v1 = v[0], v2 = v[1], v3 = v[2], v4 = v[3], v5 = v[4];
    /* the three third-order ENO candidates */
    double phi1 = v1 / 3.0 - 7.0 * v2 / 6.0 + 11.0 * v3 / 6.0;
    double phi2 = -v2 / 6.0 + 5.0 * v3 / 6.0 + v4 / 3.0;
    double phi3 = v3 / 3.0 + 5.0 * v4 / 6.0 - v5 / 6.0;
    double w1, w2, w3;
    if (ideal) {
        w1 = 0.1; w2 = 0.6; w3 = 0.3;
    } else {
        /* smoothness indicators */
        double S1 = 13.0 / 12.0 * (v1 - 2.0 * v2 + v3) * (v1 - 2.0 * v2 + v3)
                  + 0.25 * (v1 - 4.0 * v2 + 3.0 * v3) * (v1 - 4.0 * v2 + 3.0 * v3);
        double S2 = 13.0 / 12.0 * (v2 - 2.0 * v3 + v4) * (v2 - 2.0 * v3 + v4)
                  + 0.25 * (v2 - v4) * (v2 - v4);
        double S3 = 13.0 / 12.0 * (v3 - 2.0 * v4 + v5) * (v3 - 2.0 * v4 + v5)
                  + 0.25 * (3.0 * v3 - 4.0 * v4 + v5) * (3.0 * v3 - 4.0 * v4 + v5);
        double vmax2 = v1 * v1;
        if (v2 * v2 > vmax2) vmax2 = v2 * v2;
        if (v3 * v3 > vmax2) vmax2 = v3 * v3;
        if (v4 * v4 > vmax2) vmax2 = v4 * v4;
        if (v5 * v5 > vmax2) vmax2 = v5 * v5;
        double eps = 1e-6 * vmax2 + 1e-99;
        double a1 = 0.1 / ((S1 + eps) * (S1 + eps));
        double a2 = 0.6 / ((S2 + eps) * (S2 + eps));
        double a3 = 0.3 / ((S3 + eps) * (S3 + eps));
        double sum = a1 + a2 + a3;
        w1 = a1 / sum; w2 = a2 / sum; w3 = a3 / sum;
    }
    return w1 * phi1 + w2 * phi2 + w3 * phi3;
}

int orc_upwind_line(int scheme, int weno_ideal, const double* padded, int64_t n, double dx,
                    double* pm, double* pp) {
    if (!padded || !pm || !pp || n < 1 || !(dx > 0.0)) return ORC_EINVAL;
    if (scheme != ORC_ENO1 && scheme != ORC_ENO2 && scheme != ORC_ENO3 && scheme != ORC_WENO5)
        return ORC_EINVAL;
    line_t L = {padded, dx};
    for (int64_t i = 0; i < n; ++i) {
        if (scheme == ORC_WENO5) {
            /* p-: backward differences D-v at i-2..i+2; p+: forward
             * differences D+v at i+2..i-2 (mirrored stencil). */
            double vl[5] = {D1(&L, i - 3), D1(&L, i - 2), D1(&L, i - 1), D1(&L, i), D1(&L, i + 1)};
            double vr[5] = {D1(&L, i + 2), D1(&L, i + 1), D1(&L, i), D1(&L, i - 1), D1(&L, i - 2)};
            pm[i] = orc_weno5(vl, weno_ideal);
            pp[i] = orc_weno5(vr, weno_ideal);
        } else {
            int order = (scheme == ORC_ENO1) ? 1 : (scheme == ORC_ENO2 ? 2 : 3);
            pm[i] = eno_derivative(&L, order, i, i - 1);
            pp[i] = eno_derivative(&L, order, i, i);
        }
    }
    return 0;
}

static int64_t stride_of(const orc_grid* g, int d) {
    int64_t s = 1;
    for (int e = 0; e < d; ++e) s *= g->n[e];
    return s;
}

int orc_upwind(const orc_grid* g, const orc_method* m, const double* V, int dim, double* pm, double* pp) {
    if (!grid_ok(g) || !m || !V || !pm || !pp || dim < 0 || dim >= g->ndim) return ORC_EINVAL;
    int64_t n = g->n[dim];
    int64_t stride = stride_of(g, dim);
    int64_t total = orc_num_nodes(g);
    int periodic = (g->periodic_mask >> dim) & 1u;
    double dx = orc_spacing(g, dim);
    double* line = (double*)malloc(sizeof(double) * (size_t)n);
    double* padded = (double*)malloc(sizeof(double) * (size_t)(n + 6));
    double* lm = (double*)malloc(sizeof(double) * (size_t)n);
    double* lp = (double*)malloc(sizeof(double) * (size_t)n);
    if (!line || !padded || !lm || !lp) { free(line); free(padded); free(lm); free(lp); return ORC_ENOMEM; }
    int rc = 0;
    /* every line along `dim` starts at a node whose index along dim is 0 */
    for (int64_t start = 0; start < total && rc == 0; ++start) {
        if ((start / stride) % n != 0) continue;
        for (int64_t i = 0; i < n; ++i) line[i] = V[start + i * stride];
        rc = orc_pad_line(line, n, periodic, m->extrap, padded);
        if (rc == 0) rc = orc_upwind_line(m->scheme, m->weno_ideal, padded, n, dx, lm, lp);
        for (int64_t i = 0; i < n && rc == 0; ++i) {
            pm[start + i * stride] = lm[i];
            pp[start + i * stride] = lp[i];
        }
    }
    free(line); free(padded); free(lm); free(lp);
    return rc;
}

/* ------------------------------------------------------------------------
 * Hamiltonians (Sec. 4; the game form of Sec. 6.1). Hg(x, p) is the optimum
 * over bounded controls of p . f(x, u, d): a maximising player contributes
 * +bound*|coefficient|, a minimising player -bound*|coefficient|.
 * ---------------------------------------------------------------------- */
int orc_hamiltonian(const orc_method* m, int ndim, const double* x, const double* p, double* hg) {
    const double* q = m->params;
    switch (m->dynamics) {
    case ORC_DYN_DOUBLE_INTEGRATOR: /* x0' = x1, x1' = u, |u| <= umax, u minimises */
        if (ndim != 2) return ORC_EINVAL;
        *hg = p[0] * x[1] - q[0] * fabs(p[1]);
        return 0;
    case ORC_DYN_AIR3D: { /* x' = -va + vb cos(psi) + a y, y' = vb sin(psi) - a x, psi' = b - a */
        if (ndim != 3) return ORC_EINVAL;
        double va = q[0], vb = q[1], amax = q[2], bmax = q[3];
        double drift = p[0] * (-va + vb * cos(x[2])) + p[1] * (vb * sin(x[2]));
        /* a (|a| <= amax) maximises a*(p0 y - p1 x - p2); b (|b| <= bmax) minimises b*p2 */
        *hg = drift + amax * fabs(p[0] * x[1] - p[1] * x[0] - p[2]) - bmax * fabs(p[2]);
        return 0;
    }
    case ORC_DYN_DUBINS4D: { /* x' = v cos th, y' = v sin th, th' = w, v' = acc; both minimise */
        if (ndim != 4) return ORC_EINVAL;
        double wmax = q[0], accmax = q[1];
        *hg = x[3] * (p[0] * cos(x[2]) + p[1] * sin(x[2])) - wmax * fabs(p[2]) - accmax * fabs(p[3]);
        return 0;
    }
    case ORC_DYN_NORM: { /* level-set motion in the normal direction: v_t + c|grad v| = 0 */
        double s = 0.0;
        for (int d = 0; d < ndim; ++d) s += p[d] * p[d];
        *hg = -q[0] * sqrt(s);
        return 0;
    }
    case ORC_DYN_ADVECT: { /* level-set equation v_t + F . grad v = 0 with constant F = c (Sec. 3) */
        double s = 0.0;
        for (int d = 0; d < ndim; ++d) s += q[d] * p[d];
        *hg = -s;
        return 0;
    }
    case ORC_DYN_ROTATE: /* F = omega (-x1, x0) in the plane of dims 0 and 1 */
        if (ndim < 2) return ORC_EINVAL;
        *hg = -(p[0] * (-q[0] * x[1]) + p[1] * (q[0] * x[0]));
        return 0;
    case ORC_DYN_ROCKETS: {
        /* Sec. 6.1, dynamics as they stand inside the game's Hamiltonian (reading):
         * x' = a cos th + ue x, z' = a sin th + a - g + up x, th' = up - ue, the
         * evader's thrust ue maximising and the pursuer's up minimising:
         * p . f = p0 a cos th + p1 (a sin th + a - g) + ue (p0 x - p2) + up (p1 x + p2). */
        if (ndim != 3) return ORC_EINVAL;
        double a = q[0], g = q[1], ue = q[2], up = q[3];
        *hg = p[0] * a * cos(x[2]) + p[1] * (a * sin(x[2]) + a - g) + ue * fabs(p[0] * x[0] - p[2]) -
              up * fabs(p[1] * x[0] + p[2]);
        return 0;
    }
    default:
        return ORC_EINVAL;
    }
}

/* alpha_d(x) = max over controls of |f_d(x, u, d)| = sup over p of |dHg/dp_d| (R5). */
int orc_alpha(const orc_method* m, int ndim, const double* x, double* alpha) {
    const double* q = m->params;
    switch (m->dynamics) {
    case ORC_DYN_DOUBLE_INTEGRATOR:
        if (ndim != 2) return ORC_EINVAL;
        alpha[0] = fabs(x[1]);
        alpha[1] = q[0];
        return 0;
    case ORC_DYN_AIR3D: {
        if (ndim != 3) return ORC_EINVAL;
        double va = q[0], vb = q[1], amax = q[2], bmax = q[3];
        alpha[0] = fabs(-va + vb * cos(x[2])) + amax * fabs(x[1]);
        alpha[1] = fabs(vb * sin(x[2])) + amax * fabs(x[0]);
        alpha[2] = amax + bmax;
        return 0;
    }
    case ORC_DYN_DUBINS4D:
        if (ndim != 4) return ORC_EINVAL;
        alpha[0] = fabs(x[3] * cos(x[2]));
        alpha[1] = fabs(x[3] * sin(x[2]));
        alpha[2] = q[0];
        alpha[3] = q[1];
        return 0;
    case ORC_DYN_NORM:
        for (int d = 0; d < ndim; ++d) alpha[d] = q[0];
        return 0;
    case ORC_DYN_ADVECT:
        for (int d = 0; d < ndim; ++d) alpha[d] = fabs(q[d]);
        return 0;
    case ORC_DYN_ROTATE:
        if (ndim < 2) return ORC_EINVAL;
        alpha[0] = fabs(q[0] * x[1]);
        alpha[1] = fabs(q[0] * x[0]);
        for (int d = 2; d < ndim; ++d) alpha[d] = 0.0;
        return 0;
    case ORC_DYN_ROCKETS: {
        if (ndim != 3) return ORC_EINVAL;
        double a = q[0], g = q[1], ue = q[2], up = q[3];
        alpha[0] = fabs(a * cos(x[2])) + ue * fabs(x[0]);
        alpha[1] = fabs(a * sin(x[2]) + a - g) + up * fabs(x[0]);
        alpha[2] = up + ue;
        return 0;
    }
    default:
        return ORC_EINVAL;
    }
}

/* Range [*mn, *mx] of c * p over p in [lo, hi]. */
static void scaled_range(double c, double lo, double hi, double* mn, double* mx) {
    double a = c * lo, b = c * hi;
    *mn = a < b ? a : b;
    *mx = a < b ? b : a;
}

/* max |d + k sigma| over the signs sigma the box allows (plus: +1 allowed,
 * minus: -1 allowed). */
static double max_over_signs(double d, double k, int plus, int minus) {
    double best = 0.0;
    if (plus && fabs(d + k) > best) best = fabs(d + k);
    if (minus && fabs(d - k) > best) best = fabs(d - k);
    return best;
}

/* R12: the maximum of |dHg/dp_d| over the box lo <= p <= hi.
 * Linear parts of Hg contribute a constant derivative. A term c |l . p|
 * contributes c sigma l_d, sigma = sign(l . p); the box allows sigma = +1 if
 * max over the box of l . p >= 0 and sigma = -1 if its min <= 0 (both where
 * the box reaches the kink). A derivative that involves two such terms takes
 * its largest value when both signs can be equal at one point of the box,
 * which is checked on the box directly. */
int orc_alpha_box(const orc_method* m, int ndim, const double* x, const double* lo, const double* hi,
                  double* alpha) {
    const double* q = m->params;
    switch (m->dynamics) {
    case ORC_DYN_NORM: {
        /* Hg = -c |p|: |dHg/dp_d| = c |p_d| / |p|, largest at the largest |p_d|
         * and the smallest |p_j| (j != d) the box holds; at p = 0 (a box that
         * is the single point 0 along d and holds 0 along the others) the
         * generalized gradient is the ball of radius c. */
        for (int d = 0; d < ndim; ++d) {
            double big = fabs(lo[d]) > fabs(hi[d]) ? fabs(lo[d]) : fabs(hi[d]);
            double others = 0.0;
            for (int j = 0; j < ndim; ++j) {
                if (j == d) continue;
                double small = (lo[j] <= 0.0 && hi[j] >= 0.0) ? 0.0 : (fabs(lo[j]) < fabs(hi[j]) ? fabs(lo[j]) : fabs(hi[j]));
                others += small * small;
            }
            if (big == 0.0) alpha[d] = (others == 0.0) ? q[0] : 0.0;
            else alpha[d] = q[0] * big / sqrt(big * big + others);
        }
        return 0;
    }
    case ORC_DYN_AIR3D: {
        /* Hg = p0 f0 + p1 f1 + amax |s| - bmax |p2|, s = p0 y - p1 x - p2:
         * dHg/dp0 = f0 + amax y sign(s), dHg/dp1 = f1 - amax x sign(s),
         * dHg/dp2 = -amax sign(s) - bmax sign(p2). */
        if (ndim != 3) return ORC_EINVAL;
        double va = q[0], vb = q[1], amax = q[2], bmax = q[3];
        double f0 = -va + vb * cos(x[2]), f1 = vb * sin(x[2]);
        double a0, b0, a1, b1;
        scaled_range(x[1], lo[0], hi[0], &a0, &b0); /* range of p0 y */
        scaled_range(x[0], lo[1], hi[1], &a1, &b1); /* range of p1 x */
        double smax = b0 - a1 - lo[2], smin = a0 - b1 - hi[2];
        int plus = smax >= 0.0, minus = smin <= 0.0;
        alpha[0] = max_over_signs(f0, amax * x[1], plus, minus);
        alpha[1] = max_over_signs(f1, -amax * x[0], plus, minus);
        /* equal signs of s and p2: s >= 0 with p2 in [max(lo2, 0), hi2], or
         * s <= 0 with p2 in [lo2, min(hi2, 0)] */
        double top = lo[2] > 0.0 ? lo[2] : 0.0, bot = hi[2] < 0.0 ? hi[2] : 0.0;
        int same = (top <= hi[2] && b0 - a1 - top >= 0.0) || (lo[2] <= bot && a0 - b1 - bot <= 0.0);
        alpha[2] = same ? amax + bmax : fabs(amax - bmax);
        return 0;
    }
    case ORC_DYN_ROCKETS: {
        /* Hg = p0 f0 + p1 f1 + ue |s1| - up |s2|, s1 = p0 x - p2, s2 = p1 x + p2:
         * dHg/dp0 = f0 + ue x sign(s1), dHg/dp1 = f1 - up x sign(s2),
         * dHg/dp2 = -ue sign(s1) - up sign(s2). */
        if (ndim != 3) return ORC_EINVAL;
        double a = q[0], g = q[1], ue = q[2], up = q[3];
        double f0 = a * cos(x[2]), f1 = a * sin(x[2]) + a - g;
        double a0, b0, a1, b1;
        scaled_range(x[0], lo[0], hi[0], &a0, &b0); /* range of p0 x */
        scaled_range(x[0], lo[1], hi[1], &a1, &b1); /* range of p1 x */
        alpha[0] = max_over_signs(f0, ue * x[0], b0 - lo[2] >= 0.0, a0 - hi[2] <= 0.0);
        alpha[1] = max_over_signs(f1, -up * x[0], b1 + hi[2] >= 0.0, a1 + lo[2] <= 0.0);
        /* equal signs: s1, s2 >= 0 needs p2 in [max(lo2, -b1), min(hi2, b0)];
         * s1, s2 <= 0 needs p2 in [max(lo2, a0), min(hi2, -a1)] */
        double l1 = lo[2] > -b1 ? lo[2] : -b1, h1 = hi[2] < b0 ? hi[2] : b0;
        double l2 = lo[2] > a0 ? lo[2] : a0, h2 = hi[2] < -a1 ? hi[2] : -a1;
        int same = (l1 <= h1) || (l2 <= h2);
        alpha[2] = same ? ue + up : fabs(ue - up);
        return 0;
    }
    default:
        /* double integrator, Dubins car, advection, rotation: |dHg/dp_d| does
         * not depend on p (a |p_d| term has derivative of magnitude bound on
         * either side of its kink), so the box maximum is the maximum over
         * every p (R5). */
        return orc_alpha(m, ndim, x, alpha);
    }
}

static void node_coords(const orc_grid* g, int64_t idx, double* x) {
    for (int d = 0; d < g->ndim; ++d) {
        int64_t i = idx % g->n[d];
        idx /= g->n[d];
        x[d] = orc_coord(g, d, i);
    }
}

/* alpha_max[d] = max over nodes of alpha_d(x): the dissipation of the global
 * Lax-Friedrichs scheme (the listing of the rockets game names it). */
int orc_alpha_max(const orc_grid* g, const orc_method* m, double* alpha_max) {
    if (!grid_ok(g) || !m || !alpha_max) return ORC_EINVAL;
    int64_t total = orc_num_nodes(g);
    for (int d = 0; d < 4; ++d) alpha_max[d] = 0.0;
    for (int64_t idx = 0; idx < total; ++idx) {
        double x[4], alpha[4];
        node_coords(g, idx, x);
        int rc = orc_alpha(m, g->ndim, x, alpha);
        if (rc) return rc;
        for (int d = 0; d < g->ndim; ++d)
            if (alpha[d] > alpha_max[d]) alpha_max[d] = alpha[d];
    }
    return 0;
}

/* Lax-Friedrichs term (Sec. 4, Listing 5) in time-to-go form:
 *   ydot = Hg(x, (p- + p+)/2) + sum_d alpha_d (p+_d - p-_d)/2
 * with alpha_d = alpha_d(x) (local, R5), its maximum over the grid (global),
 * or the maximum over the node's box of gradients (R12), followed by the BRT
 * clamp min(0, ydot) in ORC_BRT_MIN0 mode (R7). */
int orc_term(const orc_grid* g, const orc_method* m, const double* V, double* ydot) {
    if (!grid_ok(g) || !m || !V || !ydot) return ORC_EINVAL;
    int64_t total = orc_num_nodes(g);
    int D = g->ndim;
    double* pm[4] = {0, 0, 0, 0};
    double* pp[4] = {0, 0, 0, 0};
    double amax[4];
    int rc = m->alpha_global ? orc_alpha_max(g, m, amax) : 0;
    for (int d = 0; d < D && rc == 0; ++d) {
        pm[d] = (double*)malloc(sizeof(double) * (size_t)total);
        pp[d] = (double*)malloc(sizeof(double) * (size_t)total);
        if (!pm[d] || !pp[d]) rc = ORC_ENOMEM;
        else rc = orc_upwind(g, m, V, d, pm[d], pp[d]);
    }
    for (int64_t idx = 0; idx < total && rc == 0; ++idx) {
        double x[4], pbar[4], alpha[4], hg;
        node_coords(g, idx, x);
        for (int d = 0; d < D; ++d) pbar[d] = (pm[d][idx] + pp[d][idx]) / 2.0;
        rc = orc_hamiltonian(m, D, x, pbar, &hg);
        if (rc == 0 && m->alpha_box) {
            double lo[4], hi[4];
            for (int d = 0; d < D; ++d) {
                lo[d] = pm[d][idx] < pp[d][idx] ? pm[d][idx] : pp[d][idx];
                hi[d] = pm[d][idx] < pp[d][idx] ? pp[d][idx] : pm[d][idx];
            }
            rc = orc_alpha_box(m, D, x, lo, hi, alpha);
        } else if (rc == 0) {
            rc = orc_alpha(m, D, x, alpha);
        }
        if (rc != 0) break;
        if (m->alpha_global)
            for (int d = 0; d < D; ++d) alpha[d] = amax[d];
        double y = hg;
        for (int d = 0; d < D; ++d) y += alpha[d] * (pp[d][idx] - pm[d][idx]) / 2.0;
        if (m->brt == ORC_BRT_MIN0 && y > 0.0) y = 0.0;
        ydot[idx] = y;
    }
    for (int d = 0; d < D; ++d) { free(pm[d]); free(pp[d]); }
    return rc;
}

/* CFL bound (Sec. 4): dt * max_x { sum_d |H_{p_d}| / dx_d } < 1; with the
 * global scheme, sum_d max_x |H_{p_d}| / dx_d. */
int orc_step_bound_inv(const orc_grid* g, const orc_method* m, double* out) {
    if (!grid_ok(g) || !m || !out) return ORC_EINVAL;
    if (m->alpha_global) {
        double amax[4];
        int rc = orc_alpha_max(g, m, amax);
        if (rc) return rc;
        double s = 0.0;
        for (int d = 0; d < g->ndim; ++d) s += amax[d] / orc_spacing(g, d);
        *out = s;
        return 0;
    }
    int64_t total = orc_num_nodes(g);
    double best = 0.0;
    for (int64_t idx = 0; idx < total; ++idx) {
        double x[4], alpha[4];
        node_coords(g, idx, x);
        int rc = orc_alpha(m, g->ndim, x, alpha);
        if (rc) return rc;
        double s = 0.0;
        for (int d = 0; d < g->ndim; ++d) s += alpha[d] / orc_spacing(g, d);
        if (s > best) best = s;
    }
    *out = best;
    return 0;
}

/* TVD-RK3 of Shu & Osher (Sec. 5, Listing 6):
 *   V1   = V + dt L(V)
 *   V2   = V1 + dt L(V1);     Vh = (3 V + V2) / 4
 *   V3   = Vh + dt L(Vh);     Vnew = (V + 2 V3) / 3
 * with L the Lax-Friedrichs term above; ORC_BRT_MINV then keeps
 * min(Vnew, V) (R7). */
int orc_rk3_step(const orc_grid* g, const orc_method* m, double dt, double* V) {
    if (!grid_ok(g) || !m || !V) return ORC_EINVAL;
    int64_t total = orc_num_nodes(g);
    size_t bytes = sizeof(double) * (size_t)total;
    double* V0 = (double*)malloc(bytes);
    double* U = (double*)malloc(bytes);
    double* ydot = (double*)malloc(bytes);
    if (!V0 || !U || !ydot) { free(V0); free(U); free(ydot); return ORC_ENOMEM; }
    memcpy(V0, V, bytes);
    int rc = orc_term(g, m, V0, ydot);                                  /* first substep */
    for (int64_t i = 0; i < total && rc == 0; ++i) U[i] = V0[i] + dt * ydot[i];
    if (rc == 0) rc = orc_term(g, m, U, ydot);                          /* second substep */
    for (int64_t i = 0; i < total && rc == 0; ++i) {
        double v2 = U[i] + dt * ydot[i];
        U[i] = (3.0 * V0[i] + v2) / 4.0;
    }
    if (rc == 0) rc = orc_term(g, m, U, ydot);                          /* third substep */
    for (int64_t i = 0; i < total && rc == 0; ++i) {
        double v3 = U[i] + dt * ydot[i];
        double vn = (V0[i] + 2.0 * v3) / 3.0;
        if (m->brt == ORC_BRT_MINV && V0[i] < vn) vn = V0[i];
        V[i] = vn;
    }
    free(V0); free(U); free(ydot);
    return rc;
}

/* Forward Euler and the two-stage Shu-Osher scheme (Sec. 5 names the TVD-RK
 * family; third order is the default):
 *   order 1:  Vnew = V + dt L(V)
 *   order 2:  V1 = V + dt L(V);  V2 = V1 + dt L(V1);  Vnew = (V + V2) / 2
 * ORC_BRT_MINV then keeps min(Vnew, V) (R7). */
int orc_rk_step(const orc_grid* g, const orc_method* m, double dt, double* V) {
    if (!grid_ok(g) || !m || !V) return ORC_EINVAL;
    int order = m->order == 0 ? 3 : m->order;
    if (order == 3) return orc_rk3_step(g, m, dt, V);
    if (order != 1 && order != 2) return ORC_EINVAL;
    int64_t total = orc_num_nodes(g);
    size_t bytes = sizeof(double) * (size_t)total;
    double* V0 = (double*)malloc(bytes);
    double* U = (double*)malloc(bytes);
    double* ydot = (double*)malloc(bytes);
    if (!V0 || !U || !ydot) { free(V0); free(U); free(ydot); return ORC_ENOMEM; }
    memcpy(V0, V, bytes);
    int rc = orc_term(g, m, V0, ydot);
    for (int64_t i = 0; i < total && rc == 0; ++i) U[i] = V0[i] + dt * ydot[i];
    if (rc == 0 && order == 2) {
        rc = orc_term(g, m, U, ydot);
        for (int64_t i = 0; i < total && rc == 0; ++i) {
            double v2 = U[i] + dt * ydot[i];
            U[i] = (V0[i] + v2) / 2.0;
        }
    }
    for (int64_t i = 0; i < total && rc == 0; ++i) {
        double vn = U[i];
        if (m->brt == ORC_BRT_MINV && V0[i] < vn) vn = V0[i];
        V[i] = vn;
    }
    free(V0); free(U); free(ydot);
    return rc;
}

double orc_time_eps(void) { return 100.0 * DBL_EPSILON; }

/* Time loop (Sec. 5, Listing 6), R6: per slice, step while
 * t_slice - t >= eps * t_slice, with dt clipped to land on the slice time. */
int orc_solve(const orc_grid* g, const orc_method* m, const double* V0, int n_slices,
              const double* slice_times, double* out, int64_t* out_steps, double* out_times) {
    if (!grid_ok(g) || !m || !V0 || !out || n_slices < 1 || !slice_times) return ORC_EINVAL;
    if (!(m->cfl > 0.0) || !(m->max_step > 0.0)) return ORC_EINVAL;
    for (int s = 0; s < n_slices; ++s) {
        if (!(slice_times[s] >= 0.0) || !isfinite(slice_times[s])) return ORC_EINVAL;
        if (s > 0 && slice_times[s] < slice_times[s - 1]) return ORC_EINVAL;
    }
    int64_t total = orc_num_nodes(g);
    size_t bytes = sizeof(double) * (size_t)total;
    double* V = (double*)malloc(bytes);
    if (!V) return ORC_ENOMEM;
    memcpy(V, V0, bytes);
    double t = 0.0;
    int64_t steps = 0;
    double eps = orc_time_eps();
    int rc = 0;
    for (int s = 0; s < n_slices && rc == 0; ++s) {
        double ts = slice_times[s];
        while (rc == 0 && ts > t && ts - t >= eps * ts) {
            double sbi;
            rc = orc_step_bound_inv(g, m, &sbi);
            if (rc) break;
            double step_bound = 1.0 / sbi;
            double dt = ts - t;
            if (m->max_step < dt) dt = m->max_step;
            if (m->cfl * step_bound < dt) dt = m->cfl * step_bound;
            rc = orc_rk_step(g, m, dt, V);
            t += dt;
            ++steps;
        }
        memcpy(out + (size_t)s * (size_t)total, V, bytes);
        if (out_times) out_times[s] = t;
    }
    if (out_steps) *out_steps = steps;
    free(V);
    return rc;
}
