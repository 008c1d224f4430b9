/*
 * hj_oracle.h -- plain, slow, FP64 CPU oracle for one TVD-RK3 step of the
 * Hamilton-Jacobi(-Isaacs) level-set update of LevelSetPy (arXiv 2507.11542).
 *
 * TEST INFRASTRUCTURE. Only the test-suite, the smoke check and the CPU
 * baseline of the benchmark load this code. The CUDA library never includes,
 * links or calls it, and this file includes nothing from the CUDA library.
 *
 * Conventions (identical in every function below):
 *   - A grid has ndim in 1..4 dimensions, n[d] nodes along dimension d.
 *   - Arrays hold prod(n) doubles, dimension 0 fastest ("column-major
 *     throughout the memory", Sec. 2.1): flat index
 *     i0 + n0*(i1 + n1*(i2 + n2*i3)).
 *   - Spacing: periodic dims cover [lo, hi) with n nodes, dx = (hi-lo)/n;
 *     other dims include both ends, dx = (hi-lo)/(n-1). Coordinate
 *     x_d(i) = lo_d + i*dx_d (Sec. 2.1, Listing 1).
 *   - Time is time-to-go tau >= 0. The value function obeys
 *     V_tau = Hg_LF(x, p-, p+) (or min(0, Hg_LF) for a backward reachable
 *     tube), the tau-form of the paper's v_t + H = 0 (Sec. 4) and of the
 *     variational inequality of Sec. 6.1.
 * Every function returns 0 on success and a negative code on bad arguments.
 */
#ifndef HJ_ORACLE_H
#define HJ_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int ndim;
    int64_t n[4];
    double lo[4];
    double hi[4];
    uint32_t periodic_mask; /* bit d set: dimension d is periodic */
} orc_grid;

/* upwind schemes (Sec. 3.1-3.3) */
enum { ORC_ENO1 = 1, ORC_ENO2 = 2, ORC_ENO3 = 3, ORC_WENO5 = 5 };
/* dynamics / Hamiltonians */
enum {
    ORC_DYN_DOUBLE_INTEGRATOR = 1, /* params: umax */
    ORC_DYN_AIR3D = 2,             /* params: va, vb, amax, bmax */
    ORC_DYN_DUBINS4D = 3,          /* params: wmax, accmax */
    ORC_DYN_NORM = 4,              /* params: speed c  (Hg = -c |p|) */
    ORC_DYN_ADVECT = 5,            /* params: c0..c3   (Hg = -c . p) */
    ORC_DYN_ROTATE = 6,            /* params: omega    (Hg = -p . omega(-x1, x0)) */
    ORC_DYN_ROCKETS = 7            /* params: a, g, ue_max, up_max (Sec. 6.1 rockets game) */
};
/* backward-reachable-tube rule (Sec. 6.1) */
enum { ORC_BRT_NONE = 0, ORC_BRT_MIN0 = 1, ORC_BRT_MINV = 2 };
/* extrapolated ghost cells */
enum { ORC_EXTRAP_AWAY_FROM_ZERO = 0, ORC_EXTRAP_LINEAR = 1 };

/* Settings of the numerical method (the paper's schemeData / finite_diff_data). */
typedef struct {
    int scheme;          /* ORC_ENO1 .. ORC_WENO5 */
    int dynamics;        /* ORC_DYN_* */
    double params[8];    /* dynamics parameters, see the enum above */
    int brt;             /* ORC_BRT_* */
    int extrap;          /* ORC_EXTRAP_* */
    int weno_ideal;      /* test hook: 1 = WENO5 with the ideal weights (0.1, 0.6, 0.3) */
    double cfl;          /* CFL factor (0.8) */
    double max_step;     /* upper bound on dt (use +inf for none) */
    int order;           /* TVD-RK order of a time step: 1, 2 or 3 (0 means 3) */
    int alpha_global;    /* 1: global Lax-Friedrichs, alpha_d = max over the grid of alpha_d(x) */
    int alpha_box;       /* 1: alpha_d = max of |dHg/dp_d| over the node's box of gradients (R12) */
} orc_method;

int64_t orc_num_nodes(const orc_grid* g);
double orc_spacing(const orc_grid* g, int d);
double orc_coord(const orc_grid* g, int d, int64_t i);

/* Ghost-padded copy of one grid line: out[k] holds the value at node k-3,
 * k = 0 .. n+5 (three ghost nodes per side; Sec. 2.1 boundary values). */
int orc_pad_line(const double* line, int64_t n, int periodic, int extrap, double* out);

/* Left/right derivatives p-, p+ along one padded line (Sec. 3.1-3.3). */
int orc_upwind_line(int scheme, int weno_ideal, const double* padded, int64_t n, double dx,
                    double* pm, double* pp);

/* p-, p+ along dimension `dim` for every node of the grid. */
int orc_upwind(const orc_grid* g, const orc_method* m, const double* V, int dim, double* pm, double* pp);

/* WENO5 derivative from five one-sided differences v1..v5 (Sec. 3.3). */
double orc_weno5(const double v[5], int ideal);

/* Hamiltonian Hg(x, p) = optimum over controls of p . f (or the level-set
 * Hamiltonian of the test dynamics), and per-dimension dissipation
 * alpha_d(x) = max over controls and p of |dHg/dp_d| (Sec. 4). */
int orc_hamiltonian(const orc_method* m, int ndim, const double* x, const double* p, double* hg);
int orc_alpha(const orc_method* m, int ndim, const double* x, double* alpha);
/* alpha_d = max of |dHg/dp_d| over the box of gradients p with lo[j] <= p_j <=
 * hi[j] for every j (R12), at the node with coordinates x. Where Hg has a kink
 * (|.| of a linear form) the derivative's one-sided values on both sides count
 * for a box that reaches the kink; at p = 0 the norm Hamiltonian counts c. */
int orc_alpha_box(const orc_method* m, int ndim, const double* x, const double* lo, const double* hi,
                  double* alpha);

/* ydot = [min(0, .)] (Hg(x, (p- + p+)/2) + sum_d alpha_d (p+_d - p-_d)/2) at every node. */
int orc_term(const orc_grid* g, const orc_method* m, const double* V, double* ydot);

/* max over nodes of sum_d alpha_d(x)/dx_d (Sec. 4, CFL condition). */
int orc_step_bound_inv(const orc_grid* g, const orc_method* m, double* out);

/* One TVD-RK3 step of size dt, in place (Sec. 5, Listing 6). */
int orc_rk3_step(const orc_grid* g, const orc_method* m, double dt, double* V);
/* One TVD-RK step of the method's order (Sec. 5: forward Euler, the
 * two-stage and the three-stage Shu-Osher schemes). */
int orc_rk_step(const orc_grid* g, const orc_method* m, double dt, double* V);
/* alpha_max[d] = max over the grid's nodes of alpha_d(x) (global LF). */
int orc_alpha_max(const orc_grid* g, const orc_method* m, double* alpha_max);

/* Integrate V0 from tau = 0 through each slice time; out has n_slices*prod(n)
 * doubles. out_steps (may be NULL) receives the number of RK3 steps taken,
 * out_times (may be NULL) the time reached at each slice. */
int orc_solve(const orc_grid* g, const orc_method* m, const double* V0, int n_slices,
              const double* slice_times, double* out, int64_t* out_steps, double* out_times);

/* The loop tolerance of the time integrator: stop a slice once
 * t_slice - t < ORC_TIME_EPS * t_slice (Sec. 5, Listing 6). */
double orc_time_eps(void);

#ifdef __cplusplus
}
#endif
#endif
