/*
 * hj.h -- C ABI of the GB300 (sm_103a) level-set library: one TVD-RK3 step of
 * the Hamilton-Jacobi(-Isaacs) value-function update on a dense Cartesian
 * grid, and the time loop around it, after LevelSetPy (arXiv 2507.11542).
 *
 * General rules for every entry point:
 *  - Calls return an hj_status; no C++ exception ever crosses this boundary.
 *    hj_ctx_last_error() gives a one-line description of the last failure.
 *  - Every compute call is enqueued on the context's stream. Calls that take
 *    or return host memory synchronise that stream before they return; calls
 *    on device memory only do not, unless stated.
 *  - Grid arrays hold prod(n) elements, dimension 0 fastest ("column-major",
 *    Sec. 2.1): flat index i0 + n0*(i1 + n1*(i2 + n2*i3)). Element type is
 *    given by an hj_dtype. Inputs are never modified unless stated; on an
 *    error the contents of outputs are unspecified.
 *  - Device pointers must be allocated on the context's device and aligned to
 *    the element size. The caller owns every buffer it passes in.
 *  - Time is time-to-go tau >= 0: V_tau = Hg_LF (Sec. 4), the tau-form of the
 *    paper's v_t + H = 0; a backward reachable tube clamps it at zero (Sec. 6.1).
 */
#ifndef HJ_H
#define HJ_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum hj_status {
    HJ_OK = 0,
    HJ_EINVAL = 1,      /* a malformed argument; nothing was enqueued */
    HJ_ENOMEM = 2,      /* a device or host allocation failed */
    HJ_ECUDA = 3,       /* a CUDA runtime call failed (see hj_ctx_last_error) */
    HJ_ENONFINITE = 4,  /* the initial value function or a result holds NaN/Inf */
    HJ_ETIMEOUT = 5,    /* a bounded wait ran out */
    HJ_ECANCELLED = 6,  /* a served request was cancelled */
    HJ_EBUSY = 7        /* no slot or memory for a request right now */
} hj_status;

/* Upwind derivative schemes (Sec. 3.1 first order; Sec. 3.2 ENO2/ENO3,
 * Listing 4; Sec. 3.3 WENO5). */
enum { HJ_ENO1 = 1, HJ_ENO2 = 2, HJ_ENO3 = 3, HJ_WENO5 = 5 };

/* Dynamics / Hamiltonians Hg(x, p). Reachability dynamics take the optimum of
 * p . f over bounded controls (Sec. 6.1); the level-set test Hamiltonians are
 * the equations of Sec. 3 (v_t + F . grad v = 0) and normal motion.
 *   DOUBLE_INTEGRATOR (2-D)  params {umax}:              Hg = p0 x1 - umax |p1|
 *   AIR3D (3-D)              params {va, vb, amax, bmax}: Hg = p0(-va + vb cos x2)
 *                            + p1 vb sin x2 + amax|p0 x1 - p1 x0 - p2| - bmax|p2|
 *   DUBINS4D (4-D)           params {wmax, accmax}:      Hg = x3(p0 cos x2 + p1 sin x2)
 *                            - wmax|p2| - accmax|p3|
 *   NORM (1..3-D)            params {c}:                 Hg = -c |p|
 *   ADVECT (1..3-D)          params {c0, c1, c2}:        Hg = -c . p
 *   ROTATE (2..3-D)          params {omega}:             Hg = -p . omega(-x1, x0, 0)
 *   ROCKETS (3-D)            params {a, g, ue_max, up_max}: the rockets game of
 *                            Sec. 6.1, state (x, z, theta), f = (a cos th + ue x,
 *                            a sin th + a - g + up x, up - ue), evader ue maximising,
 *                            pursuer up minimising: Hg = a p0 cos th + p1 (a sin th
 *                            + a - g) + ue_max |p0 x - p2| - up_max |p1 x + p2|
 * The dissipation alpha_d(x) is the maximum of |f_d| over the controls
 * (Sec. 4, "alpha = max |H_p|"), evaluated per node. */
enum {
    HJ_DYN_DOUBLE_INTEGRATOR = 1,
    HJ_DYN_AIR3D = 2,
    HJ_DYN_DUBINS4D = 3,
    HJ_DYN_NORM = 4,
    HJ_DYN_ADVECT = 5,
    HJ_DYN_ROTATE = 6,
    HJ_DYN_ROCKETS = 7
};

/* Backward-reachable-tube rule (Sec. 6.1): none, V_tau = min(0, Hg_LF) at each
 * RK stage, or V <- min(V_new, V_old) after each full step. */
enum { HJ_BRT_NONE = 0, HJ_BRT_MIN0 = 1, HJ_BRT_MINV = 2 };

/* Element type of grid arrays. FP32 arrays still use FP64 time, dt and CFL
 * reduction. */
enum { HJ_F32 = 1, HJ_F64 = 2 };

/* Extrapolated (non-periodic) ghost cells (Sec. 2.1 "boundary values"): the
 * outermost slope continued away from the zero level set,
 * g_m = v_0 + m |v_0 - v_1| sign(v_0), or the plain signed slope v_0 - v_1. */
enum { HJ_EXTRAP_AWAY_FROM_ZERO = 0, HJ_EXTRAP_LINEAR = 1 };

/* Lax-Friedrichs dissipation (Sec. 4, alpha_d = max |dHg/dp_d|):
 *  - HJ_ALPHA_NODE: alpha_d(x) at each node, the maximum over every p (the
 *    default); the CFL bound is max_x sum_d alpha_d(x) / dx_d.
 *  - HJ_ALPHA_GLOBAL: its maximum over the grid (global LF, the rockets
 *    listing's artificialDissipationGLF); the CFL bound is then
 *    sum_d max_x alpha_d / dx_d.
 *  - HJ_ALPHA_BOX: at each node, the maximum of |dHg/dp_d| over the box of
 *    gradients spanned by that node's one-sided derivatives, p_j in
 *    [min(p-_j, p+_j), max(p-_j, p+_j)] for every j (local in x and in p).
 *    It differs from HJ_ALPHA_NODE where |dHg/dp_d| depends on p: the norm
 *    Hamiltonian (c |p_d| / |p|) and the |.| coupling terms of air3D and the
 *    rockets game. The time step keeps the HJ_ALPHA_NODE bound, which bounds
 *    every box maximum from above, so the CFL condition holds and the step
 *    schedule is known before the first step. */
enum { HJ_ALPHA_NODE = 0, HJ_ALPHA_GLOBAL = 1, HJ_ALPHA_BOX = 2 };

/* Which stage kernel runs (hj_method.kernel): the row-tiled kernel wherever
 * the grid allows it, else the one-node-per-thread kernel (AUTO); always the
 * row kernel (ROWS: HJ_EINVAL where the grid does not allow it); always the
 * one-node-per-thread kernel (NODE). Both compute the same scheme; they
 * differ in rounding order only. */
enum { HJ_KERNEL_AUTO = 0, HJ_KERNEL_ROWS = 1, HJ_KERNEL_NODE = 2 };

/* A dense Cartesian grid (Sec. 2.1, Listing 1: createGrid(min, max, N, pdim)).
 * ndim in 1..4; n[d] >= 2 for an extrapolated dimension, >= 1 for a periodic
 * one. A periodic dimension covers [lo, hi) with spacing (hi-lo)/n, any other
 * [lo, hi] with spacing (hi-lo)/(n-1). Node coordinate lo[d] + i*dx[d]. */
typedef struct hj_grid {
    int32_t ndim;
    int64_t n[4];
    double lo[4];
    double hi[4];
    uint32_t periodic_mask; /* bit d set: dimension d is periodic */
} hj_grid;

/* The numerical method (the paper's schemeData / finite_diff_data, Listing 7). */
typedef struct hj_method {
    int32_t scheme;    /* HJ_ENO1 .. HJ_WENO5 */
    int32_t dynamics;  /* HJ_DYN_* */
    double params[8];  /* dynamics parameters, see above */
    int32_t brt;       /* HJ_BRT_* */
    int32_t extrap;    /* HJ_EXTRAP_* */
    double cfl;        /* CFL factor in (0, 1]; Sec. 4-5 (0.8 in the workloads) */
    double max_step;   /* upper bound on dt; +inf for none (Listing 6 maxStep) */
    int32_t order;     /* TVD-RK order of a time step: 1 (forward Euler), 2 or 3 (Shu-Osher); 0 means 3 */
    int32_t alpha_mode;/* HJ_ALPHA_NODE, HJ_ALPHA_GLOBAL or HJ_ALPHA_BOX */
    int32_t kernel;    /* HJ_KERNEL_AUTO (0), HJ_KERNEL_ROWS or HJ_KERNEL_NODE */
    /* Launch shape of the row kernel {ty, tz, occ, flags}, all 0 (the
     * default): picked by the context's tuner (timed once per grid, dtype,
     * dynamics and scheme, then cached). Otherwise: ty node rows per block,
     * tz planes per chunk along the last dimension (3-D and 4-D grids), occ 1
     * or 2 resident blocks per SM (2: FP32 blocks of at most 544 threads);
     * flags bit 0: blocks of n0*ty threads whose last node row also takes the
     * row ends; bit 1: tiles away from the grid's edges keep the general body
     * (the ENO schemes otherwise run them on a body compiled without ghost
     * logic). Results do not depend on the shape (bit for bit). A shape that
     * does not fit the grid is HJ_EINVAL. Used by hj_term, hj_rk3_step,
     * hj_rk3_stage and hj_solve; a problem that sets it (or kernel = NODE) is
     * solved on its own by hj_solve_batch and refused by hj_server_submit. */
    int32_t tile_override[4];
} hj_method;

/* One reachability / level-set solve (Sec. 5, Listing 6: odeCFL3(func, tspan, v0)). */
typedef struct hj_problem {
    hj_grid grid;
    hj_method method;
    int32_t dtype;             /* HJ_F32 or HJ_F64: element type of v0 and of the output */
    const void* v0;            /* initial value function, prod(n) elements */
    int32_t v0_on_device;      /* 1: v0 is device memory, 0: host memory */
    int32_t n_slices;          /* >= 1 output times */
    const double* slice_times; /* host array, non-decreasing, >= t0 */
    double t0;                 /* time of v0: 0 for a fresh solve. To resume a solve from one of
                                * its slices (a checkpoint), pass that slice as v0, the time the
                                * solve reported for it (out_times) as t0 and the later slice
                                * times: the steps that follow are those of the uninterrupted
                                * solve, bit for bit. */
} hj_problem;

typedef struct hj_stats {
    int64_t steps;           /* RK3 steps taken */
    int64_t cell_updates;    /* steps * prod(n) */
    int64_t kernel_launches; /* kernels of this library launched by the call */
    double step_bound_inv;   /* max_x sum_d alpha_d(x)/dx_d (Sec. 4 CFL bound) */
    double t_final;          /* time reached at the last slice */
    double elapsed_ms;       /* wall time of the call (served requests: submission to retirement) */
    double queued_ms;        /* served requests: submission to admission (the rest is on the
                              * device); 0 for hj_solve and hj_solve_batch */
} hj_stats;

typedef struct hj_ctx hj_ctx;

/* Context: owns device scratch (RK stage buffers, reduction words, angle
 * tables) for one device and one stream. `cuda_stream` is a cudaStream_t
 * borrowed from the caller (NULL = legacy default stream); it must outlive the
 * context. Not thread-safe: use one context per host thread.
 * Errors: HJ_EINVAL (bad device or NULL out), HJ_ECUDA, HJ_ENOMEM. */
hj_status hj_ctx_create(int32_t device, void* cuda_stream, hj_ctx** out);
/* Frees the context's device memory after synchronising its stream. NULL is a no-op. */
void hj_ctx_destroy(hj_ctx* ctx);
const char* hj_status_str(hj_status status);
/* Last error message of this context ("" if none); owned by the context. */
const char* hj_ctx_last_error(const hj_ctx* ctx);
/* The library's version string, e.g. "hj-gb300 0.1 sm_103a". */
const char* hj_version(void);

/* Rows of the hot path, one call each, on device arrays. ---------------- */

/* Upwind left/right derivatives p-, p+ along dimension `dim` at every node
 * (Sec. 3.1-3.3) from V with ghost cells per the grid (Sec. 2.1). Reads v,
 * writes pm and pp (device, prod(n) elements of `dtype` each). Asynchronous.
 * Errors: HJ_EINVAL (grid, scheme, dim, dtype or a NULL pointer), HJ_ECUDA. */
hj_status hj_upwind(hj_ctx* ctx, const hj_grid* grid, const hj_method* method, int32_t dtype,
                    const void* v, int32_t dim, void* pm, void* pp);

/* Lax-Friedrichs term ydot = Hg(x, (p- + p+)/2) + sum_d alpha_d (p+_d - p-_d)/2
 * (Sec. 4, Listing 5), clamped to min(0, ydot) when method->brt is
 * HJ_BRT_MIN0 (Sec. 6.1). Reads v, writes ydot (device). Asynchronous.
 * Errors: HJ_EINVAL, HJ_ECUDA. */
hj_status hj_term(hj_ctx* ctx, const hj_grid* grid, const hj_method* method, int32_t dtype,
                  const void* v, void* ydot);

/* CFL bound max over nodes of sum_d alpha_d(x)/dx_d in FP64 (Sec. 4), written
 * to *out (host). For every supported dynamics alpha depends on x only, so
 * the value is the same at every step. Synchronises the stream.
 * Errors: HJ_EINVAL, HJ_ECUDA. */
hj_status hj_step_bound(hj_ctx* ctx, const hj_grid* grid, const hj_method* method, double* out);

/* One TVD-RK step of size dt (Sec. 5, Listing 6) of the method's order
 * (three stages by default), in place on the device array v: one fused stage
 * kernel per stage (upwind + Hamiltonian + dissipation + BRT rule + stage
 * combination). Stage buffers come from the context.
 * Asynchronous. Errors: HJ_EINVAL (dt < 0 or not finite, ...), HJ_ENOMEM, HJ_ECUDA. */
hj_status hj_rk3_step(hj_ctx* ctx, const hj_grid* grid, const hj_method* method, int32_t dtype,
                      void* v, double dt);

/* One fused stage of the TVD-RK3 step (Sec. 5, Listing 6), with
 * w = u + dt * L(u) and L the Lax-Friedrichs term above:
 *   stage 1: out = w
 *   stage 2: out = 3/4 vn + 1/4 w
 *   stage 3: out = 1/3 vn + 2/3 w, then min(out, vn) when method->brt is HJ_BRT_MINV.
 * u, vn, out are device arrays; vn is unused (may be NULL) in stage 1. out must
 * not alias u; it may alias vn. Asynchronous.
 * Errors: HJ_EINVAL (stage not 1..3, aliasing, ...), HJ_ECUDA. */
hj_status hj_rk3_stage(hj_ctx* ctx, const hj_grid* grid, const hj_method* method, int32_t dtype, int32_t stage,
                       const void* u, const void* vn, void* out, double dt);

/* Whole solve (Sec. 5, Listing 6): V(tau = 0) = v0, then for each slice time
 * t_s, RK3 steps with dt = min(t_s - t, max_step, cfl / stepBoundInv) while
 * t_s - t >= 100 * DBL_EPSILON * t_s; V at each slice goes to
 * out_slices + s * prod(n) (device memory if out_on_device, else host).
 * out_times (host, n_slices doubles, may be NULL) receives the time reached at
 * each slice; stats may be NULL. Synchronises the stream before returning.
 * Errors: HJ_EINVAL, HJ_ENOMEM, HJ_ENONFINITE (v0 or the result holds
 * NaN/Inf), HJ_ECUDA. */
hj_status hj_solve(hj_ctx* ctx, const hj_problem* problem, void* out_slices, int32_t out_on_device,
                   double* out_times, hj_stats* stats);

/* Many independent solves at once (the batched form of hj_solve). Problem i
 * writes its slices to out_slices[i] (device memory if out_on_device[i], else
 * host memory), its slice times to out_times[i] (may be NULL, or out_times
 * itself NULL) and its statistics to stats[i] (stats may be NULL).
 * Instances (any scheme) of the row kernel's (dimension, dynamics) pairs
 * with n0 < 1024 (FP32) or n0 < 512 (FP64), the three-stage scheme and
 * per-node dissipation advance together: one launch per RK stage and
 * (element type, dimension, dynamics, scheme) group covers every tile of
 * every active instance, a small kernel advances each instance's own dt and
 * slice cursor, and blocks of steps replay as CUDA graphs. Other problems are
 * solved one by one with hj_solve. Every problem is validated before any work;
 * results equal those of hj_solve on each problem alone (same arithmetic per
 * node). elapsed_ms and kernel_launches in stats are those of the whole call.
 * The first batch with a new (element type, dimension, dynamics, scheme) group times a
 * few launch shapes. Synchronises the stream.
 * Errors: HJ_EINVAL (names the problem index), HJ_ENOMEM, HJ_ENONFINITE, HJ_ECUDA. */
hj_status hj_solve_batch(hj_ctx* ctx, int32_t n, const hj_problem* problems, void* const* out_slices,
                         const int32_t* out_on_device, double* const* out_times, hj_stats* stats);

/* Serving: a continuous-batching request loop (Sec. 6 reachability solves as
 * requests). A server owns a private stream, a private context and an HBM
 * arena of hbm_budget bytes (allocated at creation), and one engine thread.
 * Requests queue in arrival order; each engine tick admits queued requests
 * while a slot (at most max_slots) is free and the request's footprint (its
 * three grid arrays, angle tables, slice bookkeeping and, for host outputs, a
 * device copy of its slices) fits the arena, then advances every admitted
 * request by a block of RK3 steps in batched launches (as hj_solve_batch),
 * and retires requests whose steps are done. Grids stay on the device from
 * admission to retirement; requests arriving meanwhile join at the next tick.
 * Each result equals hj_solve on the same problem alone (same arithmetic per
 * node). All functions are thread-safe except destroy, which no other call
 * may overlap. */
typedef struct hj_server hj_server;

typedef struct hj_server_info {
    int64_t queued;          /* requests waiting for admission */
    int64_t running;         /* requests on the device */
    int64_t completed;       /* requests finished (any status) */
    int64_t bytes_in_use;    /* arena bytes held by admitted requests */
    int64_t budget;          /* arena size */
    int64_t kernel_launches; /* kernels launched by the engine so far */
} hj_server_info;

/* Creates a server on ctx's device (ctx itself is not used afterwards).
 * Errors: HJ_EINVAL (max_slots < 1, budget < 4096 bytes), HJ_ENOMEM, HJ_ECUDA. */
hj_status hj_server_create(hj_ctx* ctx, size_t hbm_budget, int32_t max_slots, hj_server** out);
/* Queues a request; never waits for the GPU. The problem (including its slice
 * times) is copied; v0 and out_slices (n_slices x prod(n) elements, device
 * memory if out_on_device) and out_times (host, n_slices doubles, may be
 * NULL) must stay valid until hj_server_wait returns for the ticket.
 * Errors: HJ_EINVAL (malformed, or not served by the batched row kernel:
 * the three-stage scheme, per-node dissipation, the
 * dimension/dynamics pairs of hj_solve_batch), HJ_ENOMEM (footprint
 * larger than the whole budget), HJ_ECANCELLED (server stopping). */
hj_status hj_server_submit(hj_server* srv, const hj_problem* problem, void* out_slices, int32_t out_on_device,
                           double* out_times, uint64_t* ticket);
/* Waits up to timeout_ms (< 0: no limit) for a request. On completion returns
 * its status (HJ_OK, HJ_ENONFINITE, HJ_ECANCELLED, ...) and forgets the
 * ticket; stats->elapsed_ms is the latency from submission to retirement.
 * Errors: HJ_ETIMEOUT (still running; the ticket stays valid), HJ_EINVAL
 * (unknown ticket). */
hj_status hj_server_wait(hj_server* srv, uint64_t ticket, int32_t timeout_ms, hj_stats* stats);
/* Cancels a queued request at once, or a running one at the next tick
 * boundary (its outputs are then unspecified); wait then returns
 * HJ_ECANCELLED. Errors: HJ_EINVAL (unknown or finished ticket). */
hj_status hj_server_cancel(hj_server* srv, uint64_t ticket);
/* Counters of the server; returns the server's fatal status (HJ_OK unless a
 * CUDA failure stopped the engine). */
hj_status hj_server_counters(hj_server* srv, hj_server_info* info);
/* Stops the engine (requests not finished are cancelled), frees the arena. */
void hj_server_destroy(hj_server* srv);

/* No-allocation variant of hj_rk3_step. -------------------------------- */

/* Capacity of the fixed scratch used by hj_rk3_step_static. */
#define HJ_STATIC_MAX_NODES (1 << 20)  /* grid nodes per call (101^3 fits) */
#define HJ_STATIC_MAX_ANGLES 4096      /* nodes along dimension 2 for air3D / Dubins4D */

/* The paper has no counterpart of this call; it exists for callers that may
 * not allocate device memory while they run -- for example a real-time
 * control loop (a safety filter that re-solves its reachable set every cycle)
 * where allocation after start-up is forbidden because cudaMalloc can block
 * and fragment memory, or a host application that owns the GPU's memory pool
 * and admits no other allocator. It needs no hj_ctx.
 *
 * Same arithmetic as hj_rk3_step: one TVD-RK3 step of size dt, in place on the
 * caller's device array v (prod(n) elements of dtype, on `device`), enqueued
 * on `cuda_stream` (a cudaStream_t; NULL = legacy default stream). The two
 * stage buffers and the heading-angle tables live in one fixed __device__
 * array of 2 * HJ_STATIC_MAX_NODES * 8 bytes plus 96 KiB (about 16 MiB) that
 * every GPU which loads this library holds until the process exits. The call
 * performs no cudaMalloc/cudaFree and calls no allocating routine.
 *  - The first call on a device looks up that array's device address
 *    (cudaGetSymbolAddress); make that first call before any stream capture.
 *  - All calls share the one array, and nothing in it needs to start at zero:
 *    each call writes every element it later reads. Calls whose work overlaps
 *    on the GPU (e.g. on two streams at once) race on it; serialise them.
 *  - Asynchronous: returns after enqueueing.
 * Errors: HJ_EINVAL for a malformed argument, for prod(n) > HJ_STATIC_MAX_NODES,
 * for more than HJ_STATIC_MAX_ANGLES nodes along dimension 2 with air3D,
 * Dubins4D or rockets dynamics, or for a method other than the three-stage
 * scheme with per-node dissipation (nothing is enqueued); HJ_ECUDA if a CUDA
 * call fails. */
hj_status hj_rk3_step_static(void* cuda_stream, int32_t device, const hj_grid* grid, const hj_method* method,
                             int32_t dtype, void* v, double dt);

/* Initial surfaces on the device (Sec. 2.2: implicit surfaces built on the
 * grid container, geometric primitives and Boolean operations; the ellipsoid
 * listing of that section). ------------------------------------------------ */

enum { HJ_SHAPE_SPHERE = 1, HJ_SHAPE_ELLIPSOID = 2, HJ_SHAPE_RECTANGLE = 3 };
enum { HJ_SHAPE_UNION = 1, HJ_SHAPE_INTERSECT = 2, HJ_SHAPE_SUBTRACT = 3 };
#define HJ_MAX_SHAPES 32

/* One primitive, over the dimensions in dims_mask (bit d); the others are
 * ignored, which turns a sphere into a cylinder and a rectangle into a slab.
 * With s_d = x_d - center[d]:
 *   SPHERE     sqrt(sum_d s_d^2) - radius           (signed distance)
 *   ELLIPSOID  sum_d axes[d] s_d^2 - radius         (the section's listing: an
 *              implicit quadratic, not a distance; axes[d] > 0)
 *   RECTANGLE  max_d (|s_d| - axes[d])              (axes = half-widths; the
 *              signed distance inside and along the face normals)
 * op says how the shape joins the shapes before it (ignored for the first):
 *   UNION min(v, s), INTERSECT max(v, s), SUBTRACT max(v, -s). */
typedef struct hj_shape {
    int32_t kind;       /* HJ_SHAPE_SPHERE .. HJ_SHAPE_RECTANGLE */
    int32_t op;         /* HJ_SHAPE_UNION .. HJ_SHAPE_SUBTRACT */
    uint32_t dims_mask; /* nonzero, within the grid's dimensions */
    double center[4];
    double axes[4];
    double radius;
} hj_shape;

/* V(x) of n_shapes (1..HJ_MAX_SHAPES) primitives combined in order, at every
 * grid node, into out (prod(n) elements of dtype; device memory if
 * out_on_device, else host memory, which makes the call synchronous). FP64
 * output is computed in FP64, FP32 output in FP32. Asynchronous for device
 * output. Errors: HJ_EINVAL (grid, dtype, a shape's kind, op, mask or
 * parameters, n_shapes, NULL pointers), HJ_ENOMEM, HJ_ECUDA. */
hj_status hj_implicit_surface(hj_ctx* ctx, const hj_grid* grid, int32_t n_shapes, const hj_shape* shapes,
                              int32_t dtype, void* out, int32_t out_on_device);

#ifdef __cplusplus
}
#endif
#endif /* HJ_H */
