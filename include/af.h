/*
 * af.h -- C ABI of libaf: one SSP-RK3 step of the positivity-preserving
 * Active Flux (AF) scheme for 2D ideal MHD with the Godunov-Powell source
 * term (J. Duan, P. Chandrashekar, C. Klingenberg, arXiv:2506.04857), in FP64
 * on an NVIDIA GB300 (sm_103a).
 *
 * Problem (Sec. 1, eq. 2d_mhd_gp): U_t + F1(U)_x + F2(U)_y = -(div B) Psi(U),
 * U = (rho, rho v1, rho v2, rho v3, B1, B2, B3, E), Psi = (0, B, v, v.B),
 * perfect gas p = (gamma-1)(E - |rho v|^2/(2 rho) - |B|^2/2), on a uniform
 * Cartesian grid of nx x ny cells.
 *
 * Degrees of freedom (Sec. 2, Fig. 1), in four classes, each stored as a
 * contiguous FP64 array [8][nyp][nxp] (component, row y, column x; x fastest):
 *   AF_CLASS_AVG    cell averages          at cell (i,j)               nx x ny
 *   AF_CLASS_XFACE  x-face point values    at (x0 + i dx, y_j)         nxf x ny
 *   AF_CLASS_YFACE  y-face point values    at (x_i, y0 + j dy)         nx x nyf
 *   AF_CLASS_CORNER corner point values    at (x0 + i dx, y0 + j dy)   nxf x nyf
 * with nxf = nx, nyf = ny for periodic boundaries and nx+1, ny+1 for outflow
 * (boundary point values are degrees of freedom).  af_sizes returns nxp, nyp.
 *
 * Conventions.
 *   - Return value: AF_OK (0) or a negative AF_E* code; af_last_error gives a
 *     message.  Nothing aborts the process.
 *   - The context owns its device memory (three state buffers and the stage
 *     work arrays, about 260 doubles per cell).  The caller owns every array
 *     passed in.
 *   - on_device = 1: pointers are device pointers on the context's device,
 *     used in stream order on the context's stream (af_set_stream); calls
 *     return before the GPU work ends.  on_device = 0: host pointers; the call
 *     synchronises the stream before it returns.
 *   - Device-side faults of the scheme (a degree of freedom left outside the
 *     admissible set after every safeguard, a non-finite time step) latch a
 *     device error word that the next af_status call reports as AF_ENONPHYS.
 *   - A context is not thread-safe: calls on one context must not overlap in
 *     time from several host threads.  Distinct contexts are independent (their
 *     device work is ordered only by their streams).
 */
#ifndef AF_H
#define AF_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct af_ctx af_ctx;

enum { AF_BC_PERIODIC = 0, AF_BC_OUTFLOW = 1 };
enum {
  AF_OK = 0,
  AF_EINVAL = -1,     /* bad argument */
  AF_ECUDA = -2,      /* CUDA runtime error */
  AF_ENOMEM = -3,     /* device allocation failed */
  AF_ENONPHYS = -4,   /* a DoF left the admissible set G, or dt was not finite */
  AF_EBOUNDS = -5,    /* internal capacity exceeded (round-off repair list) */
  AF_ETIMEOUT = -6    /* reserved */
};
enum { AF_CLASS_AVG = 0, AF_CLASS_XFACE = 1, AF_CLASS_YFACE = 2, AF_CLASS_CORNER = 3 };

/* Counters reported by af_status (cumulative since af_create or the last
 * af_status call with reset = 1). */
enum {
  AF_STAT_SRC_LIMITED = 0,   /* cells with theta_ij < 1 (Sec. 3.2 step (1)) */
  AF_STAT_LAMBDA_LT1,        /* cells with some Lambda_I < 1 (step (2)) */
  AF_STAT_FACE_THETA_LT1,    /* faces with theta < 1 (step (3)) */
  AF_STAT_SENSOR_LT099,      /* faces with theta^s < 0.99 (Sec. 3.4) */
  AF_STAT_NEWTON_SOLVES,     /* vertex cubics solved by Newton (step (2)) */
  AF_STAT_NEWTON_MAXIT,      /* largest Newton iteration count (a maximum, not a sum) */
  AF_STAT_SHRINK,            /* round-off shrink events (Remark 4.1) */
  AF_STAT_POINT_LIMITED,     /* point values with theta* < 1 or theta** < 1 (Sec. 3.3) */
  AF_STAT_CFL_VIOLATIONS,    /* cells violating the LLF CFL condition of Lemma 3.1 */
  AF_STAT_CENTER_LIMITED,    /* cell-centre values modified (Remark 3.2) */
  AF_STAT_NONADMISSIBLE,     /* DoFs left outside G after every safeguard */
  AF_STAT_CELL_SHRINK,       /* the cell-average part of AF_STAT_SHRINK (Remark 4.1) */
  AF_NSTAT
};

typedef struct af_params {
  double cfl;        /* dt = cfl / (max varrho_1/dx + max varrho_2/dy), maxima over all four DoF
                        classes of U^n (Sec. 2.3 eq. cf; the paper prints no formula).  Default 0.2. */
  double kappa;      /* shock-sensor strength kappa (Sec. 3.4); 0 gives theta^s = 1.  Default 0. */
  int pp_on;         /* positivity-preserving limiters of Sec. 3.2-3.3 and Remark 4.1.  Default 1. */
  int src_cell_on;   /* Godunov-Powell source in the cell-average update (eq. semi_av_src).  Default 1. */
  int src_point_on;  /* Godunov-Powell source in the point-value update (Sec. 2.3).  Default 1. */
  int src_point_upwind; /* Example 4.2 variant: the derivative of B_l in the divergence of the
                        point-value source is taken one-sided along each FVS line, upwind for v_l
                        of the point (D^+ B_l for v_l > 0, D^- B_l for v_l < 0, the central
                        (D^+ + D^-) / 2 for v_l = 0) instead of central.  The paper reports it
                        unstable; for study only.  Default 0.  Ignored by the 1D scheme (no
                        point source); the discrete adjoint rejects it (AF_EINVAL). */
} af_params;

/* Create a context for an nx x ny grid (nx, ny >= 4, ny < 262140 and
 * (nx+1)(ny+1) < 2^28, else AF_EINVAL; larger grids would not fit in device
 * memory in any case), ratio of specific heats
 * gamma > 1, boundary condition bc (AF_BC_PERIODIC or AF_BC_OUTFLOW; outflow
 * mirrors the DoFs across the boundary, the paper names the condition only).
 * Uses the current CUDA device.  The domain defaults to [0,1]^2 and the
 * parameters to the defaults above.  The state is zero until af_set_state. */
int af_create(int nx, int ny, double gamma, int bc, af_ctx **out);

/* Domain [x0,x1] x [y0,y1] (x1 > x0, y1 > y0); sets dx = (x1-x0)/nx, dy = (y1-y0)/ny. */
int af_set_domain(af_ctx *ctx, double x0, double x1, double y0, double y1);

/* Boundary kind of each side of an outflow grid (side[0] left, [1] right,
 * [2] bottom, [3] top), for problems such as the jets of Example 4.8 (the
 * paper names the conditions only; readings):
 *   AF_SIDE_OUTFLOW    ghost DoFs mirror the interior across the side (default);
 *   AF_SIDE_REFLECTIVE mirror, with the normal components of the momentum and
 *                      of B negated (a symmetry plane);
 *   AF_SIDE_INFLOW     bottom/top only: ghost DoFs whose mirror point has
 *                      inflow_lo < x < inflow_hi take the conserved state
 *                      inflow_U[8]; outflow elsewhere on that side.
 * A ghost index is resolved along x first, then along y.  Periodic grids
 * return AF_EINVAL.  The discrete adjoint (af_rhs_vjp, af_adjoint_step)
 * rejects grids with reflective or inflow sides. */
enum { AF_SIDE_OUTFLOW = 0, AF_SIDE_REFLECTIVE = 1, AF_SIDE_INFLOW = 2 };
int af_set_boundary(af_ctx *ctx, const int side[4], double inflow_lo, double inflow_hi, const double inflow_U[8]);

int af_set_params(af_ctx *ctx, const af_params *p);
int af_get_params(const af_ctx *ctx, af_params *p);

/* The CUDA stream (a cudaStream_t passed as void*; NULL = the legacy default
 * stream) on which all further work of this context is enqueued. */
int af_set_stream(af_ctx *ctx, void *stream);

/* Extents of DoF class cls (AF_CLASS_*): *nxp columns, *nyp rows. */
int af_sizes(const af_ctx *ctx, int cls, int *nxp, int *nyp);

/* Copy the state U^n in (U[cls] is a [8][nyp][nxp] array of conserved
 * variables).  The state is not validated here; af_status reports a
 * non-admissible state once a step has run on it. */
int af_set_state(af_ctx *ctx, const double *const U[4], int on_device);

/* Copy the current state U^n out (same layout). */
int af_get_state(af_ctx *ctx, double *const U[4], int on_device);

/* The semi-discrete right-hand side L(U^n) of Sec. 2.2 and 2.3 for all four
 * classes (Simpson fluxes, Powell source on the 3x3 Simpson nodes, LLF flux
 * vector splitting with the central divergence, cell-centre values limited
 * as in Remark 3.2), without the shock sensor or the PP limiters, which
 * depend on dt.  dUdt has the state layout. */
int af_rhs(af_ctx *ctx, double *const dUdt[4], int on_device);

/* The shock-sensor blending coefficients theta^s of Sec. 3.4 for the current
 * state: theta_x at the x-faces, an [ny][nxf] array (class AF_CLASS_XFACE
 * extents), theta_y at the y-faces, an [nyf][nx] array (AF_CLASS_YFACE
 * extents).  With kappa = 0 every coefficient is 1. */
int af_sensor(af_ctx *ctx, double *theta_x, double *theta_y, int on_device);

/* dt = cfl / (max varrho_1/dx + max varrho_2/dy) over the DoFs of U^n.  The
 * value stays on the device for af_stage; it is also written to *dt_out
 * (host or device pointer) when dt_out is not NULL. */
int af_dt(af_ctx *ctx, double *dt_out, int on_device);

/* One stage s in {0,1,2} of the SSP-RK3 scheme, written as convex
 * combinations of limited forward-Euler stages (Sec. 3.1):
 *   U1 = FE(U^n), U2 = 3/4 U^n + 1/4 FE(U1), U^{n+1} = 1/3 U^n + 2/3 FE(U2),
 * with FE the forward-Euler update of Sec. 2 limited by Sec. 3.2-3.4.  Stages
 * must be called in order 0, 1, 2; stage 2 makes U^{n+1} the current state.
 * dt: the time step (host or device pointer); NULL uses the value of the last
 * af_dt / af_step. */
int af_stage(af_ctx *ctx, int s, const double *dt, int on_device);

/* Copy out the result of the most recent stage: U1 after stage 0, U2 after
 * stage 1, U^{n+1} after stage 2 (same layout as the state). */
int af_get_stage(af_ctx *ctx, double *const U[4], int on_device);

/* Run diagnostics of the current state (not in the paper; for monitoring the
 * positivity that Sec. 3 preserves), written to out[9] (host or device
 * pointer): out[c] = min rho and out[4+c] = min p over the DoFs of class c
 * (0 averages, 1 x-faces, 2 y-faces, 3 corners), p = (gamma-1)(E - |rho v|^2
 * /(2 rho) - |B|^2/2); out[8] = dx dy sum of the cell-average densities (the
 * total mass).  A NaN anywhere in a class makes its minima NaN.  The sums and
 * minima are formed in a fixed order (deterministic).  With on_device = 0 the
 * call synchronises the stream.  Allocates a small workspace on first use. */
int af_diagnostics(af_ctx *ctx, double *out, int on_device);

/* The two discrete divergence measures of Example 4.4 for the current state,
 * written to out[0], out[1] (host or device pointer):
 *   out[0] = sum over cells and the 3x3 nodes of eq. (semi_av_src) of
 *            |(div B)^{l,m}| w_l w_m dx dy (centre node: the limited centre
 *            value, as in a stage);
 *   out[1] = sum over cells of |Simpson edge integral of B.n| =
 *            |dy/6 ([R] - [L]) + dx/6 ([T] - [B])|, [.] = corner + 4 face
 *            centre + corner of B1 (right, left faces) or B2 (top, bottom).
 * Reading: the text defines the second measure as the edge integral of B.n;
 * the printed sum carries dx dy instead of the edge lengths.  The sums are
 * formed in a fixed order (deterministic).  With on_device = 0 the call
 * synchronises the stream.  Allocates a small workspace on first use. */
int af_divb(af_ctx *ctx, double *out, int on_device);

/* Discrete adjoint (not in the paper; differentiates its scheme).
 * af_rhs_vjp: out = (dL/dU)^T v for the semi-discrete operator of af_rhs at
 * the current state (alpha = max varrho on each FVS line differentiated
 * through the point that attains it).  v and out have the state layout. */
int af_rhs_vjp(af_ctx *ctx, const double *const v[4], double *const out[4], int on_device);

/* lam_out = (dU^{n+1}/dU^n)^T lam_in for one SSP-RK3 step from the current
 * state U^n with the recorded time step *dt (host or device pointer, held
 * fixed: dt is not differentiated; a host dt must be > 0, a device dt is
 * taken as recorded).  Stages 0 and 1 are recomputed from U^n, and stage 2
 * too unless flags has AF_ADJ_RECORDED.  The transpose is that of the branch
 * on which the shock sensor is off (kappa = 0, else AF_EINVAL) and every
 * positivity limiter is inactive, where a limited forward-Euler stage equals
 * U + dt L(U).  If a limiter acts during the recomputed stages the call
 * returns AF_EINVAL (lam_out then holds no gradient).  AF_ADJ_RECORDED: the
 * caller has established, from the counters of the forward step (af_status),
 * that no limiter acted in its last stage, which is then not recomputed.
 * AF_ADJ_DT: dt is not held fixed but differentiated as the function of U^n
 * that af_step forms, dt = cfl / (M1/dx + M2/dy) with M_l = max varrho_l:
 * lam_out gains mu d(dt)/dU^n, mu = lam_in . dU^{n+1}/d(dt) (from the stage
 * increments), at the DoFs attaining M1 and M2 (a subgradient where the
 * maximum is not unique: the first such DoF in class, then row-major order).
 * It implies the recomputation of the last stage.  Meaningful only when the
 * forward step took its dt from U^n.
 * lam_out may alias lam_in.  The state is not advanced.  The call
 * synchronises the stream once, at its end. */
enum { AF_ADJ_RECORDED = 1, AF_ADJ_DT = 2 };
int af_adjoint_step(af_ctx *ctx, const double *dt, int dt_on_device, const double *const lam_in[4],
                    double *const lam_out[4], int on_device, int flags);

/* af_adjoint_step with the stage states of the forward step supplied instead
 * of recomputed (same result, bit for bit).  U1 and U2 (and U3 = U^{n+1},
 * needed only with AF_ADJ_DT, else may be NULL) are what af_get_stage returned
 * after stages 0, 1 (and 2) of the forward step from the current state U^n
 * with this dt; they have the state layout and, like lam_in and lam_out, are
 * device pointers when on_device = 1, host arrays otherwise.  Only the point
 * data of U^n, U1 and U2 are formed, so the call cannot tell whether a
 * positivity limiter acted in the forward stages: the caller establishes it
 * from the forward step's counters (af_status).  The cell-centre limiter,
 * which acts in the point data, is checked (AF_EINVAL).  kappa must be 0.
 * The state is not advanced.  The call synchronises the stream once, at its
 * end.  Not in the paper: it saves the adjoint two forward stages per step
 * when the stage states are kept, e.g. during a checkpoint recomputation. */
int af_adjoint_step_stages(af_ctx *ctx, const double *dt, int dt_on_device, const double *const U1[4],
                           const double *const U2[4], const double *const U3[4], const double *const lam_in[4],
                           double *const lam_out[4], int on_device, int flags);

/* ---------------------------------------------------------------------------
 * The limited branch: limiter coefficients recorded, frozen and transposed.
 * Along a recorded branch the limiters of Sec. 3 are blends with fixed
 * coefficients: theta^s per face and theta^s_ij per cell (Sec. 3.4), theta_ij
 * (Sec. 3.2 step 1), the face theta of step (3) after the Remark 4.1 shrink,
 * and the scaling-limiter theta*, theta** of every point value (Sec. 3.3,
 * after Remark 4.1; 0 for the fall-back to the LLF state) and of every cell
 * centre (Remark 3.2).  With them held at the values a forward stage took,
 * the stage is a smooth function of its input (up to the maxima inside the
 * alpha of the LLF fluxes and of the FVS lines, differentiated along the
 * branch they take), and its transpose is what the discrete adjoint of a
 * limited run needs.  Not in the paper.
 *
 * Coefficient block of one stage: AF_NCOEF arrays [nyp][nxp] (nxp, nyp: the
 * index grid, nx or nx + 1 for outflow), at the index of the face, cell or
 * point they belong to: 0 theta^s of x-faces, 1 of y-faces, 2 face theta of
 * x-faces, 3 of y-faces, 4 theta_ij, 5-6 theta*, theta** of the cell centres,
 * 7-8 of the x-face values, 9-10 of the y-face values, 11-12 of the corners.
 * A buffer for a step holds three blocks (stage s at s * af_coeff_len).  The
 * buffers are the caller's device memory, on the context's device. */
#define AF_NCOEF 13
/* *n = doubles in one stage block. */
int af_coeff_len(const af_ctx *ctx, long long *n);
/* buf (device, 3 blocks) or NULL: while set, every af_stage / af_step writes
 * its coefficients into the block of its stage index.  Not while frozen. */
int af_record_coeffs(af_ctx *ctx, double *buf);
/* buf (device, 3 blocks) or NULL: while set, every af_stage / af_step uses the
 * coefficients of its stage index from buf instead of forming them (the
 * frozen branch: no limiter test, no shrink; AF_EINVAL with the PP limiters
 * off).  Not while recording. */
int af_freeze_coeffs(af_ctx *ctx, const double *buf);
/* out = (d FE(U)/dU)^T lam for the forward-Euler stage FE of the current
 * state U with time step dt (host or device pointer) along the branch frozen
 * at coeffs (one stage block, device): lam and out have the state layout
 * (device pointers when on_device = 1, host arrays otherwise; they must not
 * alias).  Periodic or outflow sides, central point source.  The state is not
 * advanced. */
int af_stage_vjp(af_ctx *ctx, const double *dt, int dt_on_device, const double *coeffs, const double *const lam[4],
                 double *const out[4], int on_device);
/* af_adjoint_step_stages along the recorded branch: lam_out = (dU^{n+1}/dU^n)^T
 * lam_in for the step from the current state U^n whose stage states were U1,
 * U2 (and U3 = U^{n+1} with AF_ADJ_DT) and whose coefficients af_record_coeffs
 * wrote into coeffs (three blocks, device).  Any kappa; the limiters may have
 * acted.  AF_ADJ_DT as for af_adjoint_step, with the coefficients held fixed.
 * The state is not advanced.  The call synchronises the stream at its end. */
int af_adjoint_step_frozen(af_ctx *ctx, const double *dt, int dt_on_device, const double *const U1[4],
                           const double *const U2[4], const double *const U3[4], const double *coeffs,
                           const double *const lam_in[4], double *const lam_out[4], int on_device, int flags);

/* af_dt followed by the three stages.  *dt_used (host or device, may be NULL)
 * receives the step's dt. */
int af_step(af_ctx *ctx, double *dt_used, int on_device);

/* One SSP-RK3 step (as af_step) of a HOST-resident state, pipelined for
 * streams of independent states.  in[cls] and out[cls] are host arrays in the
 * state layout; in pinned memory (cudaHostAlloc / cudaHostRegister) the copies
 * run asynchronously, in pageable memory they serialise.  The call enqueues
 * the copy of `in` to the device (a context-owned copy stream), the step on
 * the context's stream with dt taken from `in`, and the copy of the result to
 * `out` (a second copy stream), and returns without waiting: the input copy
 * of the next call and the output copy of the previous one overlap this
 * step.  Two input and two output staging states (4 state buffers) are
 * allocated on first use.  `out` is complete, and `in` may be reused, only
 * after af_sync, af_status or af_destroy.  An input that overlaps the output
 * of one of the three previous calls (chained steps) is copied after that
 * output has arrived.  The resident state of af_set_state / af_get_state is
 * not changed; the limiter counters and the device error word accumulate as
 * for af_step.  Not to be called in the middle of a step (af_stage). */
int af_step_host(af_ctx *ctx, const double *const in[4], double *const out[4]);

/* Wait for all work of the context: its stream and its copy streams. */
int af_sync(af_ctx *ctx);

/* Synchronise the stream (and the copy streams of af_step_host), copy the
 * AF_NSTAT counters into counters (may be NULL) and report the device error
 * word: AF_ENONPHYS for a non-admissible DoF or a non-finite dt, AF_EBOUNDS
 * for an overflowed repair list.  reset = 1 clears counters and error word
 * afterwards. */
int af_status(af_ctx *ctx, long long *counters, int reset);

/* Kernels of one stage, in the order af_timing reports them. */
enum { AF_K_POINTDATA = 0, AF_K_DT, AF_K_POINTS, AF_K_FACES, AF_K_CELLS, AF_K_FINAL, AF_K_REPAIR,
       AF_K_POINTS_SLOW, AF_K_CELLS_SLOW, AF_NKERNEL };

/* Per-kernel device timing for measurement tools.  enable = 1 clears the
 * record and starts bracketing every kernel launch of this context with a
 * pair of CUDA events on its stream; enable = 0 stops, synchronises the
 * stream and writes, per kernel (AF_K_* order), the summed device time in
 * milliseconds to ms[AF_NKERNEL] and the number of launches to
 * launches[AF_NKERNEL] (either may be NULL). */
int af_timing(af_ctx *ctx, int enable, double *ms, long long *launches);

/* Message of the last error on this context ("" when none). */
const char *af_last_error(const af_ctx *ctx);

/* Free the context and its device memory (NULL is ignored). */
void af_destroy(af_ctx *ctx);

/* Diagnostic: n results of the FP64 helpers the kernels use, on device
 * arrays, in stream order: op 0 out = 1/x, op 1 out = x/y, op 2 out = sqrt(x),
 * op 3 out = x + y and op 4 out = x * y on the integer pipes (bitwise the IEEE
 * round-to-nearest sum and product), and the integer-pipe compares as 1.0 / 0.0:
 * op 5 x >= y, op 6 x >= y and op 7 x > y for a constant y > 0, op 8 x >= 0;
 * and the FP32 certificates as 1.0 (certified) / 0.0 (undecided): op 9, x = n
 * states of 8 conserved values, y[0] = c: q = rho E - |m|^2/2 - rho (|B|^2/2 + c)
 * >= 0; op 10, x = n cases of 40 values (Lim1, then the face values G of the
 * left, right, lower and upper faces, 8 each), y = (dt/dx, dt/dy, c): the Sec. 3.2
 * box certificate.  n is the number of results: out holds n doubles, x holds n
 * (8n for op 9, 40n for op 10), y holds n for ops 1 and 3..7, 1 for op 9 and 3
 * for op 10 and is not read by ops 0, 2 and 8.  The sizes cannot be checked here:
 * buffers shorter than that are read or written out of bounds.  Used by the tests
 * to bound the helpers' error against the CUDA operators and to check the
 * certificates.  AF_EINVAL for an op outside 0..10, n < 0 or a null x or out (or y
 * where it is read). */
int af_math_check(int op, const double *x, const double *y, double *out, long long n, void *stream);

/* ---- Batched ensembles (not in the paper: many independent runs at once) ----
 * A batch holds nruns independent runs of possibly different sizes, boundary
 * conditions, gamma, domains and parameters.  Every pass of a stage is one
 * persistent kernel launch over a (run, tile) work list for all runs, dt is
 * computed per run, and each run's result is bitwise identical to stepping it
 * alone with an af_ctx.  Device memory: one arena, about 360 doubles per cell
 * of every run.  State layout per run: as for af_ctx (af_sizes); grid
 * limits per run as for af_create. */
typedef struct af_batch af_batch;
int af_batch_create(int nruns, const int *nx, const int *ny, const double *gamma, const int *bc, af_batch **out);
int af_batch_set_domain(af_batch *b, int run, double x0, double x1, double y0, double y1);
int af_batch_set_params(af_batch *b, int run, const af_params *p);
int af_batch_set_stream(af_batch *b, void *stream);
int af_batch_set_state(af_batch *b, int run, const double *const U[4], int on_device);
int af_batch_get_state(af_batch *b, int run, double *const U[4], int on_device);
/* nsteps SSP-RK3 steps of every run (dt of each run from its own state). */
int af_batch_step(af_batch *b, int nsteps);
/* enable = 1: capture a 3-step cycle of the RK loop into a CUDA graph (needs a
 * non-default stream); af_batch_step then replays it.  enable = 0 drops it.
 * Changing domains, parameters or the stream drops the graph. */
int af_batch_graph(af_batch *b, int enable);
/* Time reps repetitions of stage 0 for each tile shape (threads per tile:
 * 32x4, 32x8, 64x2, 16x8, 64x4, 128x1) and cap on resident blocks per SM,
 * keep the fastest.  Stage 0 reads only U^n, so the state does not advance.
 * choice[4] (may be NULL) = {tile x, tile y, cap, microseconds per stage}. */
int af_batch_autotune(af_batch *b, int reps, int *choice);
/* dt used by the last step of one run (synchronises). */
int af_batch_dt(af_batch *b, int run, double *dt);
/* Counters summed over runs (newton_maxit: maximum) and the device error word, as af_status. */
int af_batch_status(af_batch *b, long long *counters, int reset);
const char *af_batch_last_error(const af_batch *b);
void af_batch_destroy(af_batch *b);

/* af_rhs without any device allocation, for callers that cannot allocate
 * device memory on their hot path (a host framework that owns all device
 * memory through its own pool, a real-time loop where cudaMalloc -- which can
 * block, synchronise the device or fail under memory pressure -- is not
 * allowed).  The paper has no counterpart: this is an interface of the
 * library, not a step of the method.
 *
 * Computes the same semi-discrete right-hand side as af_rhs (both Powell
 * source terms on) for the state U on an nx x ny grid of [x0,x1] x [y0,y1]
 * with ratio of specific heats gamma and boundary condition bc.  U[cls] and
 * dUdt[cls] are device arrays on the current device with the [8][nyp][nxp]
 * layout of af_sizes; stream is a cudaStream_t (NULL: legacy default stream);
 * the call is asynchronous in stream order and makes no allocation.  No
 * dUdt[cls] may overlap any U[cls'] (the kernels read U while they write
 * dUdt): overlapping buffers are rejected with AF_EINVAL.  The call cannot see
 * the extents of the buffers it is given, so each must hold the full class
 * array on the current device.
 *
 * Scratch: one fixed array in the library's static device memory, which every
 * GPU that loads the library holds until the process exits, sized for index
 * grids of at most AF_NOALLOC_MAX_POINTS = (nx, +1 for outflow) x (ny, +1 for
 * outflow) points; larger grids are rejected with AF_EBOUNDS.  The first call
 * on a device looks up the array's device address there (once per device);
 * make that first call before any stream capture.  All calls share the array
 * and it keeps the last call's contents; calls that overlap on the GPU race on
 * it, so serialise them (one stream, one host thread at a time).
 * Returns AF_OK, AF_EINVAL (bad argument), AF_EBOUNDS (grid too large) or
 * AF_ECUDA. */
#define AF_NOALLOC_MAX_POINTS 4225
int af_rhs_noalloc(int nx, int ny, double gamma, int bc, double x0, double x1, double y0, double y1,
                   const double *const U[4], double *const dUdt[4], void *stream);

/* Diagnostic: measured FP64 fused-multiply-add throughput of the current
 * device (a register-resident DFMA loop over all SMs, timed with CUDA events
 * on stream), written to *tflops (2 flops per FMA).  Used as the arithmetic
 * roofline of the kernels, which are bound by the FP64 pipe. */
int af_probe_fp64(void *stream, double *tflops);

/* ---------------------------------------------------------------------------
 * The 1D scheme (Sec. 4: the 1D tests use the 1D AF scheme with the LLF FVS
 * and without the Godunov-Powell source term; B1 is constant).  Reading: the
 * scheme of Sec. 2-3 restricted to one dimension.  Degrees of freedom: cell
 * averages [8][n] (class 0) and interface point values [8][nf] (class 1;
 * point f at x0 + f dx; nf = n periodic, n + 1 outflow).  Per stage: the
 * parabola centre value (6 Ubar - U_L - U_R)/4 limited by Remark 3.2; the LLF
 * FVS point update on the line (point f-1, centre f-1, point f, centre f,
 * point f+1); the Sec. 3.3 point limiter with the LLF state between
 * neighbouring points; the face flux F1 of the face point value blended with
 * the LLF flux of the adjacent averages by theta^s (Sec. 3.4, y-differences
 * zero); the Sec. 3.2 flux limiter with the faces L, R; Remark 4.1.  dt =
 * cfl dx / max varrho_1.  Conventions, parameters (af_params; the source
 * switches are ignored), counters and errors as for af_ctx.
 * ------------------------------------------------------------------------- */
typedef struct af1d_ctx af1d_ctx;
int af1d_create(int n, double gamma, int bc, af1d_ctx **out);   /* n >= 4; domain [0,1] */
int af1d_set_domain(af1d_ctx *ctx, double x0, double x1);
int af1d_set_params(af1d_ctx *ctx, const af_params *p);
int af1d_set_stream(af1d_ctx *ctx, void *stream);
/* *len = n (cls 0, averages) or nf (cls 1, point values) */
int af1d_sizes(const af1d_ctx *ctx, int cls, int *len);
int af1d_set_state(af1d_ctx *ctx, const double *const U[2], int on_device);
int af1d_get_state(af1d_ctx *ctx, double *const U[2], int on_device);
/* the output of the most recent stage (as af_get_stage) */
int af1d_get_stage(af1d_ctx *ctx, double *const U[2], int on_device);
int af1d_dt(af1d_ctx *ctx, double *dt_out, int on_device);
/* stage s in {0,1,2} as af_stage; dt NULL uses the last af1d_dt / af1d_step value */
int af1d_stage(af1d_ctx *ctx, int s, const double *dt, int on_device);
int af1d_step(af1d_ctx *ctx, double *dt_used, int on_device);
int af1d_status(af1d_ctx *ctx, long long *counters, int reset);
const char *af1d_last_error(const af1d_ctx *ctx);
/* Per-kernel device timing of the 1D stages, as af_timing (the AF_K_* ids name
 * the 1D kernels of the same passes). */
int af1d_timing(af1d_ctx *ctx, int enable, double *ms, long long *launches);
void af1d_destroy(af1d_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* AF_H */
