// af_api.cu -- host side of libaf: context, device memory, stage sequencing.
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>

#include "../../include/af.h"
#include "af_internal.h"

struct af_ctx {
  int device;
  int side[4];            // per-side boundary kinds (af_set_boundary)
  double in_lo, in_hi;
  double *inflow_dev;     // inflow state and its point data (device)
  int nx, ny, bc;
  double gamma, x0, x1, y0, y1;
  af_params prm;
  cudaStream_t stream;
  AfGrid g;
  double *state[3];       // three state buffers, 32 arrays each (4 classes x 8)
  size_t class_off[4];    // offset of each class inside a state buffer
  size_t state_len;       // doubles per state buffer
  int cur;                // buffer holding U^n
  int next_stage;         // 0, 1, 2
  int last_out;           // buffer written by the most recent stage
  double *work;           // all stage work arrays
  AfScalars *sc;
  AfStatus *st;
  AfDev dev;              // work-array pointers (state pointers set per stage)
  // adjoint workspace (allocated on first use)
  double *adj;            // af_adj_nslots() + 8 arrays per index point
  double *abuf;           // 6 state-sized buffers: lambda copies, VJP scratch, extra stage output
  double *adj_pd;         // two more point-data sets (point data and centre values of U^(0), U^(1))
  double *dts;            // dt-sensitivity work (5 * af_dt_sens_nblocks() doubles) and mu
  unsigned long long *cnt_pin;   // pinned host copy of the counters before / after a recomputation
  double *divb_buf;       // divergence measures: 2 per block, then the 2 results (allocated on first use)
  double *diag_buf;       // diagnostics: AF_NDIAG per block, then the AF_NDIAG results (allocated on first use)
  // pipelined host-buffer steps (af_step_host), created on first use: two input
  // and two output staging states, one copy stream per direction, and per slot
  // the events "input arrived", "step done with the slot", "output copied"
  double *pipe_in[2], *pipe_out[2];
  cudaStream_t h2d, d2h;
  cudaEvent_t ev_in[2], ev_used[2], ev_out[2];
  int pipe_ready;
  int pipe_slot;
  const char *recent_out[3][4];   // host output ranges of the last three af_step_host calls
  size_t recent_len[4];
  AfEventTimer tm;        // per-kernel event timing (af_timing)
  // limiter coefficients: af_record_coeffs / af_freeze_coeffs (caller's device
  // buffers of three stage blocks), and the frozen adjoint's scratch state
  double *rec_buf;
  const double *frz_buf;
  double *vscale;
  // the point work list runs on a second stream beside the face and cell passes
  cudaStream_t lstream;
  cudaEvent_t ev_fork, ev_join;
  char msg[512];
};

namespace {

int fail(af_ctx *c, int code, const char *fmt, ...) {
  if (c) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(c->msg, sizeof(c->msg), fmt, ap);
    va_end(ap);
  }
  return code;
}

int cuda_check(af_ctx *c, cudaError_t e, const char *what) {
  if (e == cudaSuccess) return AF_OK;
  return fail(c, AF_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CK(expr, what)                            \
  do {                                            \
    int rc_ = cuda_check(c, (expr), (what));      \
    if (rc_) return rc_;                          \
  } while (0)

void refresh_grid(af_ctx *c) {
  AfGrid &g = c->g;
  g.nx = c->nx;
  g.ny = c->ny;
  g.bc = c->bc;
  g.nxa = c->bc == AF_BC_OUTFLOW ? c->nx + 1 : c->nx;
  g.nya = c->bc == AF_BC_OUTFLOW ? c->ny + 1 : c->ny;
  const int fx = g.nxa, fy = g.nya;
  g.ex[0] = c->nx; g.ey[0] = c->ny;
  g.ex[1] = fx;    g.ey[1] = c->ny;
  g.ex[2] = c->nx; g.ey[2] = fy;
  g.ex[3] = fx;    g.ey[3] = fy;
  g.dx = (c->x1 - c->x0) / c->nx;
  g.dy = (c->y1 - c->y0) / c->ny;
  g.rdx = 1.0 / g.dx;
  g.rdy = 1.0 / g.dy;
  g.gamma = c->gamma;
  g.gm1 = c->gamma - 1.0;
  g.kappa = c->prm.kappa;
  g.cfl = c->prm.cfl;
  g.c13 = 1e-13 / (c->gamma - 1.0);
  g.pp_on = c->prm.pp_on;
  g.src_cell_on = c->prm.src_cell_on;
  g.src_point_on = c->prm.src_point_on;
  g.upwind = c->prm.src_point_upwind;
  g.special = 0;
  for (int k = 0; k < 4; ++k) {
    g.side[k] = c->bc == AF_BC_OUTFLOW ? c->side[k] : 0;
    if (g.side[k]) g.special = 1;
  }
  g.x0 = c->x0;
  g.in_lo = c->in_lo;
  g.in_hi = c->in_hi;
}

const double *cls_ptr(const af_ctx *c, int buf, int cls) { return c->state[buf] + c->class_off[cls]; }
double *cls_ptr_mut(af_ctx *c, int buf, int cls) { return c->state[buf] + c->class_off[cls]; }
size_t cls_len(const af_ctx *c, int cls) { return (size_t)8 * c->g.ex[cls] * c->g.ey[cls]; }

int copy_state(af_ctx *c, int buf, const double *const U[4], int on_device, bool to_ctx, double *const Uo[4]) {
  cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : (to_ctx ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToHost);
  for (int cls = 0; cls < 4; ++cls) {
    const size_t bytes = cls_len(c, cls) * sizeof(double);
    if (to_ctx) {
      if (!U[cls]) return fail(c, AF_EINVAL, "state class %d is NULL", cls);
      CK(cudaMemcpyAsync(cls_ptr_mut(c, buf, cls), U[cls], bytes, k, c->stream), "copy state in");
    } else {
      if (!Uo[cls]) return fail(c, AF_EINVAL, "state class %d is NULL", cls);
      CK(cudaMemcpyAsync(Uo[cls], cls_ptr(c, buf, cls), bytes, k, c->stream), "copy state out");
    }
  }
  if (!on_device) CK(cudaStreamSynchronize(c->stream), "synchronise");
  return AF_OK;
}

void bind_states(af_ctx *c, int bn, int bs, int bo) {
  for (int cls = 0; cls < 4; ++cls) {
    c->dev.un[cls] = cls_ptr(c, bn, cls);
    c->dev.us[cls] = cls_ptr(c, bs, cls);
    c->dev.uo[cls] = cls_ptr_mut(c, bo, cls);
  }
}

void bind_ptrs(af_ctx *c, const double *n, const double *st, double *o) {
  for (int cls = 0; cls < 4; ++cls) {
    c->dev.un[cls] = n + c->class_off[cls];
    c->dev.us[cls] = st + c->class_off[cls];
    c->dev.uo[cls] = o + c->class_off[cls];
  }
}

#define TIMED_ON(strm, kernel, call)       \
  do {                                     \
    bool on_ = c->tm.begin((kernel), strm); \
    call;                                  \
    c->tm.end(on_, strm);                  \
  } while (0)
#define TIMED(kernel, call) TIMED_ON(c->stream, kernel, call)

// One stage: P1..P5 on the bound buffers.
void run_stage(af_ctx *c, double a, double b, int reduce_dt) {
  TIMED(AF_K_POINTDATA, af_launch_pointdata(c->dev, c->g, reduce_dt, c->stream));
  if (reduce_dt) TIMED(AF_K_DT, af_launch_dt(c->dev, c->g, c->stream));
  TIMED(AF_K_POINTS, af_launch_points(c->dev, c->g, a, b, 0, c->stream));
  const bool lists = c->g.pp_on && !c->dev.frz;
  if (lists) {
    // the point list: only the next stage reads what it writes, so it runs on the
    // second stream beside the face and cell passes and joins at the end of the stage
    // (a short list would otherwise cost the latency of one thread's slow path)
    cudaEventRecord(c->ev_fork, c->stream);
    cudaStreamWaitEvent(c->lstream, c->ev_fork, 0);
    TIMED_ON(c->lstream, AF_K_POINTS_SLOW, af_launch_points_slow(c->dev, c->g, a, b, c->lstream));
    cudaEventRecord(c->ev_join, c->lstream);
  }
  TIMED(AF_K_FACES, af_launch_faces(c->dev, c->g, 0, c->stream));
  TIMED(AF_K_CELLS, af_launch_cells(c->dev, c->g, a, b, 0, c->stream));
  if (lists) TIMED(AF_K_CELLS_SLOW, af_launch_cells_slow(c->dev, c->g, c->stream));
  if (c->g.pp_on) {
    TIMED(AF_K_FINAL, af_launch_final(c->dev, c->g, a, b, c->stream));
    TIMED(AF_K_REPAIR, af_launch_repair(c->dev, c->g, a, b, c->stream));
  }
  if (lists) cudaStreamWaitEvent(c->stream, c->ev_join, 0);
}

const double RK_A[3] = {0.0, 3.0 / 4.0, 1.0 / 3.0};
const double RK_B[3] = {1.0, 1.0 / 4.0, 2.0 / 3.0};

int set_dt(af_ctx *c, const double *dt, int on_device) {
  if (!dt) return AF_OK;
  cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  if (!on_device && !(*dt > 0.0)) return fail(c, AF_EINVAL, "dt must be positive");
  CK(cudaMemcpyAsync(&c->sc->dt, dt, sizeof(double), k, c->stream), "set dt");
  if (!on_device) CK(cudaStreamSynchronize(c->stream), "synchronise");
  return AF_OK;
}

int stage_impl(af_ctx *c, int s, int reduce_dt) {
  const int n = c->cur, b1 = (c->cur + 1) % 3, b2 = (c->cur + 2) % 3;
  if (s == 0) bind_states(c, n, n, b1);
  else if (s == 1) bind_states(c, n, b1, b2);
  else bind_states(c, n, b2, b1);
  const size_t PS = (size_t)c->g.nxa * c->g.nya, blk = (size_t)AF_NCOEF * PS;
  c->dev.rec = c->rec_buf ? c->rec_buf + s * blk : nullptr;
  c->dev.frz = c->frz_buf ? c->frz_buf + s * blk : nullptr;
  run_stage(c, RK_A[s], RK_B[s], reduce_dt);
  if (c->dev.rec && c->g.pp_on) {   // face theta after the Remark 4.1 repair
    CK(cudaMemcpyAsync(c->dev.rec + AFC_THX * PS, c->dev.thx, PS * sizeof(double), cudaMemcpyDeviceToDevice,
                       c->stream), "record face theta");
    CK(cudaMemcpyAsync(c->dev.rec + AFC_THY * PS, c->dev.thy, PS * sizeof(double), cudaMemcpyDeviceToDevice,
                       c->stream), "record face theta");
  }
  c->dev.rec = nullptr;
  c->dev.frz = nullptr;
  CK(cudaGetLastError(), "stage launch");
  c->last_out = s == 1 ? b2 : b1;
  if (s == 2) c->cur = b1;
  c->next_stage = (s + 1) % 3;
  return AF_OK;
}

}  // namespace

extern "C" {

int af_create(int nx, int ny, double gamma, int bc, af_ctx **out) {
  if (!out) return AF_EINVAL;
  *out = nullptr;
  if (!af_grid_fits(nx, ny) || !(gamma > 1.0) || (bc != AF_BC_PERIODIC && bc != AF_BC_OUTFLOW)) return AF_EINVAL;
  af_ctx *c = new (std::nothrow) af_ctx();
  if (!c) return AF_ENOMEM;
  c->nx = nx;
  c->ny = ny;
  c->bc = bc;
  c->gamma = gamma;
  c->x0 = 0.0; c->x1 = 1.0; c->y0 = 0.0; c->y1 = 1.0;
  c->prm.cfl = 0.2;
  c->prm.kappa = 0.0;
  c->prm.pp_on = 1;
  c->prm.src_cell_on = 1;
  c->prm.src_point_on = 1;
  c->prm.src_point_upwind = 0;
  c->stream = nullptr;
  if (cudaGetDevice(&c->device) != cudaSuccess) {
    delete c;
    return AF_ECUDA;
  }
  refresh_grid(c);
  size_t off = 0;
  for (int cls = 0; cls < 4; ++cls) {
    c->class_off[cls] = off;
    off += cls_len(c, cls);
  }
  c->state_len = off;
  const size_t PS = (size_t)c->g.nxa * c->g.nya;
  // stage work arrays, then the limiter work lists: points (3 PS entries: an int and 8
  // doubles each), cells (PS entries: an int and 2 doubles each)
  // and the vertex list (16 PS entries, an unsigned each) with Lambda^rho of the listed cells (4 PS)
  const size_t nwork = PS * (AF_NQA + 4 * AF_NQP + 8 + 4 + 2 * AF_NQF + 4 + 8 + 2) + PS * (24 + 2) + 2 * PS + 1 +
                       PS * (8 + 4);
  int rc = AF_OK;
  for (int b = 0; b < 3; ++b) {
    if (cudaMalloc(&c->state[b], off * sizeof(double)) != cudaSuccess) rc = AF_ENOMEM;
    else if (cudaMemset(c->state[b], 0, off * sizeof(double)) != cudaSuccess) rc = AF_ECUDA;
  }
  if (!rc && cudaMalloc(&c->work, nwork * sizeof(double)) != cudaSuccess) rc = AF_ENOMEM;
  if (!rc && cudaMemset(c->work, 0, nwork * sizeof(double)) != cudaSuccess) rc = AF_ECUDA;
  if (!rc && cudaMalloc(&c->sc, sizeof(AfScalars)) != cudaSuccess) rc = AF_ENOMEM;
  if (!rc && cudaMalloc(&c->st, sizeof(AfStatus)) != cudaSuccess) rc = AF_ENOMEM;
  if (!rc && cudaMemset(c->sc, 0, sizeof(AfScalars)) != cudaSuccess) rc = AF_ECUDA;
  if (!rc && cudaMemset(c->st, 0, sizeof(AfStatus)) != cudaSuccess) rc = AF_ECUDA;
  if (!rc && cudaStreamCreateWithFlags(&c->lstream, cudaStreamNonBlocking) != cudaSuccess) rc = AF_ECUDA;
  if (!rc && cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) != cudaSuccess) rc = AF_ECUDA;
  if (!rc && cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming) != cudaSuccess) rc = AF_ECUDA;
  if (!rc && cudaDeviceSynchronize() != cudaSuccess) rc = AF_ECUDA;
  if (rc) {
    cudaGetLastError();
    af_destroy(c);
    return rc;
  }
  double *w = c->work;
  c->dev.pd[0] = w; w += AF_NQA * PS;
  for (int k = 1; k <= 4; ++k) { c->dev.pd[k] = w; w += AF_NQP * PS; }
  c->dev.uc = w; w += 8 * PS;
  c->dev.phi = w; w += 4 * PS;
  c->dev.fx = w; w += AF_NQF * PS;
  c->dev.fy = w; w += AF_NQF * PS;
  c->dev.lam = w; w += 4 * PS;
  c->dev.lim1 = w; w += 8 * PS;
  c->dev.thx = w; w += PS;
  c->dev.thy = w; w += PS;
  c->dev.pq_cap = (int)(3 * PS);
  c->dev.cq_cap = (int)PS;
  c->dev.pqu = w; w += 24 * PS;
  c->dev.cqe = w; w += 2 * PS;
  c->dev.pq = reinterpret_cast<int *>(w); w += (3 * PS + 1) / 2;
  c->dev.cq = reinterpret_cast<int *>(w); w += (PS + 1) / 2;
  c->dev.cql = w; w += 4 * PS;
  c->dev.vq_cap = (int)(16 * PS);
  c->dev.vq = reinterpret_cast<unsigned *>(w); w += 8 * PS;
  c->dev.sc = c->sc;
  c->dev.st = c->st;
  c->cur = 0;
  c->next_stage = 0;
  c->msg[0] = 0;
  *out = c;
  return AF_OK;
}

int af_set_domain(af_ctx *c, double x0, double x1, double y0, double y1) {
  if (!c) return AF_EINVAL;
  if (!(x1 > x0) || !(y1 > y0)) return fail(c, AF_EINVAL, "empty domain");
  c->x0 = x0; c->x1 = x1; c->y0 = y0; c->y1 = y1;
  refresh_grid(c);
  return AF_OK;
}

int af_set_boundary(af_ctx *c, const int side[4], double inflow_lo, double inflow_hi, const double inflow_U[8]) {
  if (!c || !side) return AF_EINVAL;
  if (c->bc != AF_BC_OUTFLOW) return fail(c, AF_EINVAL, "per-side boundary kinds need an outflow (non-periodic) grid");
  bool inflow = false;
  for (int k = 0; k < 4; ++k) {
    if (side[k] < AF_SIDE_OUTFLOW || side[k] > AF_SIDE_INFLOW) return fail(c, AF_EINVAL, "side %d: unknown kind", k);
    if (side[k] == AF_SIDE_INFLOW && k < 2) return fail(c, AF_EINVAL, "inflow is supported on the bottom and top sides");
    inflow = inflow || side[k] == AF_SIDE_INFLOW;
  }
  if (inflow && (!inflow_U || !(inflow_U[0] > 0.0))) return fail(c, AF_EINVAL, "inflow state missing or rho <= 0");
  CK(cudaSetDevice(c->device), "set device");
  for (int k = 0; k < 4; ++k) c->side[k] = side[k];
  c->in_lo = inflow_lo;
  c->in_hi = inflow_hi;
  refresh_grid(c);
  if (!c->inflow_dev) {
    if (cudaMalloc(&c->inflow_dev, sizeof(double) * (8 + AF_NQP + AF_NQA)) != cudaSuccess) {
      cudaGetLastError();
      return fail(c, AF_ENOMEM, "inflow table");
    }
    CK(cudaMemset(c->inflow_dev, 0, sizeof(double) * (8 + AF_NQP + AF_NQA)), "clear inflow table");
  }
  if (inflow) {
    CK(cudaMemcpy(c->inflow_dev, inflow_U, 8 * sizeof(double), cudaMemcpyHostToDevice), "inflow state");
    af_launch_inflow_pd(c->g, c->inflow_dev, c->inflow_dev, c->stream);
    CK(cudaGetLastError(), "inflow point data");
    CK(cudaStreamSynchronize(c->stream), "synchronise");
  }
  c->dev.inflow = c->inflow_dev;
  return AF_OK;
}

int af_set_params(af_ctx *c, const af_params *p) {
  if (!c || !p) return AF_EINVAL;
  if (!(p->cfl > 0.0) || !(p->kappa >= 0.0)) return fail(c, AF_EINVAL, "cfl must be > 0 and kappa >= 0");
  c->prm = *p;
  refresh_grid(c);
  return AF_OK;
}

int af_get_params(const af_ctx *c, af_params *p) {
  if (!c || !p) return AF_EINVAL;
  *p = c->prm;
  return AF_OK;
}

int af_set_stream(af_ctx *c, void *stream) {
  if (!c) return AF_EINVAL;
  c->stream = (cudaStream_t)stream;
  return AF_OK;
}

int af_sizes(const af_ctx *c, int cls, int *nxp, int *nyp) {
  if (!c || cls < 0 || cls > 3 || !nxp || !nyp) return AF_EINVAL;
  *nxp = c->g.ex[cls];
  *nyp = c->g.ey[cls];
  return AF_OK;
}

int af_set_state(af_ctx *c, const double *const U[4], int on_device) {
  if (!c || !U) return AF_EINVAL;
  CK(cudaSetDevice(c->device), "set device");
  c->next_stage = 0;
  return copy_state(c, c->cur, U, on_device, true, nullptr);
}

int af_get_state(af_ctx *c, double *const U[4], int on_device) {
  if (!c || !U) return AF_EINVAL;
  CK(cudaSetDevice(c->device), "set device");
  return copy_state(c, c->cur, nullptr, on_device, false, U);
}

int af_rhs(af_ctx *c, double *const dUdt[4], int on_device) {
  if (!c || !dUdt) return AF_EINVAL;
  CK(cudaSetDevice(c->device), "set device");
  const int scratch = (c->cur + 1) % 3;
  bind_states(c, c->cur, c->cur, scratch);
  af_launch_pointdata(c->dev, c->g, 0, c->stream);
  af_launch_points(c->dev, c->g, 0.0, 1.0, 1, c->stream);
  af_launch_faces(c->dev, c->g, 1, c->stream);
  af_launch_cells(c->dev, c->g, 0.0, 1.0, 1, c->stream);
  CK(cudaGetLastError(), "rhs launch");
  c->next_stage = 0;
  return copy_state(c, scratch, nullptr, on_device, false, dUdt);
}

int af_sensor(af_ctx *c, double *theta_x, double *theta_y, int on_device) {
  if (!c || !theta_x || !theta_y) return AF_EINVAL;
  CK(cudaSetDevice(c->device), "set device");
  bind_states(c, c->cur, c->cur, (c->cur + 1) % 3);
  af_launch_pointdata(c->dev, c->g, 0, c->stream);
  af_launch_points(c->dev, c->g, 0.0, 1.0, 2, c->stream);
  af_launch_faces(c->dev, c->g, 2, c->stream);
  CK(cudaGetLastError(), "sensor launch");
  const size_t PS = (size_t)c->g.nxa * c->g.nya;
  cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  const AfGrid &g = c->g;
  CK(cudaMemcpy2DAsync(theta_x, g.ex[1] * sizeof(double), c->dev.fx + QF_TS * PS, g.nxa * sizeof(double),
                       g.ex[1] * sizeof(double), g.ey[1], k, c->stream), "copy theta_x");
  CK(cudaMemcpy2DAsync(theta_y, g.ex[2] * sizeof(double), c->dev.fy + QF_TS * PS, g.nxa * sizeof(double),
                       g.ex[2] * sizeof(double), g.ey[2], k, c->stream), "copy theta_y");
  if (!on_device) CK(cudaStreamSynchronize(c->stream), "synchronise");
  c->next_stage = 0;
  return AF_OK;
}

int af_dt(af_ctx *c, double *dt_out, int on_device) {
  if (!c) return AF_EINVAL;
  CK(cudaSetDevice(c->device), "set device");
  bind_states(c, c->cur, c->cur, (c->cur + 1) % 3);
  af_launch_pointdata(c->dev, c->g, 1, c->stream);
  af_launch_dt(c->dev, c->g, c->stream);
  CK(cudaGetLastError(), "dt launch");
  if (dt_out) {
    CK(cudaMemcpyAsync(dt_out, &c->sc->dt, sizeof(double), on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                       c->stream),
       "copy dt");
    if (!on_device) CK(cudaStreamSynchronize(c->stream), "synchronise");
  }
  return AF_OK;
}

int af_stage(af_ctx *c, int s, const double *dt, int on_device) {
  AfNvtxRange nvtx_("af_stage");
  if (!c || s < 0 || s > 2) return AF_EINVAL;
  if (s != c->next_stage) return fail(c, AF_EINVAL, "stage %d called, stage %d expected", s, c->next_stage);
  CK(cudaSetDevice(c->device), "set device");
  int rc = set_dt(c, dt, on_device);
  if (rc) return rc;
  return stage_impl(c, s, 0);
}

// ---- adjoint ---------------------------------------------------------------
namespace {
// doubles of one point-data set per index point: pd classes 0..4 and the centre values
constexpr size_t kPdLen = AF_NQA + 4 * AF_NQP + 8;

int ensure_adjoint(af_ctx *c) {
  if (c->adj) return AF_OK;
  const size_t PS = (size_t)c->g.nxa * c->g.nya;
  if (cudaMalloc(&c->adj, sizeof(double) * PS * (af_adj_nslots() + 8)) != cudaSuccess ||
      cudaMalloc(&c->abuf, sizeof(double) * 6 * c->state_len) != cudaSuccess ||
      cudaMalloc(&c->adj_pd, sizeof(double) * 2 * kPdLen * PS) != cudaSuccess ||
      cudaMalloc(&c->dts, sizeof(double) * (5 * (size_t)af_dt_sens_nblocks() + 1)) != cudaSuccess ||
      cudaMallocHost(&c->cnt_pin, sizeof(unsigned long long) * 32) != cudaSuccess) {
    cudaGetLastError();
    return fail(c, AF_ENOMEM, "adjoint workspace");
  }
  return AF_OK;
}
double *abuf(af_ctx *c, int k) { return c->abuf + (size_t)k * c->state_len; }
void class_ptrs(af_ctx *c, double *base, double **out) {
  for (int cls = 0; cls < 4; ++cls) out[cls] = base + c->class_off[cls];
}
// point data (pd[0..4], uc) of set 0 or 1 (adjoint workspace) or 2 (the context's own)
void bind_pd(af_ctx *c, int set) {
  const size_t PS = (size_t)c->g.nxa * c->g.nya;
  double *w = set == 2 ? c->work : c->adj_pd + (size_t)set * kPdLen * PS;
  c->dev.pd[0] = w; w += AF_NQA * PS;
  for (int k = 1; k <= 4; ++k) { c->dev.pd[k] = w; w += AF_NQP * PS; }
  c->dev.uc = w;
}
// State pointers of every pass to the classes U[4] (the point-data pass and
// the transposed kernels read them and write nothing through them).
void bind_cls(af_ctx *c, const double *const U[4]) {
  for (int cls = 0; cls < 4; ++cls) {
    c->dev.un[cls] = U[cls];
    c->dev.us[cls] = U[cls];
    c->dev.uo[cls] = const_cast<double *>(U[cls]);
  }
}
void buf_cls(const af_ctx *c, const double *base, const double *out[4]) {
  for (int cls = 0; cls < 4; ++cls) out[cls] = base + c->class_off[cls];
}
// Transposed operator at the state U (class pointers) whose point data is in
// set `set`: the last kernel writes e.out1 (and e.out2), see AfAdjEpi.
void vjp_at(af_ctx *c, const double *const U[4], int set, const AfAdjEpi &e, const double *co = nullptr) {
  bind_pd(c, set);
  bind_cls(c, U);
  double *tp[4], *vs[4];
  class_ptrs(c, abuf(c, 1), tp);
  if (co) class_ptrs(c, c->vscale, vs);
  const size_t PS = (size_t)c->g.nxa * c->g.nya;
  af_launch_vjp(c->dev, c->g, e, c->adj, c->adj + (size_t)af_adj_nslots() * PS, tp, c->stream, co,
                co ? vs : nullptr);
  bind_pd(c, 2);
}
AfAdjEpi epi(const double *const v[4], double *const out1[4], double a, double b, const double *dt) {
  AfAdjEpi e;
  memset(&e, 0, sizeof(e));
  for (int cls = 0; cls < 4; ++cls) {
    e.v[cls] = v[cls];
    e.out1[cls] = out1[cls];
  }
  e.a = a;
  e.b = b;
  e.dt = dt;
  return e;
}
int copy_in_buf(af_ctx *c, double *dst, const double *const U[4], int on_device) {
  for (int cls = 0; cls < 4; ++cls) {
    if (!U[cls]) return fail(c, AF_EINVAL, "class %d is NULL", cls);
    CK(cudaMemcpyAsync(dst + c->class_off[cls], U[cls], cls_len(c, cls) * sizeof(double),
                       on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream),
       "copy in");
  }
  return AF_OK;
}
int copy_out_buf(af_ctx *c, const double *src, double *const U[4], int on_device) {
  for (int cls = 0; cls < 4; ++cls) {
    if (!U[cls]) return fail(c, AF_EINVAL, "class %d is NULL", cls);
    CK(cudaMemcpyAsync(U[cls], src + c->class_off[cls], cls_len(c, cls) * sizeof(double),
                       on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream),
       "copy out");
  }
  if (!on_device) CK(cudaStreamSynchronize(c->stream), "synchronise");
  return AF_OK;
}
}  // namespace

int af_rhs_vjp(af_ctx *c, const double *const v[4], double *const out[4], int on_device) {
  AfNvtxRange nvtx_("af_rhs_vjp");
  if (!c || !v || !out) return AF_EINVAL;
  if (c->g.special) return fail(c, AF_EINVAL, "the transpose covers periodic and outflow boundaries only");
  if (c->g.upwind) return fail(c, AF_EINVAL, "the transpose covers the central point source only");
  for (int cls = 0; cls < 4; ++cls)
    if (!v[cls] || !out[cls]) return fail(c, AF_EINVAL, "class %d is NULL", cls);
  CK(cudaSetDevice(c->device), "set device");
  int rc = ensure_adjoint(c);
  if (rc) return rc;
  const double *vp[4];
  double *op[4], *in_buf[4], *out_buf[4];
  class_ptrs(c, abuf(c, 0), in_buf);
  class_ptrs(c, abuf(c, 2), out_buf);
  if (!on_device) {
    rc = copy_in_buf(c, abuf(c, 0), v, 0);
    if (rc) return rc;
  }
  for (int cls = 0; cls < 4; ++cls) {
    vp[cls] = on_device ? v[cls] : in_buf[cls];
    op[cls] = on_device ? out[cls] : out_buf[cls];
  }
  bind_states(c, c->cur, c->cur, c->cur);
  af_launch_pointdata(c->dev, c->g, 0, c->stream);
  const double *Ucur[4];
  buf_cls(c, c->state[c->cur], Ucur);
  vjp_at(c, Ucur, 2, epi(vp, op, 0.0, 1.0, nullptr));
  CK(cudaGetLastError(), "vjp launch");
  c->next_stage = 0;
  if (on_device) return AF_OK;
  return copy_out_buf(c, abuf(c, 2), out, 0);
}

namespace {
// Reverse sweep of one SSP-RK3 step, shared by af_adjoint_step and
// af_adjoint_step_stages.  S[0..2] are the class pointers of the stage states
// U0, U1, U2, whose point data are in the sets 0, 1 and 2; S[3] is U3 =
// U^{n+1} (read only with_dt).  dt is on the device (c->sc->dt).
int adjoint_sweep(af_ctx *c, const double *const S[4][4], const double *const lam_in[4], double *const lam_out[4],
                  int on_device, bool with_dt, const double *coeffs = nullptr) {
  const size_t blk = (size_t)AF_NCOEF * c->g.nxa * c->g.nya;
  const double *co[3] = {coeffs, coeffs ? coeffs + blk : nullptr, coeffs ? coeffs + 2 * blk : nullptr};
  const double *dtp = &c->sc->dt;
  int rc = AF_OK;
  // reverse of U1 = FE(U0), U2 = 3/4 U0 + 1/4 FE(U1), U3 = 1/3 U0 + 2/3 FE(U2), FE(U) = U + dt L(U):
  //   L2 = 2/3 (L3 + dt T(U2) L3),  L1 = 1/4 (L2 + dt T(U1) L2),  W = 3/4 L2 + 1/3 L3,
  //   L0 = L1 + dt T(U0) L1 + W,    T(U) = (dL/dU)^T
  double *L3b[4], *L2[4], *L1[4], *W[4], *L0b[4];
  class_ptrs(c, abuf(c, 0), L3b);
  class_ptrs(c, abuf(c, 2), L2);
  class_ptrs(c, abuf(c, 3), L1);
  class_ptrs(c, abuf(c, 4), W);
  class_ptrs(c, abuf(c, 1), L0b);   // the scratch of the last VJP; L3 stays readable
  if (!on_device) {
    rc = copy_in_buf(c, abuf(c, 0), lam_in, 0);
    if (rc) return rc;
  }
  const double *L3[4];
  double *L0[4];
  for (int cls = 0; cls < 4; ++cls) {
    L3[cls] = on_device ? lam_in[cls] : L3b[cls];
    L0[cls] = on_device ? lam_out[cls] : L0b[cls];
  }
  vjp_at(c, S[2], 2, epi(L3, L2, 2.0 / 3.0, 2.0 / 3.0, dtp), co[2]);
  AfAdjEpi e1 = epi(L2, L1, 0.25, 0.25, dtp);
  for (int cls = 0; cls < 4; ++cls) {
    e1.out2[cls] = W[cls];
    e1.z2[cls] = L3[cls];
  }
  e1.e = 0.75;
  e1.f = 1.0 / 3.0;
  vjp_at(c, S[1], 1, e1, co[1]);
  if (with_dt) {   // mu dt from L3, L2, L1 and the stage states, before the last VJP may overwrite L3
    af_launch_dt_dot(c->g, L3, L2, L1, S[0], S[1], S[2], S[3], c->dts, c->stream);
  }
  AfAdjEpi e0 = epi(L1, L0, 1.0, 1.0, dtp);
  for (int cls = 0; cls < 4; ++cls) e0.z1[cls] = W[cls];
  e0.c = 1.0;
  vjp_at(c, S[0], 0, e0, co[0]);
  if (with_dt) {
    bind_pd(c, 0);
    bind_cls(c, S[0]);
    af_launch_dt_apply(c->dev, c->g, L0, c->dts, c->dts + 5 * (size_t)af_dt_sens_nblocks(), c->stream);
    bind_pd(c, 2);
  }
  CK(cudaGetLastError(), "adjoint launch");
  return AF_OK;
}

// Shared argument checks of the two adjoint steps.
int adjoint_args(af_ctx *c, const double *dt, const double *const lam_in[4], double *const lam_out[4], int flags) {
  if (!dt || !lam_in || !lam_out) return fail(c, AF_EINVAL, "NULL argument");
  for (int cls = 0; cls < 4; ++cls)
    if (!lam_in[cls] || !lam_out[cls]) return fail(c, AF_EINVAL, "class %d is NULL", cls);
  if (flags & ~(AF_ADJ_RECORDED | AF_ADJ_DT)) return fail(c, AF_EINVAL, "unknown flags %d", flags);
  if (c->g.special) return fail(c, AF_EINVAL, "the transpose covers periodic and outflow boundaries only");
  if (c->g.upwind) return fail(c, AF_EINVAL, "the transpose covers the central point source only");
  if (c->g.kappa != 0.0)
    return fail(c, AF_EINVAL, "the adjoint differentiates the scheme with the shock sensor off (kappa = 0)");
  return AF_OK;
}
}  // namespace

int af_adjoint_step(af_ctx *c, const double *dt, int dt_on_device, const double *const lam_in[4],
                    double *const lam_out[4], int on_device, int flags) {
  AfNvtxRange nvtx_("af_adjoint_step");
  if (!c) return AF_EINVAL;
  int rc = adjoint_args(c, dt, lam_in, lam_out, flags);
  if (rc) return rc;
  const bool with_dt = (flags & AF_ADJ_DT) != 0;
  CK(cudaSetDevice(c->device), "set device");
  rc = ensure_adjoint(c);
  if (!rc) rc = set_dt(c, dt, dt_on_device);
  if (rc) return rc;
  const size_t cnt_bytes = sizeof(unsigned long long) * 16;
  CK(cudaMemcpyAsync(c->cnt_pin, c->st->cnt, cnt_bytes, cudaMemcpyDeviceToHost, c->stream), "read status");
  // recompute U1 = FE(U0), U2 = 3/4 U0 + 1/4 FE(U1) with the recorded dt, each
  // stage's point data in its own set; then the point data of U2 (or stage 2
  // into a spare buffer, to see whether a limiter acts there)
  const int n = c->cur, b1 = (c->cur + 1) % 3, b2 = (c->cur + 2) % 3;
  bind_pd(c, 0);
  bind_states(c, n, n, b1);
  run_stage(c, RK_A[0], RK_B[0], 0);
  bind_pd(c, 1);
  bind_states(c, n, b1, b2);
  run_stage(c, RK_A[1], RK_B[1], 0);
  bind_pd(c, 2);
  if ((flags & AF_ADJ_RECORDED) && !with_dt) {
    bind_states(c, b2, b2, b2);
    af_launch_pointdata(c->dev, c->g, 0, c->stream);
  } else {
    bind_states(c, n, b2, b1);
    for (int cls = 0; cls < 4; ++cls) c->dev.uo[cls] = abuf(c, 5) + c->class_off[cls];
    run_stage(c, RK_A[2], RK_B[2], 0);
  }
  CK(cudaGetLastError(), "stage recompute");
  CK(cudaMemcpyAsync(c->cnt_pin + 16, c->st->cnt, cnt_bytes, cudaMemcpyDeviceToHost, c->stream), "read status");
  const double *S[4][4];
  buf_cls(c, c->state[n], S[0]);
  buf_cls(c, c->state[b1], S[1]);
  buf_cls(c, c->state[b2], S[2]);
  buf_cls(c, abuf(c, 5), S[3]);
  rc = adjoint_sweep(c, S, lam_in, lam_out, on_device, with_dt);
  if (rc) return rc;
  c->next_stage = 0;
  if (!on_device) {
    rc = copy_out_buf(c, abuf(c, 1), lam_out, 0);
    if (rc) return rc;
  }
  CK(cudaStreamSynchronize(c->stream), "synchronise");
  const int lim[] = {ST_SRC_LIMITED, ST_LAMBDA_LT1, ST_FACE_THETA_LT1, ST_SHRINK, ST_POINT_LIMITED, ST_CENTER_LIMITED,
                     ST_NONADMISSIBLE};
  for (int k : lim)
    if (c->cnt_pin[16 + k] != c->cnt_pin[k])
      return fail(c, AF_EINVAL, "af_adjoint_step: a limiter was active in this step (counter %d); the transpose "
                  "covers the branch on which every limiter is inactive", k);
  return AF_OK;
}

int af_adjoint_step_stages(af_ctx *c, const double *dt, int dt_on_device, const double *const U1[4],
                           const double *const U2[4], const double *const U3[4], const double *const lam_in[4],
                           double *const lam_out[4], int on_device, int flags) {
  AfNvtxRange nvtx_("af_adjoint_step_stages");
  if (!c) return AF_EINVAL;
  int rc = adjoint_args(c, dt, lam_in, lam_out, flags);
  if (rc) return rc;
  const bool with_dt = (flags & AF_ADJ_DT) != 0;
  if (!U1 || !U2 || (with_dt && !U3)) return fail(c, AF_EINVAL, "stage states missing");
  for (int cls = 0; cls < 4; ++cls)
    if (!U1[cls] || !U2[cls] || (with_dt && !U3[cls])) return fail(c, AF_EINVAL, "stage class %d is NULL", cls);
  CK(cudaSetDevice(c->device), "set device");
  rc = ensure_adjoint(c);
  if (!rc) rc = set_dt(c, dt, dt_on_device);
  if (rc) return rc;
  const int n = c->cur, b1 = (c->cur + 1) % 3, b2 = (c->cur + 2) % 3;
  const double *S[4][4];
  buf_cls(c, c->state[n], S[0]);
  if (on_device) {
    for (int cls = 0; cls < 4; ++cls) {
      S[1][cls] = U1[cls];
      S[2][cls] = U2[cls];
      S[3][cls] = with_dt ? U3[cls] : nullptr;
    }
  } else {   // host stage states go to the context's stage buffers (and the spare one)
    rc = copy_in_buf(c, c->state[b1], U1, 0);
    if (!rc) rc = copy_in_buf(c, c->state[b2], U2, 0);
    if (!rc && with_dt) rc = copy_in_buf(c, abuf(c, 5), U3, 0);
    if (rc) return rc;
    buf_cls(c, c->state[b1], S[1]);
    buf_cls(c, c->state[b2], S[2]);
    buf_cls(c, abuf(c, 5), S[3]);
  }
  const size_t cnt_bytes = sizeof(unsigned long long) * 16;
  CK(cudaMemcpyAsync(c->cnt_pin, c->st->cnt, cnt_bytes, cudaMemcpyDeviceToHost, c->stream), "read status");
  for (int set = 0; set < 3; ++set) {   // point data (and limited centre values) of U0, U1, U2
    bind_pd(c, set);
    bind_cls(c, S[set]);
    af_launch_pointdata(c->dev, c->g, 0, c->stream);
  }
  CK(cudaGetLastError(), "point data");
  CK(cudaMemcpyAsync(c->cnt_pin + 16, c->st->cnt, cnt_bytes, cudaMemcpyDeviceToHost, c->stream), "read status");
  rc = adjoint_sweep(c, S, lam_in, lam_out, on_device, with_dt);
  bind_pd(c, 2);
  bind_states(c, c->cur, c->cur, (c->cur + 1) % 3);
  if (rc) return rc;
  c->next_stage = 0;
  if (!on_device) {
    rc = copy_out_buf(c, abuf(c, 1), lam_out, 0);
    if (rc) return rc;
  }
  CK(cudaStreamSynchronize(c->stream), "synchronise");
  if (c->cnt_pin[16 + ST_CENTER_LIMITED] != c->cnt_pin[ST_CENTER_LIMITED])
    return fail(c, AF_EINVAL, "af_adjoint_step_stages: the cell-centre limiter acted on a stage state; the transpose "
                "covers the branch on which every limiter is inactive");
  return AF_OK;
}

// ---- the frozen branch: recorded limiter coefficients ------------------------
int af_coeff_len(const af_ctx *c, long long *n) {
  if (!c || !n) return AF_EINVAL;
  *n = (long long)AF_NCOEF * c->g.nxa * c->g.nya;
  return AF_OK;
}

int af_record_coeffs(af_ctx *c, double *buf) {
  if (!c) return AF_EINVAL;
  if (buf && c->frz_buf) return fail(c, AF_EINVAL, "coefficients are frozen; af_freeze_coeffs(ctx, NULL) first");
  c->rec_buf = buf;
  return AF_OK;
}

int af_freeze_coeffs(af_ctx *c, const double *buf) {
  if (!c) return AF_EINVAL;
  if (buf && c->rec_buf) return fail(c, AF_EINVAL, "coefficients are being recorded; af_record_coeffs(ctx, NULL) first");
  if (buf && !c->g.pp_on) return fail(c, AF_EINVAL, "the frozen branch needs the positivity limiters on");
  c->frz_buf = buf;
  return AF_OK;
}

namespace {
int frozen_args(af_ctx *c, const double *coeffs) {
  if (!coeffs) return fail(c, AF_EINVAL, "coefficients missing");
  if (c->g.special) return fail(c, AF_EINVAL, "the transpose covers periodic and outflow boundaries only");
  if (c->g.upwind) return fail(c, AF_EINVAL, "the transpose covers the central point source only");
  if (!c->g.pp_on) return fail(c, AF_EINVAL, "the frozen branch needs the positivity limiters on");
  if (!c->vscale && cudaMalloc(&c->vscale, sizeof(double) * c->state_len) != cudaSuccess) {
    cudaGetLastError();
    return fail(c, AF_ENOMEM, "frozen adjoint workspace");
  }
  return AF_OK;
}
// point data (and limited centre values, Remark 3.2 frozen at co) of U into set `set`
void frozen_pointdata(af_ctx *c, const double *const U[4], int set, const double *co) {
  bind_pd(c, set);
  bind_cls(c, U);
  c->dev.frz = co;
  af_launch_pointdata(c->dev, c->g, 0, c->stream);
  c->dev.frz = nullptr;
}
}  // namespace

int af_stage_vjp(af_ctx *c, const double *dt, int dt_on_device, const double *coeffs, const double *const lam[4],
                 double *const out[4], int on_device) {
  AfNvtxRange nvtx_("af_stage_vjp");
  if (!c || !lam || !out) return AF_EINVAL;
  for (int cls = 0; cls < 4; ++cls)
    if (!lam[cls] || !out[cls]) return fail(c, AF_EINVAL, "class %d is NULL", cls);
  int rc = frozen_args(c, coeffs);
  if (rc) return rc;
  CK(cudaSetDevice(c->device), "set device");
  rc = ensure_adjoint(c);
  if (!rc) rc = set_dt(c, dt, dt_on_device);
  if (rc) return rc;
  const double *vp[4], *Ucur[4];
  double *op[4], *in_buf[4], *out_buf[4];
  class_ptrs(c, abuf(c, 0), in_buf);
  class_ptrs(c, abuf(c, 2), out_buf);
  if (!on_device) {
    rc = copy_in_buf(c, abuf(c, 0), lam, 0);
    if (rc) return rc;
  }
  for (int cls = 0; cls < 4; ++cls) {
    vp[cls] = on_device ? lam[cls] : in_buf[cls];
    op[cls] = on_device ? out[cls] : out_buf[cls];
  }
  buf_cls(c, c->state[c->cur], Ucur);
  frozen_pointdata(c, Ucur, 2, coeffs);
  vjp_at(c, Ucur, 2, epi(vp, op, 1.0, 1.0, &c->sc->dt), coeffs);
  bind_states(c, c->cur, c->cur, (c->cur + 1) % 3);
  CK(cudaGetLastError(), "stage vjp launch");
  c->next_stage = 0;
  if (on_device) return AF_OK;
  return copy_out_buf(c, abuf(c, 2), out, 0);
}

int af_adjoint_step_frozen(af_ctx *c, const double *dt, int dt_on_device, const double *const U1[4],
                           const double *const U2[4], const double *const U3[4], const double *coeffs,
                           const double *const lam_in[4], double *const lam_out[4], int on_device, int flags) {
  AfNvtxRange nvtx_("af_adjoint_step_frozen");
  if (!c) return AF_EINVAL;
  if (!dt || !lam_in || !lam_out) return fail(c, AF_EINVAL, "NULL argument");
  for (int cls = 0; cls < 4; ++cls)
    if (!lam_in[cls] || !lam_out[cls]) return fail(c, AF_EINVAL, "class %d is NULL", cls);
  if (flags & ~AF_ADJ_DT) return fail(c, AF_EINVAL, "unknown flags %d", flags);
  const bool with_dt = (flags & AF_ADJ_DT) != 0;
  int rc = frozen_args(c, coeffs);
  if (rc) return rc;
  if (!U1 || !U2 || (with_dt && !U3)) return fail(c, AF_EINVAL, "stage states missing");
  for (int cls = 0; cls < 4; ++cls)
    if (!U1[cls] || !U2[cls] || (with_dt && !U3[cls])) return fail(c, AF_EINVAL, "stage class %d is NULL", cls);
  CK(cudaSetDevice(c->device), "set device");
  rc = ensure_adjoint(c);
  if (!rc) rc = set_dt(c, dt, dt_on_device);
  if (rc) return rc;
  const int n = c->cur, b1 = (c->cur + 1) % 3, b2 = (c->cur + 2) % 3;
  const size_t blk = (size_t)AF_NCOEF * c->g.nxa * c->g.nya;
  const double *S[4][4];
  buf_cls(c, c->state[n], S[0]);
  if (on_device) {
    for (int cls = 0; cls < 4; ++cls) {
      S[1][cls] = U1[cls];
      S[2][cls] = U2[cls];
      S[3][cls] = with_dt ? U3[cls] : nullptr;
    }
  } else {
    rc = copy_in_buf(c, c->state[b1], U1, 0);
    if (!rc) rc = copy_in_buf(c, c->state[b2], U2, 0);
    if (!rc && with_dt) rc = copy_in_buf(c, abuf(c, 5), U3, 0);
    if (rc) return rc;
    buf_cls(c, c->state[b1], S[1]);
    buf_cls(c, c->state[b2], S[2]);
    buf_cls(c, abuf(c, 5), S[3]);
  }
  for (int set = 0; set < 3; ++set) frozen_pointdata(c, S[set], set, coeffs + set * blk);
  CK(cudaGetLastError(), "point data");
  rc = adjoint_sweep(c, S, lam_in, lam_out, on_device, with_dt, coeffs);
  bind_pd(c, 2);
  bind_states(c, c->cur, c->cur, (c->cur + 1) % 3);
  if (rc) return rc;
  c->next_stage = 0;
  if (!on_device) {
    rc = copy_out_buf(c, abuf(c, 1), lam_out, 0);
    if (rc) return rc;
  }
  CK(cudaStreamSynchronize(c->stream), "synchronise");
  return AF_OK;
}

int af_diagnostics(af_ctx *c, double *out, int on_device) {
  if (!c || !out) return AF_EINVAL;
  AfNvtxRange nvtx_("af_diagnostics");
  CK(cudaSetDevice(c->device), "set device");
  const int nb = af_diag_nblocks(c->g);
  if (!c->diag_buf && cudaMalloc(&c->diag_buf, sizeof(double) * AF_NDIAG * ((size_t)nb + 1)) != cudaSuccess) {
    cudaGetLastError();
    return fail(c, AF_ENOMEM, "diagnostics workspace");
  }
  bind_states(c, c->cur, c->cur, c->cur);
  double *res = c->diag_buf + (size_t)AF_NDIAG * nb;
  af_launch_diag(c->dev, c->g, c->diag_buf, res, c->stream);
  CK(cudaGetLastError(), "diagnostics launch");
  CK(cudaMemcpyAsync(out, res, sizeof(double) * AF_NDIAG, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                     c->stream),
     "copy diagnostics");
  if (!on_device) CK(cudaStreamSynchronize(c->stream), "synchronise");
  return AF_OK;
}

int af_divb(af_ctx *c, double *out, int on_device) {
  AfNvtxRange nvtx_("af_divb");
  if (!c || !out) return AF_EINVAL;
  CK(cudaSetDevice(c->device), "set device");
  const int nb = af_divb_nblocks(c->g);
  if (!c->divb_buf && cudaMalloc(&c->divb_buf, sizeof(double) * (2 * (size_t)nb + 2)) != cudaSuccess) {
    cudaGetLastError();
    return fail(c, AF_ENOMEM, "divergence workspace");
  }
  bind_states(c, c->cur, c->cur, c->cur);
  double *res = c->divb_buf + 2 * (size_t)nb;
  af_launch_divb(c->dev, c->g, c->divb_buf, res, c->stream);
  CK(cudaGetLastError(), "divergence launch");
  CK(cudaMemcpyAsync(out, res, 2 * sizeof(double), on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                     c->stream),
     "copy divergence");
  if (!on_device) CK(cudaStreamSynchronize(c->stream), "synchronise");
  return AF_OK;
}

int af_get_stage(af_ctx *c, double *const U[4], int on_device) {
  if (!c || !U) return AF_EINVAL;
  CK(cudaSetDevice(c->device), "set device");
  return copy_state(c, c->last_out, nullptr, on_device, false, U);
}

int af_step(af_ctx *c, double *dt_used, int on_device) {
  AfNvtxRange nvtx_("af_step");
  if (!c) return AF_EINVAL;
  if (c->next_stage != 0) return fail(c, AF_EINVAL, "af_step called in the middle of a step (stage %d next)", c->next_stage);
  CK(cudaSetDevice(c->device), "set device");
  int rc = stage_impl(c, 0, 1);
  if (!rc) rc = stage_impl(c, 1, 0);
  if (!rc) rc = stage_impl(c, 2, 0);
  if (rc) return rc;
  if (dt_used) {
    CK(cudaMemcpyAsync(dt_used, &c->sc->dt, sizeof(double), on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                       c->stream),
       "copy dt");
    if (!on_device) CK(cudaStreamSynchronize(c->stream), "synchronise");
  }
  return AF_OK;
}

}  // extern "C"

namespace {
int ensure_pipe(af_ctx *c) {
  if (c->pipe_ready) return AF_OK;
  const unsigned fl = cudaEventDisableTiming;
  if (!c->h2d) CK(cudaStreamCreateWithFlags(&c->h2d, cudaStreamNonBlocking), "copy stream");
  if (!c->d2h) CK(cudaStreamCreateWithFlags(&c->d2h, cudaStreamNonBlocking), "copy stream");
  for (int k = 0; k < 2; ++k) {
    if (!c->ev_in[k]) CK(cudaEventCreateWithFlags(&c->ev_in[k], fl), "event");
    if (!c->ev_used[k]) CK(cudaEventCreateWithFlags(&c->ev_used[k], fl), "event");
    if (!c->ev_out[k]) CK(cudaEventCreateWithFlags(&c->ev_out[k], fl), "event");
    if (!c->pipe_in[k] && cudaMalloc(&c->pipe_in[k], c->state_len * sizeof(double)) != cudaSuccess) {
      cudaGetLastError();
      return fail(c, AF_ENOMEM, "staging state for af_step_host");
    }
    if (!c->pipe_out[k] && cudaMalloc(&c->pipe_out[k], c->state_len * sizeof(double)) != cudaSuccess) {
      cudaGetLastError();
      return fail(c, AF_ENOMEM, "staging state for af_step_host");
    }
  }
  for (int cls = 0; cls < 4; ++cls) c->recent_len[cls] = cls_len(c, cls) * sizeof(double);
  c->pipe_ready = 1;
  return AF_OK;
}

// Does one of the host arrays in[] overlap an output array of the last three calls?
bool reads_recent_output(const af_ctx *c, const double *const in[4]) {
  for (int a = 0; a < 4; ++a) {
    const char *lo = (const char *)in[a], *hi = lo + c->recent_len[a];
    for (int r = 0; r < 3; ++r)
      for (int b = 0; b < 4; ++b) {
        const char *olo = c->recent_out[r][b];
        if (olo && lo < olo + c->recent_len[b] && olo < hi) return true;
      }
  }
  return false;
}

int sync_copies(af_ctx *c) {
  if (c->h2d) CK(cudaStreamSynchronize(c->h2d), "synchronise copy stream");
  if (c->d2h) CK(cudaStreamSynchronize(c->d2h), "synchronise copy stream");
  return AF_OK;
}
}  // namespace

extern "C" {

int af_step_host(af_ctx *c, const double *const in[4], double *const out[4]) {
  AfNvtxRange nvtx_("af_step_host");
  if (!c || !in || !out) return AF_EINVAL;
  for (int cls = 0; cls < 4; ++cls)
    if (!in[cls] || !out[cls]) return fail(c, AF_EINVAL, "state class %d is NULL", cls);
  if (c->next_stage != 0) return fail(c, AF_EINVAL, "af_step_host called in the middle of a step (stage %d next)", c->next_stage);
  CK(cudaSetDevice(c->device), "set device");
  int rc = ensure_pipe(c);
  if (rc) return rc;
  const int k = c->pipe_slot;
  // input copy: after the step that last used this slot, and after every
  // earlier output copy if the input is (part of) a recent output
  CK(cudaStreamWaitEvent(c->h2d, c->ev_used[k], 0), "wait");
  if (reads_recent_output(c, in)) CK(cudaStreamWaitEvent(c->h2d, c->ev_out[k ^ 1], 0), "wait");
  for (int cls = 0; cls < 4; ++cls)
    CK(cudaMemcpyAsync(c->pipe_in[k] + c->class_off[cls], in[cls], c->recent_len[cls], cudaMemcpyHostToDevice, c->h2d),
       "copy state in");
  CK(cudaEventRecord(c->ev_in[k], c->h2d), "record");
  // the step: after its input arrived and after the output copy that last read this slot
  CK(cudaStreamWaitEvent(c->stream, c->ev_in[k], 0), "wait");
  CK(cudaStreamWaitEvent(c->stream, c->ev_out[k], 0), "wait");
  double *b1 = c->state[(c->cur + 1) % 3], *b2 = c->state[(c->cur + 2) % 3];
  const double *u = c->pipe_in[k];
  bind_ptrs(c, u, u, b1);
  run_stage(c, RK_A[0], RK_B[0], 1);
  bind_ptrs(c, u, b1, b2);
  run_stage(c, RK_A[1], RK_B[1], 0);
  bind_ptrs(c, u, b2, c->pipe_out[k]);
  run_stage(c, RK_A[2], RK_B[2], 0);
  CK(cudaGetLastError(), "stage launch");
  CK(cudaEventRecord(c->ev_used[k], c->stream), "record");
  // output copy
  CK(cudaStreamWaitEvent(c->d2h, c->ev_used[k], 0), "wait");
  for (int cls = 0; cls < 4; ++cls)
    CK(cudaMemcpyAsync(out[cls], c->pipe_out[k] + c->class_off[cls], c->recent_len[cls], cudaMemcpyDeviceToHost, c->d2h),
       "copy state out");
  CK(cudaEventRecord(c->ev_out[k], c->d2h), "record");
  for (int r = 2; r > 0; --r)
    for (int cls = 0; cls < 4; ++cls) c->recent_out[r][cls] = c->recent_out[r - 1][cls];
  for (int cls = 0; cls < 4; ++cls) c->recent_out[0][cls] = (const char *)out[cls];
  c->pipe_slot = k ^ 1;
  c->last_out = c->cur;
  return AF_OK;
}

int af_sync(af_ctx *c) {
  if (!c) return AF_EINVAL;
  CK(cudaSetDevice(c->device), "set device");
  CK(cudaStreamSynchronize(c->stream), "synchronise");
  return sync_copies(c);
}

int af_status(af_ctx *c, long long *counters, int reset) {
  if (!c) return AF_EINVAL;
  CK(cudaSetDevice(c->device), "set device");
  CK(cudaStreamSynchronize(c->stream), "synchronise");
  {
    const int rc = sync_copies(c);
    if (rc) return rc;
  }
  AfStatus h;
  CK(cudaMemcpy(&h, c->st, offsetof(AfStatus, repair), cudaMemcpyDeviceToHost), "read status");
  if (counters)
    for (int k = 0; k < AF_NSTAT; ++k) counters[k] = (long long)h.cnt[k];
  if (reset) CK(cudaMemset(c->st, 0, sizeof(AfStatus)), "reset status");
  if (h.err & AFE_REPAIR_OVERFLOW) return fail(c, AF_EBOUNDS, "round-off repair list overflowed (%d cells)", AF_MAX_REPAIR);
  if (h.err & (AFE_NONADMISSIBLE | AFE_NONFINITE_DT))
    return fail(c, AF_ENONPHYS, "%s", (h.err & AFE_NONFINITE_DT) ? "time step not finite/positive" : "non-admissible state");
  return AF_OK;
}

int af_timing(af_ctx *c, int enable, double *ms, long long *launches) {
  if (!c) return AF_EINVAL;
  CK(cudaSetDevice(c->device), "set device");
  if (enable) {
    c->tm.nev = 0;
    c->tm.on = 1;
    return AF_OK;
  }
  c->tm.on = 0;
  CK(cudaStreamSynchronize(c->stream), "synchronise");
  CK(c->tm.collect(AF_NKERNEL, ms, launches), "event time");
  return AF_OK;
}

const char *af_last_error(const af_ctx *c) { return c ? c->msg : "null context"; }

void af_destroy(af_ctx *c) {
  if (!c) return;
  cudaSetDevice(c->device);
  if (c->h2d) cudaStreamSynchronize(c->h2d);
  if (c->d2h) cudaStreamSynchronize(c->d2h);
  for (int b = 0; b < 3; ++b)
    if (c->state[b]) cudaFree(c->state[b]);
  if (c->work) cudaFree(c->work);
  if (c->sc) cudaFree(c->sc);
  if (c->st) cudaFree(c->st);
  if (c->adj) cudaFree(c->adj);
  if (c->adj_pd) cudaFree(c->adj_pd);
  if (c->dts) cudaFree(c->dts);
  if (c->divb_buf) cudaFree(c->divb_buf);
  if (c->diag_buf) cudaFree(c->diag_buf);
  if (c->inflow_dev) cudaFree(c->inflow_dev);
  if (c->cnt_pin) cudaFreeHost(c->cnt_pin);
  if (c->abuf) cudaFree(c->abuf);
  if (c->vscale) cudaFree(c->vscale);
  for (int k = 0; k < 2; ++k) {
    if (c->pipe_in[k]) cudaFree(c->pipe_in[k]);
    if (c->pipe_out[k]) cudaFree(c->pipe_out[k]);
    if (c->ev_in[k]) cudaEventDestroy(c->ev_in[k]);
    if (c->ev_used[k]) cudaEventDestroy(c->ev_used[k]);
    if (c->ev_out[k]) cudaEventDestroy(c->ev_out[k]);
  }
  if (c->h2d) cudaStreamDestroy(c->h2d);
  if (c->d2h) cudaStreamDestroy(c->d2h);
  if (c->lstream) {
    cudaStreamSynchronize(c->lstream);
    cudaStreamDestroy(c->lstream);
  }
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  if (c->ev_join) cudaEventDestroy(c->ev_join);
  c->tm.destroy();
  delete c;
}

int af_math_check(int op, const double *x, const double *y, double *out, long long n, void *stream) {
  if (op < 0 || op > 10 || !x || !out || (op != 0 && op != 2 && op != 8 && !y) || n < 0) return AF_EINVAL;
  af_launch_math_check(op, x, y, out, n, (cudaStream_t)stream);
  return cudaGetLastError() == cudaSuccess ? AF_OK : AF_ECUDA;
}

int af_probe_fp64(void *stream, double *tflops) {
  if (!tflops) return AF_EINVAL;
  double f = 0.0;
  const float ms = af_run_fp64_probe((cudaStream_t)stream, &f);
  if (ms <= 0.f || cudaGetLastError() != cudaSuccess) return AF_ECUDA;
  *tflops = f * 1e-12;
  return AF_OK;
}

}  // extern "C"
