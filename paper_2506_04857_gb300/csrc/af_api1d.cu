// af_api1d.cu -- host side of the 1D scheme (af1d_*): context, device memory,
// stage sequencing.  The kernels (af_kernels1d.cuh) run on the 2D data
// structures with one row.
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>

#include "../../include/af.h"
#include "af_internal.h"

struct af1d_ctx {
  int device;
  int n, nf, bc;
  double gamma, x0, x1;
  af_params prm;
  cudaStream_t stream;
  AfGrid g;
  double *state[3];   // three state buffers: averages [8][n], then point values [8][nf]
  size_t off1;        // offset of the point values in a state buffer
  size_t state_len;
  int cur, next_stage, last_out;
  double *work;
  AfScalars *sc;
  AfStatus *st;
  AfDev dev;
  AfEventTimer tm;    // per-kernel event timing (af1d_timing)
  char msg[512];
};

namespace {

int fail1(af1d_ctx *c, int code, const char *fmt, ...) {
  if (c) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(c->msg, sizeof(c->msg), fmt, ap);
    va_end(ap);
  }
  return code;
}

#define CK1(expr, what)                                                                    \
  do {                                                                                     \
    cudaError_t e_ = (expr);                                                               \
    if (e_ != cudaSuccess) return fail1(c, AF_ECUDA, "%s: %s", (what), cudaGetErrorString(e_)); \
  } while (0)

void refresh1(af1d_ctx *c) {
  AfGrid &g = c->g;
  memset(&g, 0, sizeof(g));
  g.nx = c->n;
  g.ny = 1;
  g.bc = c->bc;
  g.nxa = c->nf;
  g.nya = 1;
  g.ex[0] = c->n;  g.ey[0] = 1;
  g.ex[1] = c->nf; g.ey[1] = 1;
  g.ex[2] = c->n;  g.ey[2] = 1;
  g.ex[3] = c->nf; g.ey[3] = 1;
  g.dx = (c->x1 - c->x0) / c->n;
  g.dy = 1.0;
  g.rdx = 1.0 / g.dx;
  g.rdy = 1.0;
  g.gamma = c->gamma;
  g.gm1 = c->gamma - 1.0;
  g.kappa = c->prm.kappa;
  g.cfl = c->prm.cfl;
  g.c13 = 1e-13 / (c->gamma - 1.0);
  g.pp_on = c->prm.pp_on;
  g.src_cell_on = 0;   // 1D: no source (B1 is constant)
  g.src_point_on = 0;
  g.upwind = 0;
}

void bind1(af1d_ctx *c, int bn, int bs, int bo) {
  const int b[3] = {bn, bs, bo};
  const double **un = c->dev.un, **us = c->dev.us;
  for (int q = 0; q < 2; ++q) {
    const size_t off = q ? c->off1 : 0;
    un[q] = c->state[b[0]] + off;
    us[q] = c->state[b[1]] + off;
    c->dev.uo[q] = c->state[b[2]] + off;
  }
}

int copy1(af1d_ctx *c, int buf, const double *const *Uin, double *const *Uout, int on_device) {
  const size_t len[2] = {(size_t)8 * c->n, (size_t)8 * c->nf};
  for (int q = 0; q < 2; ++q) {
    const size_t off = q ? c->off1 : 0, bytes = len[q] * sizeof(double);
    if (Uin) {
      if (!Uin[q]) return fail1(c, AF_EINVAL, "array %d is NULL", q);
      CK1(cudaMemcpyAsync(c->state[buf] + off, Uin[q], bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                          c->stream), "copy state in");
    } else {
      if (!Uout[q]) return fail1(c, AF_EINVAL, "array %d is NULL", q);
      CK1(cudaMemcpyAsync(Uout[q], c->state[buf] + off, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                          c->stream), "copy state out");
    }
  }
  if (!on_device) CK1(cudaStreamSynchronize(c->stream), "synchronise");
  return AF_OK;
}

int set_dt1(af1d_ctx *c, const double *dt, int on_device) {
  if (!dt) return AF_OK;
  if (!on_device && !(*dt > 0.0)) return fail1(c, AF_EINVAL, "dt must be positive");
  CK1(cudaMemcpyAsync(&c->sc->dt, dt, sizeof(double), on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                      c->stream), "set dt");
  if (!on_device) CK1(cudaStreamSynchronize(c->stream), "synchronise");
  return AF_OK;
}

const double RK1_A[3] = {0.0, 3.0 / 4.0, 1.0 / 3.0};
const double RK1_B[3] = {1.0, 1.0 / 4.0, 2.0 / 3.0};

int stage1(af1d_ctx *c, int s, int reduce_dt) {
  const int n = c->cur, b1 = (c->cur + 1) % 3, b2 = (c->cur + 2) % 3;
  if (s == 0) bind1(c, n, n, b1);
  else if (s == 1) bind1(c, n, b1, b2);
  else bind1(c, n, b2, b1);
  af_launch_stage1d(c->dev, c->g, RK1_A[s], RK1_B[s], reduce_dt, c->stream, &c->tm);
  CK1(cudaGetLastError(), "stage launch");
  c->last_out = s == 1 ? b2 : b1;
  if (s == 2) c->cur = b1;
  c->next_stage = (s + 1) % 3;
  return AF_OK;
}

}  // namespace

extern "C" {

int af1d_create(int n, double gamma, int bc, af1d_ctx **out) {
  if (!out) return AF_EINVAL;
  *out = nullptr;
  if (n < 4 || !(gamma > 1.0) || (bc != AF_BC_PERIODIC && bc != AF_BC_OUTFLOW)) return AF_EINVAL;
  af1d_ctx *c = new (std::nothrow) af1d_ctx();
  if (!c) return AF_ENOMEM;
  c->n = n;
  c->nf = bc == AF_BC_OUTFLOW ? n + 1 : n;
  c->bc = bc;
  c->gamma = gamma;
  c->x0 = 0.0;
  c->x1 = 1.0;
  c->prm.cfl = 0.2;
  c->prm.kappa = 0.0;
  c->prm.pp_on = 1;
  c->prm.src_cell_on = 0;
  c->prm.src_point_on = 0;
  if (cudaGetDevice(&c->device) != cudaSuccess) {
    delete c;
    return AF_ECUDA;
  }
  refresh1(c);
  c->off1 = (size_t)8 * n;
  c->state_len = c->off1 + (size_t)8 * c->nf;
  const size_t PS = (size_t)c->nf;
  const size_t nwork = PS * (AF_NQA + 2 * AF_NQP + 8 + 4 + AF_NQF + 4 + 8 + 1);
  int rc = AF_OK;
  for (int b = 0; b < 3 && !rc; ++b)
    if (cudaMalloc(&c->state[b], c->state_len * sizeof(double)) != cudaSuccess ||
        cudaMemset(c->state[b], 0, c->state_len * sizeof(double)) != cudaSuccess)
      rc = AF_ENOMEM;
  if (!rc && (cudaMalloc(&c->work, nwork * sizeof(double)) != cudaSuccess ||
              cudaMemset(c->work, 0, nwork * sizeof(double)) != cudaSuccess))
    rc = AF_ENOMEM;
  if (!rc && (cudaMalloc(&c->sc, sizeof(AfScalars)) != cudaSuccess || cudaMalloc(&c->st, sizeof(AfStatus)) != cudaSuccess))
    rc = AF_ENOMEM;
  if (!rc && (cudaMemset(c->sc, 0, sizeof(AfScalars)) != cudaSuccess || cudaMemset(c->st, 0, sizeof(AfStatus)) != cudaSuccess ||
              cudaDeviceSynchronize() != cudaSuccess))
    rc = AF_ECUDA;
  if (rc) {
    cudaGetLastError();
    af1d_destroy(c);
    return rc;
  }
  double *w = c->work;
  memset(&c->dev, 0, sizeof(c->dev));
  c->dev.pd[0] = w; w += AF_NQA * PS;
  c->dev.pd[1] = w; w += AF_NQP * PS;
  c->dev.pd[4] = w; w += AF_NQP * PS;
  c->dev.uc = w; w += 8 * PS;
  c->dev.phi = w; w += 4 * PS;
  c->dev.fx = w; w += AF_NQF * PS;
  c->dev.lam = w; w += 4 * PS;
  c->dev.lim1 = w; w += 8 * PS;
  c->dev.thx = w; w += PS;
  c->dev.sc = c->sc;
  c->dev.st = c->st;
  c->cur = 0;
  c->next_stage = 0;
  *out = c;
  return AF_OK;
}

int af1d_set_domain(af1d_ctx *c, double x0, double x1) {
  if (!c) return AF_EINVAL;
  if (!(x1 > x0)) return fail1(c, AF_EINVAL, "empty domain");
  c->x0 = x0;
  c->x1 = x1;
  refresh1(c);
  return AF_OK;
}

int af1d_set_params(af1d_ctx *c, const af_params *p) {
  if (!c || !p) return AF_EINVAL;
  if (!(p->cfl > 0.0) || !(p->kappa >= 0.0)) return fail1(c, AF_EINVAL, "cfl must be > 0 and kappa >= 0");
  c->prm = *p;
  refresh1(c);
  return AF_OK;
}

int af1d_set_stream(af1d_ctx *c, void *stream) {
  if (!c) return AF_EINVAL;
  c->stream = (cudaStream_t)stream;
  return AF_OK;
}

int af1d_sizes(const af1d_ctx *c, int cls, int *len) {
  if (!c || !len || cls < 0 || cls > 1) return AF_EINVAL;
  *len = cls == 0 ? c->n : c->nf;
  return AF_OK;
}

int af1d_set_state(af1d_ctx *c, const double *const U[2], int on_device) {
  if (!c || !U) return AF_EINVAL;
  CK1(cudaSetDevice(c->device), "set device");
  c->next_stage = 0;
  return copy1(c, c->cur, U, nullptr, on_device);
}

int af1d_get_state(af1d_ctx *c, double *const U[2], int on_device) {
  if (!c || !U) return AF_EINVAL;
  CK1(cudaSetDevice(c->device), "set device");
  return copy1(c, c->cur, nullptr, U, on_device);
}

int af1d_get_stage(af1d_ctx *c, double *const U[2], int on_device) {
  if (!c || !U) return AF_EINVAL;
  CK1(cudaSetDevice(c->device), "set device");
  return copy1(c, c->last_out, nullptr, U, on_device);
}

int af1d_dt(af1d_ctx *c, double *dt_out, int on_device) {
  if (!c) return AF_EINVAL;
  CK1(cudaSetDevice(c->device), "set device");
  bind1(c, c->cur, c->cur, (c->cur + 1) % 3);
  af_launch_dt1d(c->dev, c->g, c->stream);
  CK1(cudaGetLastError(), "dt launch");
  if (dt_out) {
    CK1(cudaMemcpyAsync(dt_out, &c->sc->dt, sizeof(double), on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                        c->stream), "copy dt");
    if (!on_device) CK1(cudaStreamSynchronize(c->stream), "synchronise");
  }
  return AF_OK;
}

int af1d_stage(af1d_ctx *c, int s, const double *dt, int on_device) {
  AfNvtxRange nvtx_("af1d_stage");
  if (!c || s < 0 || s > 2) return AF_EINVAL;
  if (s != c->next_stage) return fail1(c, AF_EINVAL, "stage %d called, stage %d expected", s, c->next_stage);
  CK1(cudaSetDevice(c->device), "set device");
  int rc = set_dt1(c, dt, on_device);
  if (rc) return rc;
  return stage1(c, s, 0);
}

int af1d_step(af1d_ctx *c, double *dt_used, int on_device) {
  AfNvtxRange nvtx_("af1d_step");
  if (!c) return AF_EINVAL;
  if (c->next_stage != 0) return fail1(c, AF_EINVAL, "af1d_step called in the middle of a step");
  CK1(cudaSetDevice(c->device), "set device");
  int rc = stage1(c, 0, 1);
  if (!rc) rc = stage1(c, 1, 0);
  if (!rc) rc = stage1(c, 2, 0);
  if (rc) return rc;
  if (dt_used) {
    CK1(cudaMemcpyAsync(dt_used, &c->sc->dt, sizeof(double), on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                        c->stream), "copy dt");
    if (!on_device) CK1(cudaStreamSynchronize(c->stream), "synchronise");
  }
  return AF_OK;
}

int af1d_status(af1d_ctx *c, long long *counters, int reset) {
  if (!c) return AF_EINVAL;
  CK1(cudaSetDevice(c->device), "set device");
  CK1(cudaStreamSynchronize(c->stream), "synchronise");
  AfStatus h;
  CK1(cudaMemcpy(&h, c->st, offsetof(AfStatus, repair), cudaMemcpyDeviceToHost), "read status");
  if (counters)
    for (int k = 0; k < AF_NSTAT; ++k) counters[k] = (long long)h.cnt[k];
  if (reset) CK1(cudaMemset(c->st, 0, sizeof(AfStatus)), "reset status");
  if (h.err & AFE_REPAIR_OVERFLOW) return fail1(c, AF_EBOUNDS, "round-off repair list overflowed (%d cells)", AF_MAX_REPAIR);
  if (h.err & (AFE_NONADMISSIBLE | AFE_NONFINITE_DT))
    return fail1(c, AF_ENONPHYS, "%s", (h.err & AFE_NONFINITE_DT) ? "time step not finite/positive" : "non-admissible state");
  return AF_OK;
}

const char *af1d_last_error(const af1d_ctx *c) { return c ? c->msg : "null context"; }

int af1d_timing(af1d_ctx *c, int enable, double *ms, long long *launches) {
  if (!c) return AF_EINVAL;
  CK1(cudaSetDevice(c->device), "set device");
  if (enable) {
    c->tm.nev = 0;
    c->tm.on = 1;
    return AF_OK;
  }
  c->tm.on = 0;
  CK1(cudaStreamSynchronize(c->stream), "synchronise");
  CK1(c->tm.collect(AF_NKERNEL, ms, launches), "event time");
  return AF_OK;
}

void af1d_destroy(af1d_ctx *c) {
  if (!c) return;
  cudaSetDevice(c->device);
  for (int b = 0; b < 3; ++b)
    if (c->state[b]) cudaFree(c->state[b]);
  if (c->work) cudaFree(c->work);
  if (c->sc) cudaFree(c->sc);
  if (c->st) cudaFree(c->st);
  c->tm.destroy();
  delete c;
}

}  // extern "C"
