// af_batch.cu -- many independent AF runs of uneven grid sizes advanced
// together: every pass of a stage is ONE persistent launch over a (run, tile)
// work list, dt is a per-run (segmented) maximum, a 3-step cycle of the RK
// loop can be captured in a CUDA graph, and the tile shape and the number of
// resident blocks are chosen by a timing autotuner.
//
// Every run computes exactly what a single af_ctx computes (the same device
// functions, the same arithmetic), so batch results are bitwise identical to
// stepping each run on its own.
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/af.h"
#include "af_internal.h"

struct af_batch {
  int device;
  int nruns;
  std::vector<int> nx, ny, bc;
  std::vector<double> gamma, x0, x1, y0, y1;
  std::vector<af_params> prm;
  std::vector<AfGrid> grid;
  std::vector<size_t> state_off, class_len[4], work_off;
  std::vector<size_t> class_off[4];
  double *arena;              // [3 state buffers of all runs][work arrays of all runs]
  size_t state_total;         // doubles of one state buffer (all runs)
  AfScalars *sc;              // per run
  AfStatus *st;               // per run
  AfRun *tables;              // 9 tables (rotation r, stage s) x nruns
  std::vector<AfRun> host_tables;
  bool dirty;                 // host parameters changed since the tables were uploaded
  int cur;                    // rotation: buffer index of U^n (same for all runs)
  cudaStream_t stream;
  // launch configuration
  dim3 block;
  int blocks_per_sm[AF_NKERNEL];
  int sms;
  int4 *items;
  int nitems;
  int items_cap;
  int bps_cap;                // cap on resident blocks per SM chosen by the autotuner (0 = occupancy limit)
  // graph of a 3-step cycle
  cudaGraphExec_t graph;
  int graph_cur;              // rotation at capture time
  int use_graph;
  char msg[512];
};

namespace {

int bfail(af_batch *b, int code, const char *fmt, ...) {
  if (b) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(b->msg, sizeof(b->msg), fmt, ap);
    va_end(ap);
  }
  return code;
}

#define BCK(expr, what)                                                                           \
  do {                                                                                            \
    cudaError_t e_ = (expr);                                                                      \
    if (e_ != cudaSuccess) return bfail(b, AF_ECUDA, "%s: %s", (what), cudaGetErrorString(e_));   \
  } while (0)

void fill_grid(af_batch *b, int r) {
  AfGrid &g = b->grid[r];
  g.nx = b->nx[r];
  g.ny = b->ny[r];
  g.bc = b->bc[r];
  g.nxa = g.bc == AF_BC_OUTFLOW ? g.nx + 1 : g.nx;
  g.nya = g.bc == AF_BC_OUTFLOW ? g.ny + 1 : g.ny;
  g.ex[0] = g.nx;  g.ey[0] = g.ny;
  g.ex[1] = g.nxa; g.ey[1] = g.ny;
  g.ex[2] = g.nx;  g.ey[2] = g.nya;
  g.ex[3] = g.nxa; g.ey[3] = g.nya;
  g.dx = (b->x1[r] - b->x0[r]) / g.nx;
  g.dy = (b->y1[r] - b->y0[r]) / g.ny;
  g.rdx = 1.0 / g.dx;
  g.rdy = 1.0 / g.dy;
  g.gamma = b->gamma[r];
  g.gm1 = b->gamma[r] - 1.0;
  g.kappa = b->prm[r].kappa;
  g.cfl = b->prm[r].cfl;
  g.c13 = 1e-13 / (b->gamma[r] - 1.0);
  g.pp_on = b->prm[r].pp_on;
  g.src_cell_on = b->prm[r].src_cell_on;
  g.src_point_on = b->prm[r].src_point_on;
  g.upwind = b->prm[r].src_point_upwind;
  for (int k = 0; k < 4; ++k) g.side[k] = 0;
  g.special = 0;
  g.x0 = 0.0;
  g.in_lo = g.in_hi = 0.0;
}

double *state_ptr(af_batch *b, int buf, int r, int cls) {
  return b->arena + (size_t)buf * b->state_total + b->state_off[r] + b->class_off[cls][r];
}

// Tables: for rotation rot (U^n in buffer rot) and stage s, the (U^n, U^(s), out) buffers.
void build_tables(af_batch *b) {
  b->host_tables.resize((size_t)9 * b->nruns);
  for (int rot = 0; rot < 3; ++rot)
    for (int s = 0; s < 3; ++s) {
      const int n = rot, b1 = (rot + 1) % 3, b2 = (rot + 2) % 3;
      const int bs = s == 0 ? n : (s == 1 ? b1 : b2);
      const int bo = s == 1 ? b2 : b1;
      for (int r = 0; r < b->nruns; ++r) {
        AfRun &R = b->host_tables[(size_t)(rot * 3 + s) * b->nruns + r];
        R.g = b->grid[r];
        const AfGrid &g = R.g;
        const size_t PS = (size_t)g.nxa * g.nya;
        double *w = b->arena + 3 * b->state_total + b->work_off[r];
        AfDev &d = R.d;
        for (int c = 0; c < 4; ++c) {
          d.un[c] = state_ptr(b, n, r, c);
          d.us[c] = state_ptr(b, bs, r, c);
          d.uo[c] = state_ptr(b, bo, r, c);
        }
        d.pd[0] = w; w += AF_NQA * PS;
        for (int k = 1; k <= 4; ++k) { d.pd[k] = w; w += AF_NQP * PS; }
        d.uc = w; w += 8 * PS;
        d.phi = w; w += 4 * PS;
        d.fx = w; w += AF_NQF * PS;
        d.fy = w; w += AF_NQF * PS;
        d.lam = w; w += 4 * PS;
        d.lim1 = w; w += 8 * PS;
        d.thx = w; w += PS;
        d.thy = w; w += PS;
        d.sc = b->sc + r;
        d.st = b->st + r;
      }
    }
}

int upload(af_batch *b) {
  if (!b->dirty) return AF_OK;
  for (int r = 0; r < b->nruns; ++r) fill_grid(b, r);
  build_tables(b);
  BCK(cudaMemcpyAsync(b->tables, b->host_tables.data(), sizeof(AfRun) * b->host_tables.size(), cudaMemcpyHostToDevice,
                      b->stream),
      "upload run tables");
  BCK(cudaStreamSynchronize(b->stream), "synchronise");
  b->dirty = false;
  return AF_OK;
}

int build_items(af_batch *b, dim3 block) {
  std::vector<int4> items;
  for (int r = 0; r < b->nruns; ++r) {
    const int nxa = b->grid[r].nxa, nya = b->grid[r].nya;
    for (int j0 = 0; j0 < nya; j0 += (int)block.y)
      for (int i0 = 0; i0 < nxa; i0 += (int)block.x) items.push_back(make_int4(r, i0, j0, 0));
  }
  if ((int)items.size() > b->items_cap) {
    if (b->items) cudaFree(b->items);
    b->items = nullptr;
    BCK(cudaMalloc(&b->items, sizeof(int4) * items.size()), "allocate work list");
    b->items_cap = (int)items.size();
  }
  BCK(cudaMemcpyAsync(b->items, items.data(), sizeof(int4) * items.size(), cudaMemcpyHostToDevice, b->stream),
      "upload work list");
  BCK(cudaStreamSynchronize(b->stream), "synchronise");
  b->nitems = (int)items.size();
  b->block = block;
  for (int p = 0; p < AF_NKERNEL; ++p) b->blocks_per_sm[p] = af_batch_occupancy(p, block);
  return AF_OK;
}

const double RK_A[3] = {0.0, 3.0 / 4.0, 1.0 / 3.0};
const double RK_B[3] = {1.0, 1.0 / 4.0, 2.0 / 3.0};

void launch_pass(af_batch *b, int pass, const AfRun *tab, double a, double bb, int reduce_dt, int bps_cap) {
  int bps = b->blocks_per_sm[pass];
  if (bps_cap > 0 && bps > bps_cap) bps = bps_cap;
  int nblocks = b->sms * bps;
  if (nblocks > b->nitems) nblocks = b->nitems;
  af_launch_batch(pass, tab, b->nruns, b->items, b->nitems, b->block, nblocks, a, bb, reduce_dt, b->stream);
}

// Does a run use the velocity-upwind point source (its own point-pass kernel)?
int any_upwind(const af_batch *b) {
  for (const af_params &p : b->prm)
    if (p.src_point_upwind) return 1;
  return 0;
}

// One stage of every run (rotation b->cur).
void batch_stage(af_batch *b, int s, int with_dt, int bps_cap) {
  const AfRun *tab = b->tables + (size_t)(b->cur * 3 + s) * b->nruns;
  launch_pass(b, AF_K_POINTDATA, tab, 0, 0, with_dt, bps_cap);
  if (with_dt) af_launch_batch(AF_K_DT, tab, b->nruns, b->items, b->nitems, b->block, 1, 0, 0, 0, b->stream);
  launch_pass(b, AF_K_POINTS, tab, RK_A[s], RK_B[s], any_upwind(b), bps_cap);
  launch_pass(b, AF_K_FACES, tab, RK_A[s], RK_B[s], 0, bps_cap);
  launch_pass(b, AF_K_CELLS, tab, RK_A[s], RK_B[s], 0, bps_cap);
  launch_pass(b, AF_K_FINAL, tab, RK_A[s], RK_B[s], 0, bps_cap);
  af_launch_batch(AF_K_REPAIR, tab, b->nruns, b->items, b->nitems, b->block, 1, RK_A[s], RK_B[s], 0, b->stream);
}

void batch_step_direct(af_batch *b, int bps_cap) {
  batch_stage(b, 0, 1, bps_cap);
  batch_stage(b, 1, 0, bps_cap);
  batch_stage(b, 2, 0, bps_cap);
  b->cur = (b->cur + 1) % 3;
}

void drop_graph(af_batch *b) {
  if (b->graph) cudaGraphExecDestroy(b->graph);
  b->graph = nullptr;
}

}  // namespace

extern "C" {

int af_batch_create(int nruns, const int *nx, const int *ny, const double *gamma, const int *bc, af_batch **out) {
  if (!out || nruns <= 0 || !nx || !ny || !gamma || !bc) return AF_EINVAL;
  *out = nullptr;
  for (int r = 0; r < nruns; ++r)
    if (!af_grid_fits(nx[r], ny[r]) || !(gamma[r] > 1.0) || (bc[r] != AF_BC_PERIODIC && bc[r] != AF_BC_OUTFLOW))
      return AF_EINVAL;
  af_batch *b = new (std::nothrow) af_batch();
  if (!b) return AF_ENOMEM;
  if (cudaGetDevice(&b->device) != cudaSuccess) {
    delete b;
    return AF_ECUDA;
  }
  cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, b->device);
  b->nruns = nruns;
  b->nx.assign(nx, nx + nruns);
  b->ny.assign(ny, ny + nruns);
  b->bc.assign(bc, bc + nruns);
  b->gamma.assign(gamma, gamma + nruns);
  b->x0.assign(nruns, 0.0); b->x1.assign(nruns, 1.0);
  b->y0.assign(nruns, 0.0); b->y1.assign(nruns, 1.0);
  af_params p0 = {0.2, 0.0, 1, 1, 1, 0};
  b->prm.assign(nruns, p0);
  b->grid.resize(nruns);
  for (int c = 0; c < 4; ++c) b->class_off[c].resize(nruns);
  b->state_off.resize(nruns);
  b->work_off.resize(nruns);
  size_t st = 0, wk = 0;
  const size_t per_point = AF_NQA + 4 * AF_NQP + 8 + 4 + 2 * AF_NQF + 4 + 8 + 2;
  for (int r = 0; r < nruns; ++r) {
    fill_grid(b, r);
    const AfGrid &g = b->grid[r];
    b->state_off[r] = st;
    size_t off = 0;
    for (int c = 0; c < 4; ++c) {
      b->class_off[c][r] = off;
      off += (size_t)8 * g.ex[c] * g.ey[c];
    }
    st += (off + 31) / 32 * 32;   // keep every run 256-byte aligned
    b->work_off[r] = wk;
    wk += ((size_t)g.nxa * g.nya * per_point + 31) / 32 * 32;
  }
  b->state_total = st;
  int rc = AF_OK;
  if (cudaMalloc(&b->arena, (3 * st + wk) * sizeof(double)) != cudaSuccess) rc = AF_ENOMEM;
  if (!rc && cudaMemset(b->arena, 0, (3 * st + wk) * sizeof(double)) != cudaSuccess) rc = AF_ECUDA;
  if (!rc && cudaMalloc(&b->sc, sizeof(AfScalars) * nruns) != cudaSuccess) rc = AF_ENOMEM;
  if (!rc && cudaMalloc(&b->st, sizeof(AfStatus) * nruns) != cudaSuccess) rc = AF_ENOMEM;
  if (!rc && cudaMalloc(&b->tables, sizeof(AfRun) * 9 * nruns) != cudaSuccess) rc = AF_ENOMEM;
  if (!rc && cudaMemset(b->sc, 0, sizeof(AfScalars) * nruns) != cudaSuccess) rc = AF_ECUDA;
  if (!rc && cudaMemset(b->st, 0, sizeof(AfStatus) * nruns) != cudaSuccess) rc = AF_ECUDA;
  if (!rc && cudaDeviceSynchronize() != cudaSuccess) rc = AF_ECUDA;
  b->dirty = true;
  if (!rc) rc = upload(b);
  if (!rc) rc = build_items(b, dim3(32, 4));
  if (rc) {
    cudaGetLastError();
    af_batch_destroy(b);
    return rc;
  }
  *out = b;
  return AF_OK;
}

int af_batch_set_domain(af_batch *b, int run, double x0, double x1, double y0, double y1) {
  if (!b || run < 0 || run >= b->nruns) return AF_EINVAL;
  if (!(x1 > x0) || !(y1 > y0)) return bfail(b, AF_EINVAL, "empty domain");
  b->x0[run] = x0; b->x1[run] = x1; b->y0[run] = y0; b->y1[run] = y1;
  b->dirty = true;
  drop_graph(b);
  return AF_OK;
}

int af_batch_set_params(af_batch *b, int run, const af_params *p) {
  if (!b || !p || run < 0 || run >= b->nruns) return AF_EINVAL;
  if (!(p->cfl > 0.0) || !(p->kappa >= 0.0)) return bfail(b, AF_EINVAL, "cfl must be > 0 and kappa >= 0");
  b->prm[run] = *p;
  b->dirty = true;
  drop_graph(b);
  return AF_OK;
}

int af_batch_set_stream(af_batch *b, void *stream) {
  if (!b) return AF_EINVAL;
  b->stream = (cudaStream_t)stream;
  drop_graph(b);
  return AF_OK;
}

int af_batch_set_state(af_batch *b, int run, const double *const U[4], int on_device) {
  if (!b || !U || run < 0 || run >= b->nruns) return AF_EINVAL;
  BCK(cudaSetDevice(b->device), "set device");
  const AfGrid &g = b->grid[run];
  for (int c = 0; c < 4; ++c) {
    if (!U[c]) return bfail(b, AF_EINVAL, "state class %d is NULL", c);
    BCK(cudaMemcpyAsync(state_ptr(b, b->cur, run, c), U[c], sizeof(double) * 8 * g.ex[c] * g.ey[c],
                        on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, b->stream),
        "copy state in");
  }
  if (!on_device) BCK(cudaStreamSynchronize(b->stream), "synchronise");
  return AF_OK;
}

int af_batch_get_state(af_batch *b, int run, double *const U[4], int on_device) {
  if (!b || !U || run < 0 || run >= b->nruns) return AF_EINVAL;
  BCK(cudaSetDevice(b->device), "set device");
  const AfGrid &g = b->grid[run];
  for (int c = 0; c < 4; ++c) {
    if (!U[c]) return bfail(b, AF_EINVAL, "state class %d is NULL", c);
    BCK(cudaMemcpyAsync(U[c], state_ptr(b, b->cur, run, c), sizeof(double) * 8 * g.ex[c] * g.ey[c],
                        on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, b->stream),
        "copy state out");
  }
  if (!on_device) BCK(cudaStreamSynchronize(b->stream), "synchronise");
  return AF_OK;
}

int af_batch_step(af_batch *b, int nsteps) {
  AfNvtxRange nvtx_("af_batch_step");
  if (!b || nsteps < 0) return AF_EINVAL;
  BCK(cudaSetDevice(b->device), "set device");
  int rc = upload(b);
  if (rc) return rc;
  int left = nsteps;
  while (left > 0) {
    if (b->use_graph && b->graph && b->cur == b->graph_cur && left >= 3) {
      BCK(cudaGraphLaunch(b->graph, b->stream), "graph launch");
      left -= 3;   // the captured cycle leaves the rotation where it started
      continue;
    }
    batch_step_direct(b, b->bps_cap);
    --left;
  }
  BCK(cudaGetLastError(), "batch step launch");
  return AF_OK;
}

int af_batch_graph(af_batch *b, int enable) {
  if (!b) return AF_EINVAL;
  BCK(cudaSetDevice(b->device), "set device");
  drop_graph(b);
  b->use_graph = 0;
  if (!enable) return AF_OK;
  int rc = upload(b);
  if (rc) return rc;
  if (!b->stream) return bfail(b, AF_EINVAL, "graph capture needs a non-default stream (af_batch_set_stream)");
  const int cur0 = b->cur;
  cudaGraph_t graph = nullptr;
  BCK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal), "begin capture");
  for (int k = 0; k < 3; ++k) batch_step_direct(b, b->bps_cap);
  cudaError_t e = cudaStreamEndCapture(b->stream, &graph);
  b->cur = cur0;   // capture does not execute: the rotation is unchanged
  if (e != cudaSuccess) return bfail(b, AF_ECUDA, "end capture: %s", cudaGetErrorString(e));
  e = cudaGraphInstantiate(&b->graph, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    b->graph = nullptr;
    return bfail(b, AF_ECUDA, "instantiate graph: %s", cudaGetErrorString(e));
  }
  b->graph_cur = cur0;
  b->use_graph = 1;
  return AF_OK;
}

// Autotuner: for each tile shape (threads per tile) and cap on resident blocks
// per SM, time `reps` repetitions of stage 0 (which reads only U^n, so the
// state does not move) and keep the fastest.  choice (may be NULL) receives
// {tile x, tile y, blocks-per-SM cap, best time in microseconds}.
int af_batch_autotune(af_batch *b, int reps, int *choice) {
  if (!b || reps < 1) return AF_EINVAL;
  BCK(cudaSetDevice(b->device), "set device");
  int rc = upload(b);
  if (rc) return rc;
  drop_graph(b);
  const dim3 shapes[] = {dim3(32, 4), dim3(32, 8), dim3(64, 2), dim3(16, 8), dim3(64, 4), dim3(128, 1)};
  const int caps[] = {0, 1, 2, 4};
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  dim3 best_shape = b->block;
  int best_cap = 0;
  for (const dim3 &sh : shapes) {
    rc = build_items(b, sh);
    if (rc) break;
    for (int cap : caps) {
      batch_stage(b, 0, 1, cap);   // warm-up
      cudaEventRecord(e0, b->stream);
      for (int k = 0; k < reps; ++k) batch_stage(b, 0, 1, cap);
      cudaEventRecord(e1, b->stream);
      if (cudaEventSynchronize(e1) != cudaSuccess) {
        rc = bfail(b, AF_ECUDA, "autotune timing failed");
        break;
      }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best) {
        best = ms;
        best_shape = sh;
        best_cap = cap;
      }
    }
    if (rc) break;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  rc = build_items(b, best_shape);
  if (rc) return rc;
  b->bps_cap = best_cap;
  if (choice) {
    choice[0] = (int)best_shape.x;
    choice[1] = (int)best_shape.y;
    choice[2] = best_cap;
    choice[3] = (int)(1e3f * best / reps);
  }
  BCK(cudaGetLastError(), "autotune");
  return AF_OK;
}

int af_batch_dt(af_batch *b, int run, double *dt) {
  if (!b || !dt || run < 0 || run >= b->nruns) return AF_EINVAL;
  BCK(cudaSetDevice(b->device), "set device");
  BCK(cudaMemcpyAsync(dt, &b->sc[run].dt, sizeof(double), cudaMemcpyDeviceToHost, b->stream), "copy dt");
  BCK(cudaStreamSynchronize(b->stream), "synchronise");
  return AF_OK;
}

int af_batch_status(af_batch *b, long long *counters, int reset) {
  if (!b) return AF_EINVAL;
  BCK(cudaSetDevice(b->device), "set device");
  BCK(cudaStreamSynchronize(b->stream), "synchronise");
  long long acc[AF_NSTAT] = {0};
  int err = 0;
  std::vector<AfStatus> h(1);
  for (int r = 0; r < b->nruns; ++r) {
    BCK(cudaMemcpy(h.data(), b->st + r, offsetof(AfStatus, repair), cudaMemcpyDeviceToHost), "read status");
    for (int k = 0; k < AF_NSTAT; ++k)
      acc[k] = (k == AF_STAT_NEWTON_MAXIT) ? (acc[k] > (long long)h[0].cnt[k] ? acc[k] : (long long)h[0].cnt[k])
                                           : acc[k] + (long long)h[0].cnt[k];
    err |= h[0].err;
  }
  if (counters)
    for (int k = 0; k < AF_NSTAT; ++k) counters[k] = acc[k];
  if (reset) BCK(cudaMemset(b->st, 0, sizeof(AfStatus) * b->nruns), "reset status");
  if (err & AFE_REPAIR_OVERFLOW) return bfail(b, AF_EBOUNDS, "round-off repair list overflowed");
  if (err & (AFE_NONADMISSIBLE | AFE_NONFINITE_DT)) return bfail(b, AF_ENONPHYS, "non-admissible state or dt");
  return AF_OK;
}

const char *af_batch_last_error(const af_batch *b) { return b ? b->msg : "null batch"; }

void af_batch_destroy(af_batch *b) {
  if (!b) return;
  cudaSetDevice(b->device);
  drop_graph(b);
  if (b->arena) cudaFree(b->arena);
  if (b->sc) cudaFree(b->sc);
  if (b->st) cudaFree(b->st);
  if (b->tables) cudaFree(b->tables);
  if (b->items) cudaFree(b->items);
  delete b;
}

}  // extern "C"
