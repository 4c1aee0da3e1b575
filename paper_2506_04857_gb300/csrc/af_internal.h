// af_internal.h -- device-side data structures shared by the kernels and the
// host API of libaf (not part of the public C ABI).
//
// Layout in HBM (all FP64, structure of arrays):
//   state class c (0 average, 1 x-face, 2 y-face, 3 corner): [8][ey[c]][ex[c]]
//   point data of class c and of the cell centres (c = 4): [NQ][nya][nxa]
//   cell-centre values [8][nya][nxa], sensor [4][nya][nxa],
//   face data [NQF][nya][nxa] for x-faces and for y-faces,
//   Lambda [4][nya][nxa], Lim1 [8][nya][nxa], face theta [nya][nxa] (x and y).
// nxa = nx (+1 for outflow), nya = ny (+1 for outflow).
#pragma once
#include <cuda_runtime.h>
#include <cstdlib>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#define AF_NQP 20   // per point value: F1 (7), F2 (7), varrho_1, varrho_2, v (3), v.B
#define AF_NQA 21   // per cell average: F1 (7), F2 (7), c_f1, c_f2, v (3), p_t, sqrt(rho)
#define AF_NQF 18   // per face: F^LLF (8), G = theta^s (F - F^LLF) (8), theta^s, alpha^LLF
#define AF_NSTAT 12
#define AF_MAX_REPAIR 4096

// F1 is stored without its B1 component (identically 0), F2 without B2.
enum { QP_F1 = 0, QP_F2 = 7, QP_SR1 = 14, QP_SR2 = 15, QP_V1 = 16, QP_V2 = 17, QP_V3 = 18, QP_VB = 19 };
enum { QA_F1 = 0, QA_F2 = 7, QA_CF1 = 14, QA_CF2 = 15, QA_V1 = 16, QA_V2 = 17, QA_V3 = 18, QA_PT = 19, QA_SRHO = 20 };
enum { QF_FLLF = 0, QF_G = 8, QF_TS = 16, QF_AL = 17 };

// Limiter coefficients of one stage (af_record_coeffs, af_freeze_coeffs): AF_NCOEF
// arrays [nya][nxa], at the index point of the face, cell or point they belong to.
// Point classes c = 1..3 use AFC_P1 + 2 (c - 1) (theta*) and the slot after it (theta**).
enum { AFC_TSX = 0, AFC_TSY, AFC_THX, AFC_THY, AFC_TSRC, AFC_C1, AFC_C2, AFC_P1 };
#ifndef AF_NCOEF
#define AF_NCOEF 13   // also in af.h
#endif

// counters (same meaning and order as the af_status counters in af.h)
enum {
  ST_SRC_LIMITED = 0, ST_LAMBDA_LT1, ST_FACE_THETA_LT1, ST_SENSOR_LT099, ST_NEWTON_SOLVES, ST_NEWTON_MAXIT,
  ST_SHRINK, ST_POINT_LIMITED, ST_CFL_VIOLATIONS, ST_CENTER_LIMITED, ST_NONADMISSIBLE, ST_CELL_SHRINK
};

// device error bits
enum { AFE_NONADMISSIBLE = 1, AFE_REPAIR_OVERFLOW = 2, AFE_NONFINITE_DT = 4, AFE_LIST_OVERFLOW = 8 };

struct AfGrid {
  int nx, ny, bc;          // cells; 0 periodic, 1 outflow
  int nxa, nya;            // extents of the per-index work arrays
  int ex[4], ey[4];        // extents of the four DoF classes
  double dx, dy;
  double rdx, rdy;         // 1/dx, 1/dy (formed once on the host)
  double gamma, gm1;
  double kappa, cfl;
  double c13;              // 1e-13 / (gamma - 1)
  int pp_on, src_cell_on, src_point_on;
  int upwind;          // velocity-upwind divergence in the point source (Example 4.2 variant)
  // bc = 1: kind of each side (0 left, 1 right, 2 bottom, 3 top): 0 outflow
  // (mirror), 1 reflective (mirror, normal momentum and B negated), 2 inflow
  // (bottom/top: the inflow state where in_lo < x < in_hi, outflow elsewhere)
  int side[4];
  int special;             // some side is reflective or inflow
  double x0, in_lo, in_hi;
};

// Device-resident per-step scalars: dt stays on the device so that a whole
// step can be captured in a CUDA graph.
struct AfScalars {
  double dt;
  unsigned long long smax[2];   // running max of varrho_1, varrho_2 (bit patterns of non-negative doubles)
  int pad[4];
};

struct AfStatus {
  unsigned long long cnt[16];
  int err;
  int nrepair;
  int repair[AF_MAX_REPAIR];
  int npq, ncq;   // entries of the point and cell work lists of the current stage
  int nvq;        // entries of the vertex list (vertices of listed cells that need the Newton solve)
};

struct AfDev {
  const double *un[4];    // U^n
  const double *us[4];    // stage input U^(s)
  double *uo[4];          // stage output
  double *pd[5];          // point data, classes 0..3 and cell centres (4)
  double *uc;             // limited cell-centre values
  double *phi;            // phi_1x, phi_1y, phi_2, phi_3
  double *fx, *fy;        // face data
  double *lam, *lim1;     // Lambda_{L,R,D,U}, U^{Lim,1}
  double *thx, *thy;      // unique face coefficients (read back by the repair pass)
  AfScalars *sc;
  AfStatus *st;
  const double *inflow;   // inflow state [8], its point data as a point [AF_NQP] and as an average [AF_NQA]
  double *rec;            // when set: the stage writes its limiter coefficients here (AFC_* slots)
  const double *frz;      // when set: the stage takes its limiter coefficients from here (frozen branch)
  // work lists of the limiter slow paths (single runs; NULL: slow paths inline, as in batches):
  // points whose update leaves the 1e-13 floors (packed class << 28 | index, and their
  // high-order update, component-major), cells whose Sec. 3.2 box is not certified
  // (index, eps_rho, eps_p)
  int *pq, *cq;
  double *pqu, *cqe;
  int pq_cap, cq_cap;
  // vertices of R_rho (listed cell << 4 | vertex) whose pressure falls below eps_p, and
  // Lambda^rho of each listed cell
  unsigned *vq;
  double *cql;
  int vq_cap;
};

// one member of a batch (af_batch.cu): its work pointers and grid
struct AfRun {
  AfDev d;
  AfGrid g;
};

// kernel launchers (af_kernels.cu)
void af_launch_pointdata(const AfDev &d, const AfGrid &g, int reduce_dt, cudaStream_t s);
void af_launch_dt(const AfDev &d, const AfGrid &g, cudaStream_t s);
void af_launch_points(const AfDev &d, const AfGrid &g, double a, double b, int mode, cudaStream_t s);
void af_launch_faces(const AfDev &d, const AfGrid &g, int mode, cudaStream_t s);
void af_launch_cells(const AfDev &d, const AfGrid &g, double a, double b, int mode, cudaStream_t s);
void af_launch_final(const AfDev &d, const AfGrid &g, double a, double b, cudaStream_t s);
// the limiter slow paths over the work lists the point and cell passes filled
void af_launch_points_slow(const AfDev &d, const AfGrid &g, double a, double b, cudaStream_t s);
void af_launch_cells_slow(const AfDev &d, const AfGrid &g, cudaStream_t s);
void af_launch_repair(const AfDev &d, const AfGrid &g, double a, double b, cudaStream_t s);
float af_run_fp64_probe(cudaStream_t s, double *flops);
// point data of the inflow state U (device, 8 doubles) into out (8 + AF_NQP + AF_NQA doubles)
void af_launch_inflow_pd(const AfGrid &g, const double *U, double *out, cudaStream_t s);
// sensitivity of one step to its dt (af_adjoint.cu), in two launches: the dot
// product mu dt of the reverse-sweep variables with the stage increments
// (before the last VJP, which may overwrite L3), then the maximising DoFs of
// varrho_1, varrho_2 over U^n (point data of U^n bound in d, d.un = U^n) and
// lam += mu d(dt)/dU^n there.  work: 5 * af_dt_sens_nblocks() doubles; mu_out
// (device, may be NULL) receives mu = dJ/d(dt).
int af_dt_sens_nblocks();
void af_launch_dt_dot(const AfGrid &g, const double *const *L3, const double *const *L2, const double *const *L1,
                      const double *const *U0, const double *const *U1, const double *const *U2,
                      const double *const *U3, double *work, cudaStream_t s);
void af_launch_dt_apply(const AfDev &d, const AfGrid &g, double *const *lam, double *work, double *mu_out,
                        cudaStream_t s);
// the 1D scheme (af_kernels1d.cuh) on the 2D structures with ny = 1: one stage
// out = a U^n + b FE(U^s) (the dt pass first when reduce_dt), and the dt pass alone
// A named NVTX range around one library call (visible in nsys timelines; the
// header-only NVTX3 costs nothing when no tool is attached).
struct AfNvtxRange {
  explicit AfNvtxRange(const char *name) { nvtxRangePushA(name); }
  ~AfNvtxRange() { nvtxRangePop(); }
  AfNvtxRange(const AfNvtxRange &) = delete;
  AfNvtxRange &operator=(const AfNvtxRange &) = delete;
};

// Largest grids: the launch shape (32 x 4 thread blocks, at most 65535 block
// rows) bounds ny, and the adjoint's DoF ids (class << 28 | index) bound the
// points of a class.  Either bound lies far beyond what fits in device memory.
inline bool af_grid_fits(int nx, int ny) {
  return nx >= 4 && ny >= 4 && (long long)ny + 1 <= 4LL * 65535 && ((long long)nx + 1) * ((long long)ny + 1) < (1LL << 28);
}

// Per-kernel CUDA-event timing of a context's launches (af_timing, af1d_timing):
// an event pair around every launch while enabled; events are created lazily in
// chunks and kept until destroy().
struct AfEventTimer {
  int on = 0, nev = 0, cap = 0;
  cudaEvent_t *ev = nullptr;      // 2 * cap events
  unsigned char *kid = nullptr;   // kernel id of each pair
  bool begin(int kernel, cudaStream_t s) {
    if (!on) return false;
    if (nev == cap) {
      const int nc = cap ? 2 * cap : 256;
      cudaEvent_t *e = (cudaEvent_t *)realloc(ev, sizeof(cudaEvent_t) * 2 * nc);
      if (e) ev = e;
      unsigned char *k = (unsigned char *)realloc(kid, nc);
      if (k) kid = k;
      if (!e || !k) return false;
      for (int q = 2 * cap; q < 2 * nc; ++q) cudaEventCreate(&ev[q]);
      cap = nc;
    }
    kid[nev] = (unsigned char)kernel;
    cudaEventRecord(ev[2 * nev], s);
    return true;
  }
  void end(bool started, cudaStream_t s) {
    if (!started) return;
    cudaEventRecord(ev[2 * nev + 1], s);
    nev++;
  }
  // Sums per kernel id (nk ids) after the caller synchronised the stream; clears the record.
  cudaError_t collect(int nk, double *ms, long long *launches) {
    for (int k = 0; k < nk; ++k) {
      if (ms) ms[k] = 0.0;
      if (launches) launches[k] = 0;
    }
    for (int p = 0; p < nev; ++p) {
      float t = 0.f;
      const cudaError_t e = cudaEventElapsedTime(&t, ev[2 * p], ev[2 * p + 1]);
      if (e != cudaSuccess) return e;
      if (kid[p] < nk) {
        if (ms) ms[kid[p]] += t;
        if (launches) launches[kid[p]]++;
      }
    }
    nev = 0;
    return cudaSuccess;
  }
  void destroy() {
    for (int q = 0; q < 2 * cap; ++q) cudaEventDestroy(ev[q]);
    free(ev);
    free(kid);
    ev = nullptr;
    kid = nullptr;
    cap = nev = on = 0;
  }
};
// One 1D stage; t (may be NULL) times each launch.
void af_launch_stage1d(const AfDev &d, const AfGrid &g, double a, double b, int reduce_dt, cudaStream_t s,
                       AfEventTimer *t);
void af_launch_dt1d(const AfDev &d, const AfGrid &g, cudaStream_t s);
// divergence measures of Example 4.4 of the state bound in d.us into out[2]
// (device); partials: 2 * af_divb_nblocks(g) doubles
int af_divb_nblocks(const AfGrid &g);
// run diagnostics (af_diagnostics): AF_NDIAG partials per block of af_diag_nblocks(g), then out[AF_NDIAG]
#define AF_NDIAG 9
int af_diag_nblocks(const AfGrid &g);
void af_launch_diag(const AfDev &d, const AfGrid &g, double *partials, double *out, cudaStream_t s);
void af_launch_divb(const AfDev &d, const AfGrid &g, double *partials, double *out, cudaStream_t s);
// persistent batched launch of one pass (AF_K_* id) over a (run, i0, j0) tile
// list; flag: reduce_dt for the point-data pass, "some run uses the upwind
// point source" for the point pass
void af_launch_batch(int pass, const AfRun *runs, int nruns, const int4 *items, int nitems, dim3 block, int nblocks,
                     double a, double b, int flag, cudaStream_t s);
int af_batch_occupancy(int pass, dim3 block);   // resident blocks per SM
// adjoint (af_adjoint.cu).  With T = (dL/dU)^T v at the state bound in d (after
// the point-data pass on it), the last kernel writes
//   out1 = a v + b s T + c z1   and, when out2[0] is not NULL,   out2 = e v + f z2,
// s = *dt (device pointer) or 1 when dt is NULL; every array in state layout
// (four class pointers).  out1 may alias v; nothing else may alias.
struct AfAdjEpi {
  const double *v[4];
  double *out1[4];
  const double *z1[4];
  double *out2[4];
  const double *z2[4];
  double a, b, c, e, f;
  const double *dt;
};
// a: af_adj_nslots() work arrays, zc: 8 work arrays (per index point),
// tpart: a state-sized scratch buffer (four class pointers)
int af_adj_nslots();
// co: one stage's frozen limiter coefficients (NULL: the branch on which every limiter
// is inactive); vscaled: a state-sized scratch (four class pointers) used when co is set
void af_launch_vjp(const AfDev &d, const AfGrid &g, const AfAdjEpi &e, double *a, double *zc, double *const *tpart,
                   cudaStream_t s, const double *co = nullptr, double *const *vscaled = nullptr);
void af_launch_math_check(int op, const double *x, const double *y, double *out, long long n, cudaStream_t s);
