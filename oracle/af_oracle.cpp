// af_oracle.cpp -- CPU FP64 oracle for one SSP-RK3 step of the positivity-
// preserving Active Flux (AF) scheme for 2D ideal MHD with the Godunov-Powell
// source term (Duan, Chandrashekar, Klingenberg, arXiv:2506.04857).
//
// TEST INFRASTRUCTURE ONLY.  This file is the parity oracle: a plain, slow,
// literal transcription of the paper's definitions, in the paper's order and
// notation.  Only the test suite, the smoke check and the benchmark's CPU
// baseline / reference arm load it.  It shares no code, header, table or
// constant with the CUDA path; the product never links or calls it.
//
// Build: g++ -O2 -ffp-contract=off -fopenmp -shared -fPIC (no FMA contraction,
// so every rounding follows the written expression).  With -DAF_ORACLE_COUNT
// the scalar type becomes a counting wrapper and the same source reports the
// number of floating-point operations per phase (single-threaded).
//
// Citations are to sections / equations of the paper.  Where the paper is
// silent or ambiguous the reading taken is marked "Reading:".
//
// Parity unpinned: the values that the positivity limiters (theta, Lambda of
// Sec. 3.2, theta* and theta** of Sec. 3.3) take on shocked data.  The paper
// prints none, so only their invariants are pinned (ranges in [0,1], the
// limited states in the admissible set, Lambda = 1 on smooth data, brute force
// on tiny boxes); the GPU path is compared with this file where both take the
// same branch.
//
// Data layout of every user array: one DoF class is [8][nyp][nxp] doubles,
// conserved variables U = (rho, rho v1, rho v2, rho v3, B1, B2, B3, E), x
// fastest.  Classes: 0 cell average, 1 x-face (vertical face) value, 2 y-face
// (horizontal face) value, 3 corner value.  Indices: cell (i,j) covers
// [x0+i dx, x0+(i+1) dx] x [y0+j dy, ...]; x-face (f,j) sits at (x0+f dx,
// y_j); y-face (i,g) at (x_i, y0+g dy); corner (f,g) at (x0+f dx, y0+g dy).
// Periodic: all classes nx x ny.  Outflow: x-faces (nx+1) x ny, y-faces
// nx x (ny+1), corners (nx+1) x (ny+1).

#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>
#include <algorithm>

// ---------------------------------------------------------------------------
// Scalar type.  double normally; a counting wrapper under AF_ORACLE_COUNT.
// ---------------------------------------------------------------------------
enum Phase {
  PH_DT = 0,        // max wave speed for the time step (A16)
  PH_POINTDATA,     // primitives, fluxes F1 F2, fast speeds per DoF and centre
  PH_CENTER,        // cell-centre reconstruction + its limiter (Remark 3.2)
  PH_POINT_HO,      // LLF-FVS point update (Sec. 2.3)
  PH_POINT_PP,      // first-order LLF point schemes, scaling limiter, round-off check (Sec. 3.3)
  PH_SENSOR_PHI,    // shock sensor phi_1..phi_3 per cell (Sec. 3.4)
  PH_SENSOR_THETA,  // theta^s per face (Sec. 3.4)
  PH_FACE,          // Simpson flux + LLF flux per face (Sec. 2.2, eq. 2d_llf_flux)
  PH_CELL_SRC,      // Powell source S_ij (eq. semi_av_src) and S^LLF
  PH_CELL_UPDATE,   // sensor blend, and with PP on the flux limiter steps (1)-(2) (Sec. 3.2)
  PH_CELL_FINAL,    // step (3) face theta, limited update, round-off check
  PH_RK,            // SSP-RK3 convex combination
  NPHASE
};
enum Kind { K_ADD = 0, K_MUL, K_DIV, K_SQRT, K_EXP, K_MINMAX, K_CMP, NKIND };

#ifdef AF_ORACLE_COUNT
static long long g_cnt[NPHASE][NKIND];
static int g_phase = 0;
static int g_count_on = 1;
static inline void tick(int k) { if (g_count_on) g_cnt[g_phase][k]++; }
struct Counted {
  double v;
  Counted() : v(0) {}
  Counted(double x) : v(x) {}
};
typedef Counted real;
static inline double val(real x) { return x.v; }
static inline real operator+(real a, real b) { tick(K_ADD); return a.v + b.v; }
static inline real operator-(real a, real b) { tick(K_ADD); return a.v - b.v; }
static inline real operator*(real a, real b) { tick(K_MUL); return a.v * b.v; }
static inline real operator/(real a, real b) { tick(K_DIV); return a.v / b.v; }
static inline real operator-(real a) { return -a.v; }
static inline real &operator+=(real &a, real b) { a = a + b; return a; }
static inline real &operator-=(real &a, real b) { a = a - b; return a; }
static inline bool operator<(real a, real b) { tick(K_CMP); return a.v < b.v; }
static inline bool operator>(real a, real b) { tick(K_CMP); return a.v > b.v; }
static inline bool operator<=(real a, real b) { tick(K_CMP); return a.v <= b.v; }
static inline bool operator>=(real a, real b) { tick(K_CMP); return a.v >= b.v; }
static inline real sqrt(real a) { tick(K_SQRT); return std::sqrt(a.v); }
static inline real exp(real a) { tick(K_EXP); return std::exp(a.v); }
static inline real fabs(real a) { tick(K_MINMAX); return std::fabs(a.v); }
static inline bool is_finite(real a) { return std::isfinite(a.v); }
static inline void set_phase(int p) { g_phase = p; }
#elif defined(AF_ORACLE_COMPLEX)
// Complex-step build: a + i b carries the directional derivative b of every
// quantity along the perturbation of the input; branches (comparisons,
// min/max, |.|) follow the real part.
struct Cx {
  double re, im;
  Cx() : re(0), im(0) {}
  Cx(double x) : re(x), im(0) {}
  Cx(double a, double b) : re(a), im(b) {}
};
typedef Cx real;
static inline double val(real x) { return x.re; }
static inline real operator+(real a, real b) { return Cx(a.re + b.re, a.im + b.im); }
static inline real operator-(real a, real b) { return Cx(a.re - b.re, a.im - b.im); }
static inline real operator*(real a, real b) { return Cx(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re); }
static inline real operator/(real a, real b) {
  const double d = b.re * b.re + b.im * b.im;
  return Cx((a.re * b.re + a.im * b.im) / d, (a.im * b.re - a.re * b.im) / d);
}
static inline real operator-(real a) { return Cx(-a.re, -a.im); }
static inline real &operator+=(real &a, real b) { a = a + b; return a; }
static inline real &operator-=(real &a, real b) { a = a - b; return a; }
static inline bool operator<(real a, real b) { return a.re < b.re; }
static inline bool operator>(real a, real b) { return a.re > b.re; }
static inline bool operator<=(real a, real b) { return a.re <= b.re; }
static inline bool operator>=(real a, real b) { return a.re >= b.re; }
static inline real sqrt(real a) {
  // principal square root; for the step size used the imaginary part is tiny
  const double r = std::sqrt(a.re);
  if (r == 0.0) return Cx(0.0, 0.0);
  return Cx(r, a.im / (2.0 * r));
}
static inline real exp(real a) {
  const double e = std::exp(a.re);
  return Cx(e * std::cos(a.im), e * std::sin(a.im));
}
static inline real fabs(real a) { return a.re < 0.0 ? -a : a; }
static inline bool is_finite(real a) { return std::isfinite(a.re) && std::isfinite(a.im); }
static inline void set_phase(int) {}
#else
typedef double real;
static inline double val(real x) { return x; }
static inline bool is_finite(real a) { return std::isfinite(a); }
static inline void set_phase(int) {}
#endif

#ifdef AF_ORACLE_COUNT
static inline real rmax(real a, real b) { tick(K_MINMAX); return (a.v < b.v) ? b : a; }
static inline real rmin(real a, real b) { tick(K_MINMAX); return (b.v < a.v) ? b : a; }
#else
static inline real rmax(real a, real b) { return (a < b) ? b : a; }
static inline real rmin(real a, real b) { return (b < a) ? b : a; }
#endif

// ---------------------------------------------------------------------------
// Parameters (mirrors the fields the test-suite passes in).
// ---------------------------------------------------------------------------
extern "C" {
typedef struct {
  double gamma;
  double x0, x1, y0, y1;
  double cfl;        // dt = cfl / (max rho_1/dx + max rho_2/dy)
  double kappa;      // shock-sensor strength; 0 gives theta^s = 1
  int bc;            // 0 periodic, 1 outflow
  int pp_on;         // positivity-preserving limiters
  int src_cell_on;   // Godunov-Powell source in the cell-average update
  int src_point_on;  // Godunov-Powell source in the point-value update
  // Per-side boundary kinds for bc = 1 (sides: 0 left, 1 right, 2 bottom, 3
  // top): 0 outflow (mirror), 1 reflective (mirror with the normal components
  // of the momentum and of B negated), 2 inflow (bottom/top only: ghost DoFs
  // whose mirror point lies in inflow_lo < x < inflow_hi take inflow_U, the
  // conserved inflow state; outflow elsewhere on that side).
  int side[4];
  double inflow_lo, inflow_hi;
  double inflow_U[8];
  // Example 4.2 variant: the derivative of B_l in the divergence of the
  // point-value source is one-sided along each FVS line, upwind with respect
  // to v_l of the point (D^+ for v_l > 0, D^- for v_l < 0, the central
  // average for v_l = 0) instead of the central (D^+ + D^-)/2 of Sec. 2.3.
  int src_point_upwind;
} or_params;

// Stats slots (cumulative over the call).
enum {
  ST_SRC_LIMITED = 0,   // cells with theta_ij < 1 (step (1))
  ST_LAMBDA_LT1,        // cells with some Lambda_I < 1 (step (2))
  ST_FACE_THETA_LT1,    // faces with theta < 1 (step (3))
  ST_SENSOR_LT099,      // faces with theta^s < 0.99
  ST_NEWTON_SOLVES,     // vertices that needed the cubic solve
  ST_NEWTON_MAXIT,      // maximum Newton iterations seen
  ST_SHRINK,            // round-off shrink events (cells + points)
  ST_POINT_LIMITED,     // points with theta* < 1 or theta** < 1
  ST_CFL_VIOLATIONS,    // cells violating the LLF CFL condition of Lemma 3.1
  ST_CENTER_LIMITED,    // cell-centre values modified by Remark 3.2
  ST_NONADMISSIBLE,     // DoFs left outside G after every safeguard
  ST_CELL_SHRINK,       // the cell-average part of ST_SHRINK (Remark 4.1 for the averages)
  ST_NSTATS
};

// The limiter coefficients of one forward-Euler stage.  Every pointer may be
// NULL.  A stage given a record writes the coefficients it took there; a stage
// given a frozen record uses those values instead of forming them (the sensor,
// the flux limiter and the scaling limiters are then plain blends, and the
// Remark 4.1 shrink is already in the recorded values), so that its result is a
// smooth function of the state along the recorded branch.  The LLF and FVS
// coefficients alpha (maxima) are not recorded: they follow the state.
// Layouts, row-major over the index set named:
//   ths_x, th_x: [ny][nxf] x-faces; ths_y, th_y: [nyf][nx] y-faces;
//   ths_c, th_src: [ny][nx] cells; lam: [4][ny][nx] cells (L, R, D, U);
//   th_pt[cls]: [2][ey][ex] of class cls, theta* then theta** (Sec. 3.3);
//     class 0 holds the cell-centre limiter (Remark 3.2), classes 1..3 the
//     point values after Remark 4.1 (theta** = 0 for the LLF fallback).
typedef struct {
  double *ths_x, *ths_y;   // theta^s per face (Sec. 3.4)
  double *ths_c;           // theta^s_ij, the minimum over the cell's four faces
  double *th_src;          // theta_ij (Sec. 3.2 step 1)
  double *lam;             // Lambda_I (Sec. 3.2 step 2); not read when frozen
  double *th_x, *th_y;     // face theta (Sec. 3.2 step 3, after Remark 4.1)
  double *th_pt[4];        // scaling-limiter theta*, theta**
} or_coeffs;
}

static const int G = 2;  // ghost width (the shock sensor reaches two cells)

struct Ctx {
  int side[4];       // per-side boundary kinds (bc = 1)
  bool special;      // a reflective or inflow side is present
  double x0, y0, in_lo, in_hi, inU[8];
  int nx, ny, bc;
  double dx, dy, gamma, cfl, kappa;
  int pp_on, src_cell_on, src_point_on, src_point_upwind;
  int P, R;          // padded extents (x, y)
  int ext[4][2];     // interior extents per DoF class
  const or_coeffs *rec = nullptr;   // write the stage's limiter coefficients here
  const or_coeffs *frz = nullptr;   // use these limiter coefficients (frozen branch)
  size_t cid(int cls, int i, int j) const { return (size_t)j * ext[cls][0] + (size_t)i; }
  size_t csz(int cls) const { return (size_t)ext[cls][0] * ext[cls][1]; }
  size_t plane() const { return (size_t)P * R; }
  size_t id(int i, int j) const { return (size_t)(j + G) * P + (size_t)(i + G); }
};

static void make_ctx(const or_params *p, int nx, int ny, Ctx &C) {
  C.nx = nx; C.ny = ny; C.bc = p->bc;
  C.dx = (p->x1 - p->x0) / nx; C.dy = (p->y1 - p->y0) / ny;
  C.gamma = p->gamma; C.cfl = p->cfl; C.kappa = p->kappa;
  C.pp_on = p->pp_on; C.src_cell_on = p->src_cell_on; C.src_point_on = p->src_point_on;
  C.src_point_upwind = p->src_point_upwind;
  C.P = nx + 2 * G + 1; C.R = ny + 2 * G + 1;
  int fx = (p->bc == 0) ? nx : nx + 1, fy = (p->bc == 0) ? ny : ny + 1;
  C.ext[0][0] = nx; C.ext[0][1] = ny;
  C.ext[1][0] = fx; C.ext[1][1] = ny;
  C.ext[2][0] = nx; C.ext[2][1] = fy;
  C.ext[3][0] = fx; C.ext[3][1] = fy;
  C.x0 = p->x0; C.y0 = p->y0;
  C.special = false;
  for (int k = 0; k < 4; ++k) {
    C.side[k] = p->bc == 0 ? 0 : p->side[k];
    if (C.side[k] != 0) C.special = true;
  }
  C.in_lo = p->inflow_lo; C.in_hi = p->inflow_hi;
  for (int k = 0; k < 8; ++k) C.inU[k] = p->inflow_U[k];
  C.rec = nullptr;
  C.frz = nullptr;
}

// Axis kind of each class: 0 = cell-centred index, 1 = face/node index.
static const int AXK[4][2] = {{0, 0}, {1, 0}, {0, 1}, {1, 1}};

static inline int imod(int a, int n) { int r = a % n; return r < 0 ? r + n : r; }
// Boundary maps.  Periodic: wrap.  Outflow (Reading: the paper names the
// condition only): ghost DoFs are mirror images of interior DoFs across the
// boundary face, without sign changes (cell -1 <- 0, face -1 <- face 1).
static inline int map_idx(int i, int n, int kind, int bc) {
  if (bc == 0) return imod(i, n);
  if (kind == 0) {
    if (i < 0) return -1 - i;
    if (i >= n) return 2 * n - 1 - i;
    return i;
  }
  if (i < 0) return -i;
  if (i > n) return 2 * n - i;
  return i;
}

// A field with ncomp components on the padded grid.
struct Arr {
  int nc = 0; size_t pl = 0;
  std::vector<real> a;
  void init(const Ctx &C, int ncomp) { nc = ncomp; pl = C.plane(); a.assign((size_t)nc * pl, real(0.0)); }
  real &at(const Ctx &C, int k, int i, int j) { return a[(size_t)k * pl + C.id(i, j)]; }
};

// Fill ghosts of an array that lives on a class's index set.
static void ghost_fill(const Ctx &C, Arr &A, int cls) {
  int ex = C.ext[cls][0], ey = C.ext[cls][1];
  int nx = C.nx, ny = C.ny;
  for (int j = -G; j < ey + G; ++j)
    for (int i = -G; i < ex + G; ++i) {
      if (i >= 0 && i < ex && j >= 0 && j < ey) continue;
      int si = map_idx(i, nx, AXK[cls][0], C.bc), sj = map_idx(j, ny, AXK[cls][1], C.bc);
      for (int k = 0; k < A.nc; ++k) A.at(C, k, i, j) = A.at(C, k, si, sj);
    }
}

// Ghosts of an 8-component state on a class's index set, with the per-side
// kinds.  A ghost index is mapped along x first (mirror; a reflective side
// negates m1 and B1), then along y (mirror; a reflective side negates m2 and
// B2; an inflow side gives the inflow state where the x coordinate of the
// x-mapped index lies strictly inside the inflow range).  Reading: the paper
// names the conditions only (Example 4.8).
static void ghost_fill_state(const Ctx &C, Arr &A, int cls) {
  if (!C.special) {
    ghost_fill(C, A, cls);
    return;
  }
  int ex = C.ext[cls][0], ey = C.ext[cls][1];
  for (int j = -G; j < ey + G; ++j)
    for (int i = -G; i < ex + G; ++i) {
      if (i >= 0 && i < ex && j >= 0 && j < ey) continue;
      int si = map_idx(i, C.nx, AXK[cls][0], C.bc), sj = map_idx(j, C.ny, AXK[cls][1], C.bc);
      bool fx = false, fy = false, inflow = false;
      if (i < 0 || i >= ex) fx = C.side[i < 0 ? 0 : 1] == 1;
      if (j < 0 || j >= ey) {
        const int sd = C.side[j < 0 ? 2 : 3];
        fy = sd == 1;
        if (sd == 2) {
          const double x = C.x0 + (si + (AXK[cls][0] == 0 ? 0.5 : 0.0)) * C.dx;
          inflow = x > C.in_lo && x < C.in_hi;
        }
      }
      for (int k = 0; k < 8; ++k) {
        real v = A.at(C, k, si, sj);
        if ((fx && (k == 1 || k == 4)) || (fy && (k == 2 || k == 5))) v = real(0.0) - v;
        A.at(C, k, i, j) = inflow ? real(C.inU[k]) : v;
      }
    }
}

// ---------------------------------------------------------------------------
// L0: physics (Sec. 1).
// ---------------------------------------------------------------------------
// Perfect-gas pressure p = (gamma-1)(E - |rho v|^2/(2 rho) - |B|^2/2)  (Sec. 1; set G, Sec. 3).
static real pressure(const real *U, double gamma) {
  real m2 = U[1] * U[1] + U[2] * U[2] + U[3] * U[3];
  real b2 = U[4] * U[4] + U[5] * U[5] + U[6] * U[6];
  return real(gamma - 1.0) * (U[7] - m2 / (real(2.0) * U[0]) - b2 / real(2.0));
}

// Everything the scheme needs at one point value: primitives, the fluxes F1,
// F2 (Sec. 1), the fast magnetosonic speeds c_{f,l} and spectral radii
// varrho_l = |v_l| + c_{f,l} (eq. cf), and sqrt(rho) for the LLF bound.
struct PD {
  real U[8];
  real rho, v[3], B[3], p, pt, vB;
  real F[2][8];
  real cf[2], sr[2];
  real srho;
};

static void point_data(const real *U, double gamma, PD &d) {
  for (int k = 0; k < 8; ++k) d.U[k] = U[k];
  d.rho = U[0];
  for (int k = 0; k < 3; ++k) d.v[k] = U[1 + k] / d.rho;
  for (int k = 0; k < 3; ++k) d.B[k] = U[4 + k];
  d.p = pressure(U, gamma);
  real B2 = d.B[0] * d.B[0] + d.B[1] * d.B[1] + d.B[2] * d.B[2];
  d.pt = d.p + real(0.5) * B2;                          // p_t = p + |B|^2/2
  d.vB = d.v[0] * d.B[0] + d.v[1] * d.B[1] + d.v[2] * d.B[2];
  const real rho = d.rho, E = U[7], v1 = d.v[0], v2 = d.v[1], v3 = d.v[2];
  const real B1 = d.B[0], Bb2 = d.B[1], B3 = d.B[2], pt = d.pt, vB = d.vB;
  real *F1 = d.F[0], *F2 = d.F[1];
  F1[0] = rho * v1;
  F1[1] = rho * v1 * v1 - B1 * B1 + pt;
  F1[2] = rho * v1 * v2 - B1 * Bb2;
  F1[3] = rho * v1 * v3 - B1 * B3;
  F1[4] = real(0.0);
  F1[5] = v1 * Bb2 - B1 * v2;
  F1[6] = v1 * B3 - B1 * v3;
  F1[7] = (E + pt) * v1 - B1 * vB;
  F2[0] = rho * v2;
  F2[1] = rho * v1 * v2 - B1 * Bb2;
  F2[2] = rho * v2 * v2 - Bb2 * Bb2 + pt;
  F2[3] = rho * v2 * v3 - Bb2 * B3;
  F2[4] = v2 * B1 - Bb2 * v1;
  F2[5] = real(0.0);
  F2[6] = v2 * B3 - Bb2 * v3;
  F2[7] = (E + pt) * v2 - Bb2 * vB;
  // eq. (cf): c = sqrt(gamma p / rho),
  // c_{f,l} = sqrt( (c^2 + |B|^2/rho + sqrt((c^2 + |B|^2/rho)^2 - 4 c^2 B_l^2/rho)) / 2 ).
  real c2 = real(gamma) * d.p / rho;
  real a = c2 + B2 / rho;
  for (int l = 0; l < 2; ++l) {
    real disc = a * a - real(4.0) * c2 * d.B[l] * d.B[l] / rho;
    // Reading: the discriminant is >= 0 in exact arithmetic; clamp round-off.
    disc = rmax(disc, real(0.0));
    d.cf[l] = sqrt(real(0.5) * (a + sqrt(disc)));
    d.sr[l] = fabs(d.v[l]) + d.cf[l];
  }
  d.srho = sqrt(rho);
}

// Lemma 3.1: alpha_{l,*}(U, Ut).
static real alpha_star(int l, const PD &u, const PD &w) {
  real den = u.srho + w.srho;
  real roe = fabs(u.srho * u.v[l] + w.srho * w.v[l]) / den;
  real db0 = u.B[0] - w.B[0], db1 = u.B[1] - w.B[1], db2 = u.B[2] - w.B[2];
  real nb = sqrt(db0 * db0 + db1 * db1 + db2 * db2);
  return rmax(fabs(u.v[l]), roe) + rmax(u.cf[l], w.cf[l]) + nb / den;
}

// Lemma 3.1 with equality: alpha^LLF = max{varrho(U), varrho(Ut), alpha*(U,Ut), alpha*(Ut,U)}.
static real alpha_llf(int l, const PD &u, const PD &w) {
  return rmax(rmax(u.sr[l], w.sr[l]), rmax(alpha_star(l, u, w), alpha_star(l, w, u)));
}

// eq. (2d_llf_flux): F^LLF_l(U, Ut) = (F_l(U) + F_l(Ut) - alpha (Ut - U)) / 2.
static void llf_flux(int l, const PD &u, const PD &w, real *F, real *alpha_out) {
  real al = alpha_llf(l, u, w);
  for (int k = 0; k < 8; ++k) F[k] = real(0.5) * (u.F[l][k] + w.F[l][k] - al * (w.U[k] - u.U[k]));
  if (alpha_out) *alpha_out = al;
}

// eq. (gp_src): Psi = (0, B, v, v.B).
static void psi(const PD &d, real *P) {
  P[0] = real(0.0);
  P[1] = d.B[0]; P[2] = d.B[1]; P[3] = d.B[2];
  P[4] = d.v[0]; P[5] = d.v[1]; P[6] = d.v[2];
  P[7] = d.vB;
}

static bool in_G(const real *U, double gamma) {
  for (int k = 0; k < 8; ++k) if (!is_finite(U[k])) return false;
  if (!(U[0] > real(0.0))) return false;
  return pressure(U, gamma) > real(0.0);
}

// ---------------------------------------------------------------------------
// Sec. 2.1: finite-difference operators on the bi-parabola of one cell, along
// one line with end values a (left/lower), b (middle), c (right/upper).
// ---------------------------------------------------------------------------
static inline real Dplus(real a, real b, real c, double h) { return (a - real(4.0) * b + real(3.0) * c) / real(h); }   // at the right end
static inline real Dminus(real a, real b, real c, double h) { return (real(-3.0) * a + real(4.0) * b - c) / real(h); } // at the left end
static inline real Dcen(real a, real c, double h) { return (c - a) / real(h); }                                        // at the middle

// Sec. 2.1: cell-centre value of the bi-parabola,
// U_ij = [36 Ubar - 4 (4 face values) - (4 corner values)] / 16.
// Reading: the face and corner sums are taken in pairs, (L+R)+(D+U) and
// (DL+DR)+(UL+UR).
static void center_value(const real *avg, const real *L, const real *R, const real *D, const real *Uu,
                         const real *DL, const real *DR, const real *UL, const real *UR, real *out) {
  for (int k = 0; k < 8; ++k) {
    real faces = (L[k] + R[k]) + (D[k] + Uu[k]);
    real corners = (DL[k] + DR[k]) + (UL[k] + UR[k]);
    out[k] = (real(36.0) * avg[k] - real(4.0) * faces - corners) / real(16.0);
  }
}

// ---------------------------------------------------------------------------
// Sec. 3.3 scaling limiter: blend U^H toward the safe state U^L so that
// rho >= eps_rho, p >= eps_p with eps = min{1e-13, value at U^L}.
// Reading: the density typo rho(U^L) / rho(U^LLF_{i+1/2}) means the safe
// state; step (1) replaces only the density component.  Returns the state;
// theta1 = theta*, theta2 = theta**.
// ---------------------------------------------------------------------------
static void scaling_limiter(const real *UH, const real *UL, double gamma, real *out, real &theta1, real &theta2) {
  real rhoL = UL[0], pL = pressure(UL, gamma);
  real eps_rho = rmin(real(1e-13), rhoL), eps_p = rmin(real(1e-13), pL);
  theta1 = real(1.0);
  if (UH[0] < eps_rho) theta1 = (rhoL - eps_rho) / (rhoL - UH[0]);
  real Us[8];
  for (int k = 0; k < 8; ++k) Us[k] = UH[k];
  Us[0] = theta1 * UH[0] + (real(1.0) - theta1) * rhoL;
  real ps = pressure(Us, gamma);
  theta2 = real(1.0);
  if (ps < eps_p) theta2 = (pL - eps_p) / (pL - ps);
  for (int k = 0; k < 8; ++k) out[k] = theta2 * Us[k] + (real(1.0) - theta2) * UL[k];
}

// The scaling limiter's result for given theta* and theta** (frozen branch).
static void scaling_blend(const real *UH, const real *UL, real theta1, real theta2, real *out) {
  real Us[8];
  for (int k = 0; k < 8; ++k) Us[k] = UH[k];
  Us[0] = theta1 * UH[0] + (real(1.0) - theta1) * UL[0];
  for (int k = 0; k < 8; ++k) out[k] = theta2 * Us[k] + (real(1.0) - theta2) * UL[k];
}

// ---------------------------------------------------------------------------
// Sec. 3.2 step (2): the rectangle [0,Lambda_L]x...x[0,Lambda_U] for one cell,
// from Lim1 = U^{Lim,1} and the anti-diffusive fluxes H[I], I = L,R,D,U.
// ---------------------------------------------------------------------------
struct NewtonLog { long long solves = 0; int maxit = 0; };

// Reading of "solve a cubic equation by Newton's method": along the ray
// V(r) = Lim1 + r D (D = sum_I A_I H_I) the vertex is admissible exactly when
// the cubic q(r) = rho E - |m|^2/2 - rho |B|^2/2 - rho eps_p/(gamma-1)
// = rho (p - eps_p)/(gamma-1) is >= 0 (rho > 0 on the ray).  By concavity of
// the pressure (Sec. 3.2) and q(0) >= 0 > q(1) the root in (0,1) is unique.
// Newton's method on q starts at r = 1 and keeps a sign bracket [lo, hi]
// (q(lo) >= 0 > q(hi)).  A Newton iterate that leaves the open bracket is
// replaced by the Newton iterate from the other end of the bracket, and if
// that one leaves it too, by the bisection point.  Stop when the Newton step
// is <= 1e-14, when the bracket is narrower than 1e-14, or after 40 steps.
struct CubicRay {
  const real *L1, *Dd;
  real ce;
  void eval(real r, real &q, real &dq) const {
    real rho = L1[0] + r * Dd[0];
    real m0 = L1[1] + r * Dd[1], m1 = L1[2] + r * Dd[2], m2 = L1[3] + r * Dd[3];
    real b0 = L1[4] + r * Dd[4], b1 = L1[5] + r * Dd[5], b2 = L1[6] + r * Dd[6];
    real E = L1[7] + r * Dd[7];
    real mm = m0 * m0 + m1 * m1 + m2 * m2;
    real bb = b0 * b0 + b1 * b1 + b2 * b2;
    q = rho * E - real(0.5) * mm - real(0.5) * rho * bb - rho * ce;
    real mdm = m0 * Dd[1] + m1 * Dd[2] + m2 * Dd[3];
    real bdb = b0 * Dd[4] + b1 * Dd[5] + b2 * Dd[6];
    dq = Dd[0] * E + rho * Dd[7] - mdm - real(0.5) * Dd[0] * bb - rho * bdb - Dd[0] * ce;
  }
};

static real newton_root(const real *L1, const real *Dd, real eps_p, double gamma, NewtonLog &nl) {
  CubicRay cr{L1, Dd, eps_p / real(gamma - 1.0)};
  real lo = real(0.0), hi = real(1.0), r = real(1.0);
  real qlo, dqlo, qhi, dqhi, q, dq;
  cr.eval(lo, qlo, dqlo);
  cr.eval(hi, qhi, dqhi);
  q = qhi; dq = dqhi;
  bool at_hi = true;  // the current iterate is the upper end of the bracket
  int it = 0;
  for (; it < 40; ++it) {
    real rn = r - q / dq;
    if (fabs(rn - r) <= real(1e-14)) { r = rn; ++it; break; }   // converged Newton step
    if (!(rn > lo && rn < hi)) {
      real ro = at_hi ? lo - qlo / dqlo : hi - qhi / dqhi;
      rn = (ro > lo && ro < hi) ? ro : real(0.5) * (lo + hi);
    }
    real dr = rn - r;
    r = rn;
    cr.eval(r, q, dq);
    at_hi = !(q >= real(0.0));
    if (!at_hi) { lo = r; qlo = q; dqlo = dq; } else { hi = r; qhi = q; dqhi = dq; }
    if (fabs(dr) <= real(1e-14) || hi - lo <= real(1e-14)) { ++it; break; }
  }
  nl.solves++;
  nl.maxit = std::max(nl.maxit, it);
  return r;
}

static void flux_limiter_box(const real *L1, const real H[4][8], real eps_rho, real eps_p, double gamma,
                             real *Lam, NewtonLog &nl) {
  // Rectangle R_rho of S_rho.
  real negsum = real(0.0);
  for (int J = 0; J < 4; ++J)
    if (H[J][0] < real(0.0)) negsum = negsum + H[J][0];
  real LamRho[4];
  for (int I = 0; I < 4; ++I) {
    LamRho[I] = real(1.0);
    if (H[I][0] < real(0.0)) LamRho[I] = rmin(real(1.0), (L1[0] - eps_rho) / (real(1e-12) - negsum));
  }
  // Shrink R_rho into S_p vertex by vertex.
  for (int I = 0; I < 4; ++I) Lam[I] = LamRho[I];
  for (int kk = 0; kk < 16; ++kk) {
    real A[4];
    for (int I = 0; I < 4; ++I) A[I] = ((kk >> I) & 1) ? LamRho[I] : real(0.0);
    real V[8];
    for (int k = 0; k < 8; ++k) {
      V[k] = L1[k];
      for (int I = 0; I < 4; ++I) V[k] = V[k] + A[I] * H[I][k];
    }
    real r = real(1.0);
    if (pressure(V, gamma) < eps_p) {
      real Dd[8];
      for (int k = 0; k < 8; ++k) {
        Dd[k] = real(0.0);
        for (int I = 0; I < 4; ++I) Dd[k] = Dd[k] + A[I] * H[I][k];
      }
      r = newton_root(L1, Dd, eps_p, gamma, nl);
    }
    // Lambda_I = min over vertices with k_I = 1 of B_I = r A_I.
    for (int I = 0; I < 4; ++I)
      if ((kk >> I) & 1) Lam[I] = rmin(Lam[I], r * A[I]);
  }
}

// ---------------------------------------------------------------------------
// The stage.
// ---------------------------------------------------------------------------
struct State {
  Arr c[4];
  void init(const Ctx &C) { for (int k = 0; k < 4; ++k) c[k].init(C, 8); }
  void get(const Ctx &C, int cls, int i, int j, real *U) { for (int k = 0; k < 8; ++k) U[k] = c[cls].at(C, k, i, j); }
  void put(const Ctx &C, int cls, int i, int j, const real *U) { for (int k = 0; k < 8; ++k) c[cls].at(C, k, i, j) = U[k]; }
};

static void load_state(const Ctx &C, const double *const *U, State &S) {
  S.init(C);
  for (int cls = 0; cls < 4; ++cls) {
    int ex = C.ext[cls][0], ey = C.ext[cls][1];
    for (int k = 0; k < 8; ++k)
      for (int j = 0; j < ey; ++j)
        for (int i = 0; i < ex; ++i)
          S.c[cls].at(C, k, i, j) = real(U[cls][((size_t)k * ey + j) * ex + i]);
  }
}

static void store_state(const Ctx &C, State &S, double *const *U) {
  for (int cls = 0; cls < 4; ++cls) {
    int ex = C.ext[cls][0], ey = C.ext[cls][1];
    for (int k = 0; k < 8; ++k)
      for (int j = 0; j < ey; ++j)
        for (int i = 0; i < ex; ++i)
          U[cls][((size_t)k * ey + j) * ex + i] = val(S.c[cls].at(C, k, i, j));
  }
}

// A point-data grid for one class (or the cell centres).
struct PDGrid {
  std::vector<PD> d;
  void init(const Ctx &C) { d.assign(C.plane(), PD()); }
  PD &at(const Ctx &C, int i, int j) { return d[C.id(i, j)]; }
};

// Point data of the ghost DoFs: copies of the mapped interior DoFs, or, with
// reflective / inflow sides, the point data of the ghost states in A.
static void pd_ghost_fill(const Ctx &C, PDGrid &Pg, int cls, Arr *A = nullptr) {
  int ex = C.ext[cls][0], ey = C.ext[cls][1];
  if (C.special && A) {
    for (int j = -G; j < ey + G; ++j)
      for (int i = -G; i < ex + G; ++i) {
        if (i >= 0 && i < ex && j >= 0 && j < ey) continue;
        real U[8];
        for (int k = 0; k < 8; ++k) U[k] = A->at(C, k, i, j);
        point_data(U, C.gamma, Pg.at(C, i, j));
      }
    return;
  }
  for (int j = -G; j < ey + G; ++j)
    for (int i = -G; i < ex + G; ++i) {
      if (i >= 0 && i < ex && j >= 0 && j < ey) continue;
      int si = map_idx(i, C.nx, AXK[cls][0], C.bc), sj = map_idx(j, C.ny, AXK[cls][1], C.bc);
      Pg.at(C, i, j) = Pg.at(C, si, sj);
    }
}

struct StageOut {
  long long st[ST_NSTATS];
};

// Everything one forward-Euler stage computes, kept for the diagnostics.
struct Work {
  PDGrid pd[4], pdc;     // point data of the 4 classes and of the (limited) cell centres
  Arr Uc;                // limited cell-centre values
  Arr UH[4];             // high-order point updates (classes 1..3)
  Arr FE[4];             // forward-Euler results
  Arr phi;               // phi1x, phi1y, phi2, phi3 per cell
  Arr fx, fy;            // per face: Simpson flux (0..7), LLF flux (8..15), theta^s (16), alpha^LLF (17)
  Arr lim1, H, lam;      // per cell: Lim1 (8), H (4x8), Lambda (4)
  Arr ths;               // theta^s_ij
};

static void compute_point_data(const Ctx &C, State &S, Work &W) {
  set_phase(PH_POINTDATA);
  for (int cls = 0; cls < 4; ++cls) {
    W.pd[cls].init(C);
    int ex = C.ext[cls][0], ey = C.ext[cls][1];
#ifndef AF_ORACLE_COUNT
#pragma omp parallel for schedule(static)
#endif
    for (int j = 0; j < ey; ++j)
      for (int i = 0; i < ex; ++i) {
        real U[8];
        S.get(C, cls, i, j, U);
        point_data(U, C.gamma, W.pd[cls].at(C, i, j));
      }
    pd_ghost_fill(C, W.pd[cls], cls, &S.c[cls]);
  }
}

// Sec. 2.1 reconstruction + Remark 3.2 (cell-centre limiter).  Reading: the
// limiter is the Sec. 3.3 scaling limiter with the cell average as the safe
// state.  Ghost cell-centre values are those of the mapped interior cell.
static void compute_centers(const Ctx &C, State &S, Work &W, long long *st) {
  set_phase(PH_CENTER);
  W.Uc.init(C, 8);
  long long nlim = 0;
#ifndef AF_ORACLE_COUNT
#pragma omp parallel for schedule(static) reduction(+ : nlim)
#endif
  for (int j = 0; j < C.ny; ++j)
    for (int i = 0; i < C.nx; ++i) {
      real avg[8], L[8], R[8], D[8], Uu[8], DL[8], DR[8], UL[8], UR[8], uc[8], out[8];
      S.get(C, 0, i, j, avg);
      S.get(C, 1, i, j, L); S.get(C, 1, i + 1, j, R);
      S.get(C, 2, i, j, D); S.get(C, 2, i, j + 1, Uu);
      S.get(C, 3, i, j, DL); S.get(C, 3, i + 1, j, DR);
      S.get(C, 3, i, j + 1, UL); S.get(C, 3, i + 1, j + 1, UR);
      center_value(avg, L, R, D, Uu, DL, DR, UL, UR, uc);
      real t1, t2;
      if (C.frz && C.frz->th_pt[0]) {
        t1 = real(C.frz->th_pt[0][C.cid(0, i, j)]);
        t2 = real(C.frz->th_pt[0][C.csz(0) + C.cid(0, i, j)]);
        scaling_blend(uc, avg, t1, t2, out);
      } else {
        scaling_limiter(uc, avg, C.gamma, out, t1, t2);
      }
      if (C.rec && C.rec->th_pt[0]) {
        C.rec->th_pt[0][C.cid(0, i, j)] = val(t1);
        C.rec->th_pt[0][C.csz(0) + C.cid(0, i, j)] = val(t2);
      }
      if (t1 < real(1.0) || t2 < real(1.0)) nlim++;
      for (int k = 0; k < 8; ++k) W.Uc.at(C, k, i, j) = out[k];
    }
  st[ST_CENTER_LIMITED] += nlim;
  ghost_fill_state(C, W.Uc, 0);
  set_phase(PH_POINTDATA);
  W.pdc.init(C);
#ifndef AF_ORACLE_COUNT
#pragma omp parallel for schedule(static)
#endif
  for (int j = 0; j < C.ny; ++j)
    for (int i = 0; i < C.nx; ++i) {
      real U[8];
      for (int k = 0; k < 8; ++k) U[k] = W.Uc.at(C, k, i, j);
      point_data(U, C.gamma, W.pdc.at(C, i, j));
    }
  pd_ghost_fill(C, W.pdc, 0, &W.Uc);
}

// Sec. 2.3: the 5-point line through a point value and its LLF-FVS derivative
// -(D^+ F^+ + D^- F^-) with F^pm = (F +- alpha U)/2 and alpha the largest
// spectral radius on the line.  P[0..4] are the points at offsets -1, -1/2, 0,
// +1/2, +1 (in units of the mesh size); the cell to the left/below holds
// P[0..2], the one to the right/above holds P[2..4].
// With upw = 0 the derivative of B_l in the point source is the central
// (D^+ B_l + D^- B_l)/2 of Sec. 2.3; upw = +1 / -1 selects D^+ / D^- alone (the
// velocity-upwind variant of Example 4.2).
static void fvs_derivative(int l, const PD *const P[5], double h, real *out, real &dBl, int upw = 0) {
  real al = P[0]->sr[l];
  for (int q = 1; q < 5; ++q) al = rmax(al, P[q]->sr[l]);
  for (int k = 0; k < 8; ++k) {
    real Fp[3], Fm[3];
    for (int q = 0; q < 3; ++q) Fp[q] = real(0.5) * (P[q]->F[l][k] + al * P[q]->U[k]);
    for (int q = 0; q < 3; ++q) Fm[q] = real(0.5) * (P[q + 2]->F[l][k] - al * P[q + 2]->U[k]);
    out[k] = Dplus(Fp[0], Fp[1], Fp[2], h) + Dminus(Fm[0], Fm[1], Fm[2], h);
  }
  const real Dp = Dplus(P[0]->B[l], P[1]->B[l], P[2]->B[l], h), Dm = Dminus(P[2]->B[l], P[3]->B[l], P[4]->B[l], h);
  if (upw > 0) dBl = Dp;
  else if (upw < 0) dBl = Dm;
  else dBl = real(0.5) * (Dp + Dm);   // central discrete derivative of B_l
}

// Direction selector of the upwind variant for the FVS line of direction l through point d.
static int upwind_sign(const Ctx &C, const PD &d, int l) {
  if (!C.src_point_upwind) return 0;
  const double v = val(d.v[l]);
  return v > 0.0 ? 1 : (v < 0.0 ? -1 : 0);
}

static void point_ho_updates(const Ctx &C, real dt, Work &W) {
  set_phase(PH_POINT_HO);
  for (int cls = 1; cls < 4; ++cls) W.UH[cls].init(C, 8);
  const double dx = C.dx, dy = C.dy;
  for (int cls = 1; cls < 4; ++cls) {
    int ex = C.ext[cls][0], ey = C.ext[cls][1];
#ifndef AF_ORACLE_COUNT
#pragma omp parallel for schedule(static)
#endif
    for (int j = 0; j < ey; ++j)
      for (int i = 0; i < ex; ++i) {
        real rhs[8], d1[8], d2[8], dB1, dB2;
        const PD &me = W.pd[cls].at(C, i, j);
        if (cls == 3) {
          // corner (f,g) = (i,j): x-line of corners and y-face values on row g,
          // y-line of corners and x-face values on column f.
          const PD *Px[5] = {&W.pd[3].at(C, i - 1, j), &W.pd[2].at(C, i - 1, j), &me, &W.pd[2].at(C, i, j), &W.pd[3].at(C, i + 1, j)};
          const PD *Py[5] = {&W.pd[3].at(C, i, j - 1), &W.pd[1].at(C, i, j - 1), &me, &W.pd[1].at(C, i, j), &W.pd[3].at(C, i, j + 1)};
          fvs_derivative(0, Px, dx, d1, dB1, upwind_sign(C, me, 0));
          fvs_derivative(1, Py, dy, d2, dB2, upwind_sign(C, me, 1));
        } else if (cls == 1) {
          // x-face (f,j): x-line through the cell-centre values of cells f-1, f;
          // central D_2 F_2 between the corners (f,j) and (f,j+1).
          const PD *Px[5] = {&W.pd[1].at(C, i - 1, j), &W.pdc.at(C, i - 1, j), &me, &W.pdc.at(C, i, j), &W.pd[1].at(C, i + 1, j)};
          fvs_derivative(0, Px, dx, d1, dB1, upwind_sign(C, me, 0));
          const PD &lo = W.pd[3].at(C, i, j), &hi = W.pd[3].at(C, i, j + 1);
          for (int k = 0; k < 8; ++k) d2[k] = Dcen(lo.F[1][k], hi.F[1][k], dy);
          dB2 = Dcen(lo.B[1], hi.B[1], dy);
        } else {
          // y-face (i,g): central D_1 F_1 between corners (i,g), (i+1,g);
          // y-line through the cell-centre values of cells (i,g-1), (i,g).
          const PD &lo = W.pd[3].at(C, i, j), &hi = W.pd[3].at(C, i + 1, j);
          for (int k = 0; k < 8; ++k) d1[k] = Dcen(lo.F[0][k], hi.F[0][k], dx);
          dB1 = Dcen(lo.B[0], hi.B[0], dx);
          const PD *Py[5] = {&W.pd[2].at(C, i, j - 1), &W.pdc.at(C, i, j - 1), &me, &W.pdc.at(C, i, j), &W.pd[2].at(C, i, j + 1)};
          fvs_derivative(1, Py, dy, d2, dB2, upwind_sign(C, me, 1));
        }
        real divB = dB1 + dB2;
        real Ps[8];
        psi(me, Ps);
        for (int k = 0; k < 8; ++k) {
          rhs[k] = real(0.0) - d1[k] - d2[k];
          if (C.src_point_on) rhs[k] = rhs[k] - divB * Ps[k];
        }
        for (int k = 0; k < 8; ++k) W.UH[cls].at(C, k, i, j) = me.U[k] + dt * rhs[k];
      }
  }
}

// Sec. 3.3: first-order LLF schemes for the three point classes, then the
// scaling limiter and the round-off safeguard (Remark 4.1).
// Reading (transverse spacing): the printed stencils are used literally,
// i.e. the face/corner fluxes half a cell apart are divided by dx or dy.
static void point_limit(const Ctx &C, real dt, Work &W, long long *st) {
  const double dx = C.dx, dy = C.dy;
  long long nlim = 0, nshrink = 0, nbad = 0;
  for (int cls = 1; cls < 4; ++cls) {
    W.FE[cls].init(C, 8);
    int ex = C.ext[cls][0], ey = C.ext[cls][1];
#ifndef AF_ORACLE_COUNT
#pragma omp parallel for schedule(static) reduction(+ : nlim, nshrink, nbad)
#endif
    for (int j = 0; j < ey; ++j)
      for (int i = 0; i < ex; ++i) {
        const PD &me = W.pd[cls].at(C, i, j);
        real UH[8];
        for (int k = 0; k < 8; ++k) UH[k] = W.UH[cls].at(C, k, i, j);
        if (!C.pp_on) {
          for (int k = 0; k < 8; ++k) W.FE[cls].at(C, k, i, j) = UH[k];
          continue;
        }
        set_phase(PH_POINT_PP);
        const PD *xl, *xr, *yl, *yr;   // neighbours for F1 (x) and F2 (y) LLF fluxes
        if (cls == 3) {
          xl = &W.pd[3].at(C, i - 1, j); xr = &W.pd[3].at(C, i + 1, j);
          yl = &W.pd[3].at(C, i, j - 1); yr = &W.pd[3].at(C, i, j + 1);
        } else if (cls == 1) {
          xl = &W.pd[1].at(C, i - 1, j); xr = &W.pd[1].at(C, i + 1, j);
          yl = &W.pd[3].at(C, i, j); yr = &W.pd[3].at(C, i, j + 1);
        } else {
          xl = &W.pd[3].at(C, i, j); xr = &W.pd[3].at(C, i + 1, j);
          yl = &W.pd[2].at(C, i, j - 1); yr = &W.pd[2].at(C, i, j + 1);
        }
        real Fxr[8], Fxl[8], Fyr[8], Fyl[8];
        llf_flux(0, me, *xr, Fxr, nullptr);
        llf_flux(0, *xl, me, Fxl, nullptr);
        llf_flux(1, me, *yr, Fyr, nullptr);
        llf_flux(1, *yl, me, Fyl, nullptr);
        real divB = (xr->B[0] - xl->B[0]) / real(2.0 * dx) + (yr->B[1] - yl->B[1]) / real(2.0 * dy);
        real Ps[8], UL[8];
        psi(me, Ps);
        for (int k = 0; k < 8; ++k) {
          UL[k] = me.U[k] - dt / real(dx) * (Fxr[k] - Fxl[k]) - dt / real(dy) * (Fyr[k] - Fyl[k]);
          if (C.src_point_on) UL[k] = UL[k] - dt * divB * Ps[k];
        }
        real out[8], t1, t2;
        if (C.frz && C.frz->th_pt[cls]) {
          t1 = real(C.frz->th_pt[cls][C.cid(cls, i, j)]);
          t2 = real(C.frz->th_pt[cls][C.csz(cls) + C.cid(cls, i, j)]);
          scaling_blend(UH, UL, t1, t2, out);
          if (t1 < real(1.0) || t2 < real(1.0)) nlim++;
          for (int k = 0; k < 8; ++k) W.FE[cls].at(C, k, i, j) = out[k];
          continue;
        }
        scaling_limiter(UH, UL, C.gamma, out, t1, t2);
        if (t1 < real(1.0) || t2 < real(1.0)) nlim++;
        real t2_used = t2;
        if (!in_G(out, C.gamma)) {
          // Remark 4.1: shrink theta** by 2^m 1e-8, m = 0..9 (Reading: from
          // its first value, not cumulatively), else fall back to U^L.
          nshrink++;
          real Us[8];
          for (int k = 0; k < 8; ++k) Us[k] = UH[k];
          Us[0] = t1 * UH[0] + (real(1.0) - t1) * UL[0];
          bool ok = false;
          for (int m = 0; m < 10 && !ok; ++m) {
            real th = rmax(real(0.0), t2 - real(std::ldexp(1e-8, m)));
            for (int k = 0; k < 8; ++k) out[k] = th * Us[k] + (real(1.0) - th) * UL[k];
            ok = in_G(out, C.gamma);
            t2_used = th;
          }
          if (!ok) { for (int k = 0; k < 8; ++k) out[k] = UL[k]; t2_used = real(0.0); }
          if (!in_G(out, C.gamma)) nbad++;
        }
        if (C.rec && C.rec->th_pt[cls]) {
          C.rec->th_pt[cls][C.cid(cls, i, j)] = val(t1);
          C.rec->th_pt[cls][C.csz(cls) + C.cid(cls, i, j)] = val(t2_used);
        }
        for (int k = 0; k < 8; ++k) W.FE[cls].at(C, k, i, j) = out[k];
      }
  }
  st[ST_POINT_LIMITED] += nlim;
  st[ST_SHRINK] += nshrink;
  st[ST_NONADMISSIBLE] += nbad;
}

// Sec. 3.4 shock sensor.  phi values are computed on the cells [-1, n] from
// the (ghost-filled) cell averages.  Reading: the printed phi_1 (Jameson on
// p_t) differences along x and serves x-faces; its transpose (along y)
// serves y-faces.  phi_2 (modified Ducros) and phi_3 (divergence) are as printed.
// phi_1 (x and y), phi_2, phi_3 of one cell from the point data of its cell
// average (c) and of the averages east, west, north and south of it.
static void sensor_phi(const PD &c, const PD &e, const PD &w, const PD &n, const PD &s, double dx, double dy,
                       real *phi) {
  phi[0] = fabs(e.pt - real(2.0) * c.pt + w.pt) / fabs(e.pt + real(2.0) * c.pt + w.pt);
  phi[1] = fabs(n.pt - real(2.0) * c.pt + s.pt) / fabs(n.pt + real(2.0) * c.pt + s.pt);
  real divv = (e.v[0] - w.v[0]) / real(2.0 * dx) + (n.v[1] - s.v[1]) / real(2.0 * dy);
  real curlv = (e.v[1] - w.v[1]) / real(2.0 * dx) - (n.v[0] - s.v[0]) / real(2.0 * dy);
  phi[2] = rmax((real(0.0) - divv) / sqrt(divv * divv + curlv * curlv + real(1e-40)), real(0.0));
  phi[3] = fabs(e.B[0] - w.B[0] + n.B[1] - s.B[1]) / (fabs(c.B[0] + c.B[1]) + real(1e-40));
}

static void compute_sensor(const Ctx &C, Work &W) {
  set_phase(PH_SENSOR_PHI);
  W.phi.init(C, 4);
  const double dx = C.dx, dy = C.dy;
  // pass 1: p_t, v, B from each cell average (extended range, from point data of class 0)
#ifndef AF_ORACLE_COUNT
#pragma omp parallel for schedule(static)
#endif
  for (int j = -1; j <= C.ny; ++j)
    for (int i = -1; i <= C.nx; ++i) {
#ifdef AF_ORACLE_COUNT
      g_count_on = (i >= 0 && i < C.nx && j >= 0 && j < C.ny);
#endif
      real ph[4];
      sensor_phi(W.pd[0].at(C, i, j), W.pd[0].at(C, i + 1, j), W.pd[0].at(C, i - 1, j), W.pd[0].at(C, i, j + 1),
                 W.pd[0].at(C, i, j - 1), dx, dy, ph);
      for (int q = 0; q < 4; ++q) W.phi.at(C, q, i, j) = ph[q];
    }
#ifdef AF_ORACLE_COUNT
  g_count_on = 1;
#endif
}

// theta^s at a face from the phi of the two adjacent cells (a: left/below, b: right/above).
static real theta_s(const Ctx &C, Work &W, int dir, int ia, int ja, int ib, int jb) {
  if (C.kappa == 0.0) return real(1.0);
  real p1 = rmax(W.phi.at(C, dir, ia, ja), W.phi.at(C, dir, ib, jb));
  real p2 = rmax(W.phi.at(C, 2, ia, ja), W.phi.at(C, 2, ib, jb));
  real p3 = rmax(W.phi.at(C, 3, ia, ja), W.phi.at(C, 3, ib, jb));
  return exp(real(0.0) - real(C.kappa) * (p1 * p2 + p3));
}

// Per-face data: Simpson flux (Sec. 2.2), LLF flux between the adjacent cell
// averages (eq. 2d_llf_flux) and theta^s (Sec. 3.4).
static void compute_faces(const Ctx &C, Work &W, long long *st) {
  set_phase(PH_FACE);
  W.fx.init(C, 18); W.fy.init(C, 18);
  long long nsens = 0;
  // x-faces: index set of class 1
#ifndef AF_ORACLE_COUNT
#pragma omp parallel for schedule(static) reduction(+ : nsens)
#endif
  for (int j = 0; j < C.ext[1][1]; ++j)
    for (int f = 0; f < C.ext[1][0]; ++f) {
      const PD &lo = W.pd[3].at(C, f, j), &mid = W.pd[1].at(C, f, j), &hi = W.pd[3].at(C, f, j + 1);
      for (int k = 0; k < 8; ++k) W.fx.at(C, k, f, j) = (lo.F[0][k] + real(4.0) * mid.F[0][k] + hi.F[0][k]) / real(6.0);
      real Fl[8], al;
      llf_flux(0, W.pd[0].at(C, f - 1, j), W.pd[0].at(C, f, j), Fl, &al);
      for (int k = 0; k < 8; ++k) W.fx.at(C, 8 + k, f, j) = Fl[k];
      set_phase(PH_SENSOR_THETA);
      real ts = (C.frz && C.frz->ths_x) ? real(C.frz->ths_x[C.cid(1, f, j)]) : theta_s(C, W, 0, f - 1, j, f, j);
      if (C.rec && C.rec->ths_x) C.rec->ths_x[C.cid(1, f, j)] = val(ts);
      set_phase(PH_FACE);
      W.fx.at(C, 16, f, j) = ts;
      W.fx.at(C, 17, f, j) = al;
      if (val(ts) < 0.99) nsens++;
    }
#ifndef AF_ORACLE_COUNT
#pragma omp parallel for schedule(static) reduction(+ : nsens)
#endif
  for (int g = 0; g < C.ext[2][1]; ++g)
    for (int i = 0; i < C.ext[2][0]; ++i) {
      const PD &lo = W.pd[3].at(C, i, g), &mid = W.pd[2].at(C, i, g), &hi = W.pd[3].at(C, i + 1, g);
      for (int k = 0; k < 8; ++k) W.fy.at(C, k, i, g) = (lo.F[1][k] + real(4.0) * mid.F[1][k] + hi.F[1][k]) / real(6.0);
      real Fl[8], al;
      llf_flux(1, W.pd[0].at(C, i, g - 1), W.pd[0].at(C, i, g), Fl, &al);
      for (int k = 0; k < 8; ++k) W.fy.at(C, 8 + k, i, g) = Fl[k];
      set_phase(PH_SENSOR_THETA);
      real ts = (C.frz && C.frz->ths_y) ? real(C.frz->ths_y[C.cid(2, i, g)]) : theta_s(C, W, 1, i, g - 1, i, g);
      if (C.rec && C.rec->ths_y) C.rec->ths_y[C.cid(2, i, g)] = val(ts);
      set_phase(PH_FACE);
      W.fy.at(C, 16, i, g) = ts;
      W.fy.at(C, 17, i, g) = al;
      if (val(ts) < 0.99) nsens++;
    }
  st[ST_SENSOR_LT099] += nsens;
  ghost_fill(C, W.fx, 1);
  ghost_fill(C, W.fy, 2);
}

// eq. (semi_av_src): S_ij = sum_{l,m} w_l w_m (div B)^{l,m} Psi(U^{l,m}) on the
// 3x3 Simpson nodes of cell (i,j).  Reading: nodes are numbered 0,1,2 with 1
// the cell centre (the printed divergence list uses 0,1,2).
static void cell_source(const Ctx &C, Work &W, int i, int j, real *S) {
  const PD *N[3][3];  // N[l][m]: l along x, m along y
  N[0][0] = &W.pd[3].at(C, i, j);     N[1][0] = &W.pd[2].at(C, i, j);     N[2][0] = &W.pd[3].at(C, i + 1, j);
  N[0][1] = &W.pd[1].at(C, i, j);     N[1][1] = &W.pdc.at(C, i, j);       N[2][1] = &W.pd[1].at(C, i + 1, j);
  N[0][2] = &W.pd[3].at(C, i, j + 1); N[1][2] = &W.pd[2].at(C, i, j + 1); N[2][2] = &W.pd[3].at(C, i + 1, j + 1);
  const real w[3] = {real(1.0) / real(6.0), real(2.0) / real(3.0), real(1.0) / real(6.0)};
  for (int k = 0; k < 8; ++k) S[k] = real(0.0);
  for (int l = 0; l < 3; ++l)
    for (int m = 0; m < 3; ++m) {
      real dB1, dB2;
      // d B1 / dx along row m
      if (l == 0) dB1 = Dminus(N[0][m]->B[0], N[1][m]->B[0], N[2][m]->B[0], C.dx);
      else if (l == 1) dB1 = Dcen(N[0][m]->B[0], N[2][m]->B[0], C.dx);
      else dB1 = Dplus(N[0][m]->B[0], N[1][m]->B[0], N[2][m]->B[0], C.dx);
      // d B2 / dy along column l
      if (m == 0) dB2 = Dminus(N[l][0]->B[1], N[l][1]->B[1], N[l][2]->B[1], C.dy);
      else if (m == 1) dB2 = Dcen(N[l][0]->B[1], N[l][2]->B[1], C.dy);
      else dB2 = Dplus(N[l][0]->B[1], N[l][1]->B[1], N[l][2]->B[1], C.dy);
      real divB = dB1 + dB2;
      real Ps[8];
      psi(*N[l][m], Ps);
      for (int k = 0; k < 8; ++k) S[k] = S[k] + w[l] * w[m] * divB * Ps[k];
    }
}

// Sec. 3.2: the parametrized flux limiter for the cell averages, with the
// sensor blend of Sec. 3.4 applied first (Reading: the sensor-blended flux and
// source play the role of the high-order terms in the PP limiter).
static void cell_update(const Ctx &C, real dt, Work &W, long long *st) {
  const double dx = C.dx, dy = C.dy;
  W.FE[0].init(C, 8);
  W.lim1.init(C, 8); W.H.init(C, 32); W.lam.init(C, 4); W.ths.init(C, 1);
  long long nsrc = 0, nlam = 0, ncfl = 0;
  NewtonLog nl_total;
#ifndef AF_ORACLE_COUNT
#pragma omp parallel
#endif
  {
    NewtonLog nl;
    long long a_src = 0, a_lam = 0, a_cfl = 0;
#ifndef AF_ORACLE_COUNT
#pragma omp for schedule(static)
#endif
    for (int j = 0; j < C.ny; ++j)
      for (int i = 0; i < C.nx; ++i) {
        set_phase(PH_CELL_SRC);
        const PD &cb = W.pd[0].at(C, i, j);
        real S[8], SL[8];
        cell_source(C, W, i, j, S);
        // S^LLF = (central div Bbar) Psi(Ubar)
        const PD &e = W.pd[0].at(C, i + 1, j), &w = W.pd[0].at(C, i - 1, j);
        const PD &n = W.pd[0].at(C, i, j + 1), &s = W.pd[0].at(C, i, j - 1);
        real divBbar = (e.B[0] - w.B[0]) / real(2.0 * dx) + (n.B[1] - s.B[1]) / real(2.0 * dy);
        real Pb[8];
        psi(cb, Pb);
        for (int k = 0; k < 8; ++k) SL[k] = divBbar * Pb[k];
        if (!C.src_cell_on) for (int k = 0; k < 8; ++k) { S[k] = real(0.0); SL[k] = real(0.0); }
        set_phase(PH_CELL_UPDATE);
        // faces: L = x-face i, R = x-face i+1, D = y-face j, U = y-face j+1
        real tsL = W.fx.at(C, 16, i, j), tsR = W.fx.at(C, 16, i + 1, j);
        real tsD = W.fy.at(C, 16, i, j), tsU = W.fy.at(C, 16, i, j + 1);
        real tsc = rmin(rmin(tsL, tsR), rmin(tsD, tsU));   // theta^s_ij
        W.ths.at(C, 0, i, j) = tsc;
        if (C.rec && C.rec->ths_c) C.rec->ths_c[C.cid(0, i, j)] = val(tsc);
        real Fss[4][8], Fll[4][8];
        const real tsf[4] = {tsL, tsR, tsD, tsU};
        for (int k = 0; k < 8; ++k) {
          Fll[0][k] = W.fx.at(C, 8 + k, i, j); Fll[1][k] = W.fx.at(C, 8 + k, i + 1, j);
          Fll[2][k] = W.fy.at(C, 8 + k, i, j); Fll[3][k] = W.fy.at(C, 8 + k, i, j + 1);
          real Fh[4] = {W.fx.at(C, k, i, j), W.fx.at(C, k, i + 1, j), W.fy.at(C, k, i, j), W.fy.at(C, k, i, j + 1)};
          for (int I = 0; I < 4; ++I) {
            if (C.kappa == 0.0) Fss[I][k] = Fh[I];
            else Fss[I][k] = tsf[I] * Fh[I] + (real(1.0) - tsf[I]) * Fll[I][k];
          }
        }
        real Sss[8];
        for (int k = 0; k < 8; ++k) Sss[k] = (C.kappa == 0.0) ? S[k] : tsc * S[k] + (real(1.0) - tsc) * SL[k];
        const real *Ub = cb.U;
        real out[8];
        if (!C.pp_on) {
          for (int k = 0; k < 8; ++k)
            out[k] = Ub[k] - dt / real(dx) * (Fss[1][k] - Fss[0][k]) - dt / real(dy) * (Fss[3][k] - Fss[2][k]) - dt * Sss[k];
          for (int k = 0; k < 8; ++k) W.FE[0].at(C, k, i, j) = out[k];
          continue;
        }
        // eq. (2d_llf) and U^src.
        real Ullf[8], Usrc[8];
        for (int k = 0; k < 8; ++k) {
          real flux = Ub[k] - dt / real(dx) * (Fll[1][k] - Fll[0][k]) - dt / real(dy) * (Fll[3][k] - Fll[2][k]);
          Ullf[k] = flux - dt * SL[k];
          Usrc[k] = flux - dt * Sss[k];
        }
        // Lemma 3.1 CFL condition (diagnostic only; dt is not changed).
        {
          real lhs = dt * (W.fx.at(C, 17, i, j) / real(dx) + W.fx.at(C, 17, i + 1, j) / real(dx) +
                           W.fy.at(C, 17, i, j) / real(dy) + W.fy.at(C, 17, i, j + 1) / real(dy) +
                           fabs(divBbar) / cb.srho);
          if (val(lhs) > 1.0 + 1e-12) a_cfl++;
        }
        real eps_rho = rmin(real(1e-13), Ullf[0]);
        real pllf = pressure(Ullf, C.gamma);
        real eps_p = rmin(real(1e-13), pllf);
        // step (1): theta_ij.  Reading: theta_ij = 1 when p(U^src) >= eps_p.
        real th = real(1.0);
        if (C.frz && C.frz->th_src) {
          th = real(C.frz->th_src[C.cid(0, i, j)]);
          if (th < real(1.0)) a_src++;
        } else {
          real psrc = pressure(Usrc, C.gamma);
          if (psrc < eps_p) { th = rmin(real(1.0), (pllf - eps_p) / (pllf - psrc)); a_src++; }
        }
        if (C.rec && C.rec->th_src) C.rec->th_src[C.cid(0, i, j)] = val(th);
        real L1[8];
        // Lim1 = theta U^src + (1-theta) U^LLF, written as U^LLF + theta (U^src - U^LLF)
        // so that its density equals that of U^LLF exactly (Psi_1 = 0).
        for (int k = 0; k < 8; ++k) L1[k] = Ullf[k] + th * (Usrc[k] - Ullf[k]);
        // step (2): anti-diffusive fluxes
        real H[4][8];
        for (int k = 0; k < 8; ++k) {
          H[0][k] = dt / real(dx) * (Fss[0][k] - Fll[0][k]);
          H[1][k] = real(0.0) - dt / real(dx) * (Fss[1][k] - Fll[1][k]);
          H[2][k] = dt / real(dy) * (Fss[2][k] - Fll[2][k]);
          H[3][k] = real(0.0) - dt / real(dy) * (Fss[3][k] - Fll[3][k]);
        }
        real Lam[4] = {real(1.0), real(1.0), real(1.0), real(1.0)};
        if (!(C.frz && C.frz->th_x && C.frz->th_y)) flux_limiter_box(L1, H, eps_rho, eps_p, C.gamma, Lam, nl);
        if (Lam[0] < real(1.0) || Lam[1] < real(1.0) || Lam[2] < real(1.0) || Lam[3] < real(1.0)) a_lam++;
        if (C.rec && C.rec->lam)
          for (int I = 0; I < 4; ++I) C.rec->lam[(size_t)I * C.csz(0) + C.cid(0, i, j)] = val(Lam[I]);
        for (int k = 0; k < 8; ++k) W.lim1.at(C, k, i, j) = L1[k];
        for (int I = 0; I < 4; ++I)
          for (int k = 0; k < 8; ++k) W.H.at(C, I * 8 + k, i, j) = H[I][k];
        for (int I = 0; I < 4; ++I) W.lam.at(C, I, i, j) = Lam[I];
      }
#ifndef AF_ORACLE_COUNT
#pragma omp critical
#endif
    {
      nsrc += a_src; nlam += a_lam; ncfl += a_cfl;
      nl_total.solves += nl.solves;
      nl_total.maxit = std::max(nl_total.maxit, nl.maxit);
    }
  }
  st[ST_SRC_LIMITED] += nsrc;
  st[ST_LAMBDA_LT1] += nlam;
  st[ST_CFL_VIOLATIONS] += ncfl;
  st[ST_NEWTON_SOLVES] += nl_total.solves;
  st[ST_NEWTON_MAXIT] = std::max<long long>(st[ST_NEWTON_MAXIT], nl_total.maxit);
}

// Sec. 3.2 step (3): unique face coefficients and the limited update.
// Reading (outflow): a boundary face takes the Lambda of its one interior cell.
static real face_theta_x(const Ctx &C, Work &W, int f, int j) {
  if (C.bc == 1 && f == 0) return W.lam.at(C, 0, 0, j);
  if (C.bc == 1 && f == C.nx) return W.lam.at(C, 1, C.nx - 1, j);
  return rmin(W.lam.at(C, 1, f - 1, j), W.lam.at(C, 0, f, j));
}
static real face_theta_y(const Ctx &C, Work &W, int i, int g) {
  if (C.bc == 1 && g == 0) return W.lam.at(C, 2, i, 0);
  if (C.bc == 1 && g == C.ny) return W.lam.at(C, 3, i, C.ny - 1);
  return rmin(W.lam.at(C, 3, i, g - 1), W.lam.at(C, 2, i, g));
}

static void cell_value(const Ctx &C, Work &W, const real th[4], int i, int j, real *out) {
  for (int k = 0; k < 8; ++k) {
    real u = W.lim1.at(C, k, i, j);
    for (int I = 0; I < 4; ++I) u = u + th[I] * W.H.at(C, I * 8 + k, i, j);
    out[k] = u;
  }
}

static void cell_final(const Ctx &C, Work &W, long long *st) {
  if (!C.pp_on) return;
  set_phase(PH_CELL_FINAL);
  if (C.bc == 0) ghost_fill(C, W.lam, 0);
  // face coefficients (x: class-1 index set, y: class-2 index set)
  Arr thx, thy;
  thx.init(C, 1); thy.init(C, 1);
  long long nface = 0;
  const bool frozen = C.frz && C.frz->th_x && C.frz->th_y;
  for (int j = 0; j < C.ext[1][1]; ++j)
    for (int f = 0; f < C.ext[1][0]; ++f) {
      thx.at(C, 0, f, j) = frozen ? real(C.frz->th_x[C.cid(1, f, j)]) : face_theta_x(C, W, f, j);
      if (val(thx.at(C, 0, f, j)) < 1.0) nface++;
    }
  for (int g = 0; g < C.ext[2][1]; ++g)
    for (int i = 0; i < C.ext[2][0]; ++i) {
      thy.at(C, 0, i, g) = frozen ? real(C.frz->th_y[C.cid(2, i, g)]) : face_theta_y(C, W, i, g);
      if (val(thy.at(C, 0, i, g)) < 1.0) nface++;
    }
  st[ST_FACE_THETA_LT1] += nface;
  ghost_fill(C, thx, 1);
  ghost_fill(C, thy, 2);
  auto thetas = [&](int i, int j, real th[4]) {
    th[0] = thx.at(C, 0, i, j); th[1] = thx.at(C, 0, i + 1, j);
    th[2] = thy.at(C, 0, i, j); th[3] = thy.at(C, 0, i, j + 1);
  };
#ifndef AF_ORACLE_COUNT
#pragma omp parallel for schedule(static)
#endif
  for (int j = 0; j < C.ny; ++j)
    for (int i = 0; i < C.nx; ++i) {
      real th[4], out[8];
      thetas(i, j, th);
      cell_value(C, W, th, i, j, out);
      for (int k = 0; k < 8; ++k) W.FE[0].at(C, k, i, j) = out[k];
    }
  // Remark 4.1 round-off safeguard, sequential in cell order (Reading: the
  // four face coefficients of a non-admissible cell are lowered to
  // max(0, theta - 2^m 1e-8), m = 0..9, else set to 0; the cells sharing a
  // lowered face are recomputed).
  long long nshrink = 0, nbad = 0;
  for (int j = 0; j < C.ny && !frozen; ++j)
    for (int i = 0; i < C.nx; ++i) {
      real cur[8];
      for (int k = 0; k < 8; ++k) cur[k] = W.FE[0].at(C, k, i, j);
      if (in_G(cur, C.gamma)) continue;
      nshrink++;
      real th0[4];
      thetas(i, j, th0);
      bool ok = false;
      for (int m = 0; m <= 10 && !ok; ++m) {
        real th[4];
        for (int I = 0; I < 4; ++I) th[I] = (m < 10) ? rmax(real(0.0), th0[I] - real(std::ldexp(1e-8, m))) : real(0.0);
        real out[8];
        cell_value(C, W, th, i, j, out);
        ok = in_G(out, C.gamma) || m == 10;
        if (ok) {
          thx.at(C, 0, i, j) = th[0]; thx.at(C, 0, i + 1, j) = th[1];
          thy.at(C, 0, i, j) = th[2]; thy.at(C, 0, i, j + 1) = th[3];
          for (int k = 0; k < 8; ++k) W.FE[0].at(C, k, i, j) = out[k];
          if (!in_G(out, C.gamma)) nbad++;
        }
      }
      // keep periodic images of the changed faces in step
      ghost_fill(C, thx, 1);
      ghost_fill(C, thy, 2);
      const int nb[4][2] = {{i - 1, j}, {i + 1, j}, {i, j - 1}, {i, j + 1}};
      for (int q = 0; q < 4; ++q) {
        int ii = nb[q][0], jj = nb[q][1];
        if (C.bc == 1 && (ii < 0 || ii >= C.nx || jj < 0 || jj >= C.ny)) continue;
        ii = imod(ii, C.nx); jj = imod(jj, C.ny);
        real t2[4], o2[8];
        thetas(ii, jj, t2);
        cell_value(C, W, t2, ii, jj, o2);
        for (int k = 0; k < 8; ++k) W.FE[0].at(C, k, ii, jj) = o2[k];
      }
    }
  if (C.rec && C.rec->th_x && C.rec->th_y) {
    for (int j = 0; j < C.ext[1][1]; ++j)
      for (int f = 0; f < C.ext[1][0]; ++f) C.rec->th_x[C.cid(1, f, j)] = val(thx.at(C, 0, f, j));
    for (int g = 0; g < C.ext[2][1]; ++g)
      for (int i = 0; i < C.ext[2][0]; ++i) C.rec->th_y[C.cid(2, i, g)] = val(thy.at(C, 0, i, g));
  }
  st[ST_SHRINK] += nshrink;
  st[ST_CELL_SHRINK] += nshrink;
  st[ST_NONADMISSIBLE] += nbad;
}

// A16, Reading: dt = cfl / (max_sigma varrho_1(U_sigma)/dx + max_sigma varrho_2(U_sigma)/dy)
// over all four DoF classes (the paper prints no explicit formula).
static real compute_dt(const Ctx &C, State &S) {
  set_phase(PH_DT);
  real m1 = real(0.0), m2 = real(0.0);
  for (int cls = 0; cls < 4; ++cls)
    for (int j = 0; j < C.ext[cls][1]; ++j)
      for (int i = 0; i < C.ext[cls][0]; ++i) {
        real U[8];
        S.get(C, cls, i, j, U);
        PD d;
        point_data(U, C.gamma, d);
        m1 = rmax(m1, d.sr[0]);
        m2 = rmax(m2, d.sr[1]);
      }
  return real(C.cfl) / (m1 / real(C.dx) + m2 / real(C.dy));
}

// One forward-Euler stage with all limiters, followed by the SSP-RK3 convex
// combination out = a Un + b FE(Us).
static int stage(const Ctx &C, State &Un, State &Us, real dt, real a, real b, State &out, long long *st) {
  Work W;
  for (int cls = 0; cls < 4; ++cls) ghost_fill_state(C, Us.c[cls], cls);
  compute_point_data(C, Us, W);
  compute_centers(C, Us, W, st);
  point_ho_updates(C, dt, W);
  point_limit(C, dt, W, st);
  compute_sensor(C, W);
  compute_faces(C, W, st);
  cell_update(C, dt, W, st);
  cell_final(C, W, st);
  set_phase(PH_RK);
  out.init(C);
  for (int cls = 0; cls < 4; ++cls) {
    int ex = C.ext[cls][0], ey = C.ext[cls][1];
    for (int k = 0; k < 8; ++k)
      for (int j = 0; j < ey; ++j)
        for (int i = 0; i < ex; ++i) {
          real fe = W.FE[cls].at(C, k, i, j);
          real o = (val(a) == 0.0) ? fe : a * Un.c[cls].at(C, k, i, j) + b * fe;
          out.c[cls].at(C, k, i, j) = o;
        }
  }
  return 0;
}

// The unlimited semi-discrete operator L(U): the high-order cell-average and
// point-value right-hand sides (Sec. 2.2, 2.3) with the cell-centre limiter
// of Remark 3.2 (no shock sensor, no PP limiting).
static void rhs(const Ctx &C, State &S, State &out) {
  Work W;
  long long st[ST_NSTATS] = {0};
  for (int cls = 0; cls < 4; ++cls) ghost_fill_state(C, S.c[cls], cls);
  compute_point_data(C, S, W);
  compute_centers(C, S, W, st);
  out.init(C);
  const double dx = C.dx, dy = C.dy;
  for (int cls = 1; cls < 4; ++cls)
    for (int j = 0; j < C.ext[cls][1]; ++j)
      for (int i = 0; i < C.ext[cls][0]; ++i) {
        real d1[8], d2[8], dB1, dB2;
        const PD &me = W.pd[cls].at(C, i, j);
        if (cls == 3) {
          const PD *Px[5] = {&W.pd[3].at(C, i - 1, j), &W.pd[2].at(C, i - 1, j), &me, &W.pd[2].at(C, i, j), &W.pd[3].at(C, i + 1, j)};
          const PD *Py[5] = {&W.pd[3].at(C, i, j - 1), &W.pd[1].at(C, i, j - 1), &me, &W.pd[1].at(C, i, j), &W.pd[3].at(C, i, j + 1)};
          fvs_derivative(0, Px, dx, d1, dB1, upwind_sign(C, me, 0));
          fvs_derivative(1, Py, dy, d2, dB2, upwind_sign(C, me, 1));
        } else if (cls == 1) {
          const PD *Px[5] = {&W.pd[1].at(C, i - 1, j), &W.pdc.at(C, i - 1, j), &me, &W.pdc.at(C, i, j), &W.pd[1].at(C, i + 1, j)};
          fvs_derivative(0, Px, dx, d1, dB1, upwind_sign(C, me, 0));
          const PD &lo = W.pd[3].at(C, i, j), &hi = W.pd[3].at(C, i, j + 1);
          for (int k = 0; k < 8; ++k) d2[k] = Dcen(lo.F[1][k], hi.F[1][k], dy);
          dB2 = Dcen(lo.B[1], hi.B[1], dy);
        } else {
          const PD &lo = W.pd[3].at(C, i, j), &hi = W.pd[3].at(C, i + 1, j);
          for (int k = 0; k < 8; ++k) d1[k] = Dcen(lo.F[0][k], hi.F[0][k], dx);
          dB1 = Dcen(lo.B[0], hi.B[0], dx);
          const PD *Py[5] = {&W.pd[2].at(C, i, j - 1), &W.pdc.at(C, i, j - 1), &me, &W.pdc.at(C, i, j), &W.pd[2].at(C, i, j + 1)};
          fvs_derivative(1, Py, dy, d2, dB2, upwind_sign(C, me, 1));
        }
        real divB = dB1 + dB2, Ps[8];
        psi(me, Ps);
        for (int k = 0; k < 8; ++k) {
          real r = real(0.0) - d1[k] - d2[k];
          if (C.src_point_on) r = r - divB * Ps[k];
          out.c[cls].at(C, k, i, j) = r;
        }
      }
  for (int j = 0; j < C.ny; ++j)
    for (int i = 0; i < C.nx; ++i) {
      real Sv[8];
      cell_source(C, W, i, j, Sv);
      if (!C.src_cell_on) for (int k = 0; k < 8; ++k) Sv[k] = real(0.0);
      for (int k = 0; k < 8; ++k) {
        // Simpson fluxes on the four faces of the cell (Sec. 2.2)
        real FL = (W.pd[3].at(C, i, j).F[0][k] + real(4.0) * W.pd[1].at(C, i, j).F[0][k] + W.pd[3].at(C, i, j + 1).F[0][k]) / real(6.0);
        real FR = (W.pd[3].at(C, i + 1, j).F[0][k] + real(4.0) * W.pd[1].at(C, i + 1, j).F[0][k] + W.pd[3].at(C, i + 1, j + 1).F[0][k]) / real(6.0);
        real FD = (W.pd[3].at(C, i, j).F[1][k] + real(4.0) * W.pd[2].at(C, i, j).F[1][k] + W.pd[3].at(C, i + 1, j).F[1][k]) / real(6.0);
        real FU = (W.pd[3].at(C, i, j + 1).F[1][k] + real(4.0) * W.pd[2].at(C, i, j + 1).F[1][k] + W.pd[3].at(C, i + 1, j + 1).F[1][k]) / real(6.0);
        out.c[0].at(C, k, i, j) = real(0.0) - (FR - FL) / real(dx) - (FU - FD) / real(dy) - Sv[k];
      }
    }
}

// ---------------------------------------------------------------------------
// C ABI used by the test-suite (ctypes).
// ---------------------------------------------------------------------------
// ===========================================================================
// The 1D AF scheme (Sec. 4: the 1D tests use the 1D AF scheme with the LLF
// FVS and without the Godunov-Powell source).  Reading: the scheme of
// Sec. 2-3 restricted to one dimension.  Degrees of freedom: cell averages
// and the point values at the interfaces (point f at x0 + f dx, the left face
// of cell f).  Per stage:
//   - centre value of the cell parabola, (6 Ubar - U_L - U_R)/4 (Simpson),
//     limited as in Remark 3.2;
//   - point update by the LLF FVS on the line (point f-1, centre f-1,
//     point f, centre f, point f+1), alpha = max varrho_1 on the line;
//   - the Sec. 3.3 point limiter, its LLF state from the LLF fluxes between
//     point f and its neighbouring points f-1, f+1;
//   - the Sec. 3.4 sensor with every y-difference zero;
//   - cell averages: the face flux is F1 of the face point value, blended
//     with the LLF flux between the adjacent averages by theta^s; the flux
//     limiter of Sec. 3.2 with the two faces L, R (no source, so
//     U^{Lim,1} = U^LLF), face theta = min of the adjacent Lambda, and the
//     round-off shrink of Remark 4.1;
//   - SSP-RK3, dt = cfl dx / max varrho_1 over averages and points.
// Boundaries as in 2D: periodic, or outflow mirrors across the boundary face.
// ===========================================================================
struct Ctx1 {
  int n, nf, bc;
  double dx, gamma, cfl, kappa;
  int pp_on;
};

static void make_ctx1(const or_params *p, int n, Ctx1 &C) {
  C.n = n; C.nf = p->bc == 0 ? n : n + 1; C.bc = p->bc;
  C.dx = (p->x1 - p->x0) / n; C.gamma = p->gamma; C.cfl = p->cfl; C.kappa = p->kappa; C.pp_on = p->pp_on;
}

// ncomp components on an index range [-G, len + G)
struct Arr1 {
  int nc = 0, len = 0;
  std::vector<real> a;
  void init(int ncomp, int n) { nc = ncomp; len = n; a.assign((size_t)nc * (n + 2 * G), real(0.0)); }
  real &at(int k, int i) { return a[(size_t)k * (len + 2 * G) + (size_t)(i + G)]; }
};
// kind 0: cell index set (len n), kind 1: point index set (len nf)
static void ghost_fill1(const Ctx1 &C, Arr1 &A, int kind) {
  for (int i = -G; i < A.len + G; ++i) {
    if (i >= 0 && i < A.len) continue;
    int si = map_idx(i, C.n, kind, C.bc);
    for (int k = 0; k < A.nc; ++k) A.at(k, i) = A.at(k, si);
  }
}
struct PD1 {
  int len = 0;
  std::vector<PD> d;
  void init(int n) { len = n; d.assign((size_t)(n + 2 * G), PD()); }
  PD &at(int i) { return d[(size_t)(i + G)]; }
};
static void pd_fill1(const Ctx1 &C, Arr1 &U, PD1 &P) {
  P.init(U.len);
  for (int i = -G; i < U.len + G; ++i) {
    real u[8];
    for (int k = 0; k < 8; ++k) u[k] = U.at(k, i);
    point_data(u, C.gamma, P.at(i));
  }
}

static real compute_dt1(const Ctx1 &C, Arr1 &A, Arr1 &P) {
  set_phase(PH_DT);
  real m = real(0.0);
  Arr1 *S[2] = {&A, &P};
  for (int c = 0; c < 2; ++c)
    for (int i = 0; i < S[c]->len; ++i) {
      real u[8];
      for (int k = 0; k < 8; ++k) u[k] = S[c]->at(k, i);
      PD d;
      point_data(u, C.gamma, d);
      m = rmax(m, d.sr[0]);
    }
  return real(C.cfl) / (m / real(C.dx));
}

// One limited forward-Euler stage of the 1D scheme and the RK combination
// out = a Un + b FE(Us) for the averages (A) and the point values (P).
static void stage1(const Ctx1 &C, Arr1 &An, Arr1 &Pn, Arr1 &As, Arr1 &Ps, real dt, real a, real b, Arr1 &Ao, Arr1 &Po,
                   long long *st) {
  const double dx = C.dx;
  ghost_fill1(C, As, 0);
  ghost_fill1(C, Ps, 1);
  set_phase(PH_POINTDATA);
  PD1 pa, pp, pc;
  pd_fill1(C, As, pa);
  pd_fill1(C, Ps, pp);
  // centre values (Simpson on the cell parabola) + Remark 3.2
  set_phase(PH_CENTER);
  Arr1 Uc;
  Uc.init(8, C.n);
  for (int i = 0; i < C.n; ++i) {
    real avg[8], uc[8], out[8], t1, t2;
    for (int k = 0; k < 8; ++k) {
      avg[k] = As.at(k, i);
      uc[k] = (real(6.0) * avg[k] - Ps.at(k, i) - Ps.at(k, i + 1)) / real(4.0);
    }
    scaling_limiter(uc, avg, C.gamma, out, t1, t2);
    if (t1 < real(1.0) || t2 < real(1.0)) st[ST_CENTER_LIMITED]++;
    for (int k = 0; k < 8; ++k) Uc.at(k, i) = out[k];
  }
  ghost_fill1(C, Uc, 0);
  set_phase(PH_POINTDATA);
  pd_fill1(C, Uc, pc);
  // point values: LLF FVS, then the Sec. 3.3 limiter
  Arr1 PF;
  PF.init(8, C.nf);
  for (int f = 0; f < C.nf; ++f) {
    set_phase(PH_POINT_HO);
    const PD &me = pp.at(f);
    const PD *L[5] = {&pp.at(f - 1), &pc.at(f - 1), &me, &pc.at(f), &pp.at(f + 1)};
    real d1[8], dB1, UH[8];
    fvs_derivative(0, L, dx, d1, dB1);
    for (int k = 0; k < 8; ++k) UH[k] = me.U[k] + dt * (real(0.0) - d1[k]);
    real out[8];
    if (!C.pp_on) {
      for (int k = 0; k < 8; ++k) out[k] = UH[k];
    } else {
      set_phase(PH_POINT_PP);
      real Fr[8], Fl[8], UL[8], t1, t2;
      llf_flux(0, me, pp.at(f + 1), Fr, nullptr);
      llf_flux(0, pp.at(f - 1), me, Fl, nullptr);
      for (int k = 0; k < 8; ++k) UL[k] = me.U[k] - dt / real(dx) * (Fr[k] - Fl[k]);
      scaling_limiter(UH, UL, C.gamma, out, t1, t2);
      if (t1 < real(1.0) || t2 < real(1.0)) st[ST_POINT_LIMITED]++;
      if (!in_G(out, C.gamma)) {   // Remark 4.1, as in 2D
        st[ST_SHRINK]++;
        real Us[8];
        for (int k = 0; k < 8; ++k) Us[k] = UH[k];
        Us[0] = t1 * UH[0] + (real(1.0) - t1) * UL[0];
        bool ok = false;
        for (int m = 0; m < 10 && !ok; ++m) {
          real th = rmax(real(0.0), t2 - real(std::ldexp(1e-8, m)));
          for (int k = 0; k < 8; ++k) out[k] = th * Us[k] + (real(1.0) - th) * UL[k];
          ok = in_G(out, C.gamma);
        }
        if (!ok) for (int k = 0; k < 8; ++k) out[k] = UL[k];
        if (!in_G(out, C.gamma)) st[ST_NONADMISSIBLE]++;
      }
    }
    for (int k = 0; k < 8; ++k) PF.at(k, f) = out[k];
  }
  // sensor phi on cells [-1, n] (y-differences zero)
  set_phase(PH_SENSOR_PHI);
  Arr1 phi;
  phi.init(3, C.n);
  for (int i = -1; i <= C.n; ++i) {
    real ph[4];
    const PD &c = pa.at(i);
    sensor_phi(c, pa.at(i + 1), pa.at(i - 1), c, c, dx, dx, ph);
    phi.at(0, i) = ph[0];
    phi.at(1, i) = ph[2];
    phi.at(2, i) = ph[3];
  }
  // faces: F1 of the point value, LLF flux between the adjacent averages, theta^s
  set_phase(PH_FACE);
  Arr1 Fh, Fl, ts, al;
  Fh.init(8, C.nf); Fl.init(8, C.nf); ts.init(1, C.nf); al.init(1, C.nf);
  for (int f = 0; f < C.nf; ++f) {
    real F[8], alpha;
    llf_flux(0, pa.at(f - 1), pa.at(f), F, &alpha);
    for (int k = 0; k < 8; ++k) {
      Fh.at(k, f) = pp.at(f).F[0][k];
      Fl.at(k, f) = F[k];
    }
    al.at(0, f) = alpha;
    set_phase(PH_SENSOR_THETA);
    real t = real(1.0);
    if (C.kappa != 0.0) {
      real p1 = rmax(phi.at(0, f - 1), phi.at(0, f)), p2 = rmax(phi.at(1, f - 1), phi.at(1, f));
      real p3 = rmax(phi.at(2, f - 1), phi.at(2, f));
      t = exp(real(0.0) - real(C.kappa) * (p1 * p2 + p3));
    }
    ts.at(0, f) = t;
    if (val(t) < 0.99) st[ST_SENSOR_LT099]++;
    set_phase(PH_FACE);
  }
  ghost_fill1(C, Fh, 1);
  ghost_fill1(C, Fl, 1);
  ghost_fill1(C, ts, 1);
  ghost_fill1(C, al, 1);
  // cell averages
  set_phase(PH_CELL_UPDATE);
  Arr1 AF, L1, H, Lam;
  AF.init(8, C.n); L1.init(8, C.n); H.init(16, C.n); Lam.init(2, C.n);
  NewtonLog nl;
  for (int i = 0; i < C.n; ++i) {
    real Fss[2][8], Fll[2][8];
    for (int I = 0; I < 2; ++I)
      for (int k = 0; k < 8; ++k) {
        const int f = i + I;
        Fll[I][k] = Fl.at(k, f);
        Fss[I][k] = (C.kappa == 0.0) ? Fh.at(k, f) : ts.at(0, f) * Fh.at(k, f) + (real(1.0) - ts.at(0, f)) * Fll[I][k];
      }
    if (!C.pp_on) {
      for (int k = 0; k < 8; ++k) AF.at(k, i) = As.at(k, i) - dt / real(dx) * (Fss[1][k] - Fss[0][k]);
      continue;
    }
    real Ullf[8];
    for (int k = 0; k < 8; ++k) Ullf[k] = As.at(k, i) - dt / real(dx) * (Fll[1][k] - Fll[0][k]);
    // Lemma 3.1 CFL condition restricted to x (diagnostic only)
    if (val(dt * (al.at(0, i) / real(dx) + al.at(0, i + 1) / real(dx))) > 1.0 + 1e-12) st[ST_CFL_VIOLATIONS]++;
    real eps_rho = rmin(real(1e-13), Ullf[0]);
    real eps_p = rmin(real(1e-13), pressure(Ullf, C.gamma));
    real Hb[4][8];
    for (int k = 0; k < 8; ++k) {
      Hb[0][k] = dt / real(dx) * (Fss[0][k] - Fll[0][k]);
      Hb[1][k] = real(0.0) - dt / real(dx) * (Fss[1][k] - Fll[1][k]);
      Hb[2][k] = real(0.0);
      Hb[3][k] = real(0.0);
    }
    real lam[4];
    flux_limiter_box(Ullf, Hb, eps_rho, eps_p, C.gamma, lam, nl);   // the zero directions leave 4 vertices
    if (lam[0] < real(1.0) || lam[1] < real(1.0)) st[ST_LAMBDA_LT1]++;
    for (int k = 0; k < 8; ++k) {
      L1.at(k, i) = Ullf[k];
      H.at(k, i) = Hb[0][k];
      H.at(8 + k, i) = Hb[1][k];
    }
    Lam.at(0, i) = lam[0];
    Lam.at(1, i) = lam[1];
  }
  st[ST_NEWTON_SOLVES] += nl.solves;
  st[ST_NEWTON_MAXIT] = std::max<long long>(st[ST_NEWTON_MAXIT], nl.maxit);
  if (C.pp_on) {
    set_phase(PH_CELL_FINAL);
    ghost_fill1(C, Lam, 0);
    Arr1 th;
    th.init(1, C.nf);
    for (int f = 0; f < C.nf; ++f) {
      if (C.bc == 1 && f == 0) th.at(0, f) = Lam.at(0, 0);
      else if (C.bc == 1 && f == C.n) th.at(0, f) = Lam.at(1, C.n - 1);
      else th.at(0, f) = rmin(Lam.at(1, f - 1), Lam.at(0, f));
      if (val(th.at(0, f)) < 1.0) st[ST_FACE_THETA_LT1]++;
    }
    ghost_fill1(C, th, 1);
    auto value = [&](int i, real tl, real tr, real *out) {
      for (int k = 0; k < 8; ++k) out[k] = L1.at(k, i) + tl * H.at(k, i) + tr * H.at(8 + k, i);
    };
    for (int i = 0; i < C.n; ++i) {
      real out[8];
      value(i, th.at(0, i), th.at(0, i + 1), out);
      for (int k = 0; k < 8; ++k) AF.at(k, i) = out[k];
    }
    // Remark 4.1, in cell order; neighbours sharing a lowered face are recomputed
    for (int i = 0; i < C.n; ++i) {
      real cur[8];
      for (int k = 0; k < 8; ++k) cur[k] = AF.at(k, i);
      if (in_G(cur, C.gamma)) continue;
      st[ST_SHRINK]++;
      st[ST_CELL_SHRINK]++;
      const real t0[2] = {th.at(0, i), th.at(0, i + 1)};
      for (int m = 0; m <= 10; ++m) {
        real t[2], out[8];
        for (int I = 0; I < 2; ++I) t[I] = (m < 10) ? rmax(real(0.0), t0[I] - real(std::ldexp(1e-8, m))) : real(0.0);
        value(i, t[0], t[1], out);
        if (in_G(out, C.gamma) || m == 10) {
          th.at(0, i) = t[0];
          th.at(0, i + 1) = t[1];
          for (int k = 0; k < 8; ++k) AF.at(k, i) = out[k];
          if (!in_G(out, C.gamma)) st[ST_NONADMISSIBLE]++;
          break;
        }
      }
      ghost_fill1(C, th, 1);
      for (int q = -1; q <= 1; q += 2) {
        int ii = i + q;
        if (C.bc == 1 && (ii < 0 || ii >= C.n)) continue;
        ii = imod(ii, C.n);
        real o2[8];
        value(ii, th.at(0, ii), th.at(0, ii + 1), o2);
        for (int k = 0; k < 8; ++k) AF.at(k, ii) = o2[k];
      }
    }
  }
  set_phase(PH_RK);
  Ao.init(8, C.n);
  Po.init(8, C.nf);
  for (int k = 0; k < 8; ++k) {
    for (int i = 0; i < C.n; ++i) Ao.at(k, i) = (val(a) == 0.0) ? AF.at(k, i) : a * An.at(k, i) + b * AF.at(k, i);
    for (int f = 0; f < C.nf; ++f) Po.at(k, f) = (val(a) == 0.0) ? PF.at(k, f) : a * Pn.at(k, f) + b * PF.at(k, f);
  }
}

static void load1(const Ctx1 &C, const double *const *U, Arr1 &A, Arr1 &P) {
  A.init(8, C.n);
  P.init(8, C.nf);
  for (int k = 0; k < 8; ++k) {
    for (int i = 0; i < C.n; ++i) A.at(k, i) = real(U[0][(size_t)k * C.n + i]);
    for (int f = 0; f < C.nf; ++f) P.at(k, f) = real(U[1][(size_t)k * C.nf + f]);
  }
}
static void store1(const Ctx1 &C, Arr1 &A, Arr1 &P, double *const *U) {
  for (int k = 0; k < 8; ++k) {
    for (int i = 0; i < C.n; ++i) U[0][(size_t)k * C.n + i] = val(A.at(k, i));
    for (int f = 0; f < C.nf; ++f) U[1][(size_t)k * C.nf + f] = val(P.at(k, f));
  }
}

extern "C" {

int or_sizes(int nx, int ny, int bc, int cls, int *nxp, int *nyp) {
  if (cls < 0 || cls > 3) return -1;
  int fx = (bc == 0) ? nx : nx + 1, fy = (bc == 0) ? ny : ny + 1;
  *nxp = (cls == 1 || cls == 3) ? fx : nx;
  *nyp = (cls == 2 || cls == 3) ? fy : ny;
  return 0;
}

double or_dt(const or_params *p, int nx, int ny, const double *const *U) {
  Ctx C;
  make_ctx(p, nx, ny, C);
  State S;
  load_state(C, U, S);
  return val(compute_dt(C, S));
}

// out = a * Un + b * FE(Us, dt); stats accumulate into st[ST_NSTATS].
int or_stage(const or_params *p, int nx, int ny, const double *const *Un, const double *const *Us, double dt,
             double a, double b, double *const *out, long long *st) {
  Ctx C;
  make_ctx(p, nx, ny, C);
  State Sn, Ss, So;
  load_state(C, Un, Sn);
  load_state(C, Us, Ss);
  long long loc[ST_NSTATS] = {0};
  stage(C, Sn, Ss, real(dt), real(a), real(b), So, loc);
  store_state(C, So, out);
  if (st) for (int k = 0; k < ST_NSTATS; ++k) st[k] = (k == ST_NEWTON_MAXIT) ? std::max(st[k], loc[k]) : st[k] + loc[k];
  return 0;
}

// or_stage that also writes the limiter coefficients it took into *rec, or,
// given *frz, takes them from there (either may be NULL; see or_coeffs).
int or_stage_rec(const or_params *p, int nx, int ny, const double *const *Un, const double *const *Us, double dt,
                 double a, double b, double *const *out, long long *st, const or_coeffs *rec, const or_coeffs *frz) {
  Ctx C;
  make_ctx(p, nx, ny, C);
  C.rec = rec;
  C.frz = frz;
  State Sn, Ss, So;
  load_state(C, Un, Sn);
  load_state(C, Us, Ss);
  long long loc[ST_NSTATS] = {0};
  stage(C, Sn, Ss, real(dt), real(a), real(b), So, loc);
  store_state(C, So, out);
  if (st) for (int k = 0; k < ST_NSTATS; ++k) st[k] = (k == ST_NEWTON_MAXIT) ? std::max(st[k], loc[k]) : st[k] + loc[k];
  return 0;
}

// One SSP-RK3 step in place.  dt_in > 0 fixes dt; otherwise dt comes from U^n.
// The three stages use the Shu-Osher coefficients (a,b) = (0,1), (3/4,1/4), (1/3,2/3).
int or_step(const or_params *p, int nx, int ny, double *const *U, double dt_in, double *dt_used, long long *st) {
  Ctx C;
  make_ctx(p, nx, ny, C);
  State Sn;
  load_state(C, U, Sn);
  real dt = (dt_in > 0.0) ? real(dt_in) : compute_dt(C, Sn);
  long long loc[ST_NSTATS] = {0};
  State S1, S2, S3;
  stage(C, Sn, Sn, dt, real(0.0), real(1.0), S1, loc);
  stage(C, Sn, S1, dt, real(3.0) / real(4.0), real(1.0) / real(4.0), S2, loc);
  stage(C, Sn, S2, dt, real(1.0) / real(3.0), real(2.0) / real(3.0), S3, loc);
  store_state(C, S3, U);
  if (dt_used) *dt_used = val(dt);
  if (st) for (int k = 0; k < ST_NSTATS; ++k) st[k] = (k == ST_NEWTON_MAXIT) ? std::max(st[k], loc[k]) : st[k] + loc[k];
  return 0;
}

// Unlimited semi-discrete right-hand side L(U) of all four classes.
int or_rhs(const or_params *p, int nx, int ny, const double *const *U, double *const *dUdt) {
  Ctx C;
  make_ctx(p, nx, ny, C);
  State S, O;
  load_state(C, U, S);
  rhs(C, S, O);
  store_state(C, O, dUdt);
  return 0;
}

// Shock-sensor coefficients theta^s (Sec. 3.4) of the state U: x-faces
// [ny][nxf] and y-faces [nyf][nx] (class-1 and class-2 extents).
int or_sensor(const or_params *p, int nx, int ny, const double *const *U, double *ths_x, double *ths_y) {
  Ctx C;
  make_ctx(p, nx, ny, C);
  State S;
  load_state(C, U, S);
  long long st[ST_NSTATS] = {0};
  Work W;
  for (int cls = 0; cls < 4; ++cls) ghost_fill_state(C, S.c[cls], cls);
  compute_point_data(C, S, W);
  compute_sensor(C, W);
  compute_faces(C, W, st);
  for (int j = 0; j < C.ext[1][1]; ++j)
    for (int f = 0; f < C.ext[1][0]; ++f) ths_x[(size_t)j * C.ext[1][0] + f] = val(W.fx.at(C, 16, f, j));
  for (int g = 0; g < C.ext[2][1]; ++g)
    for (int i = 0; i < C.ext[2][0]; ++i) ths_y[(size_t)g * C.ext[2][0] + i] = val(W.fy.at(C, 16, i, g));
  return 0;
}

// Example 4.4: the two discrete divergence measures of the state U.
//   out[0] = sum_ij sum_{l,m} |(div B)_ij^{l,m}| w_l w_m dx dy, the node
//            divergences of eq. (semi_av_src) (centre node: the limited
//            centre value, as in the stage);
//   out[1] = sum_ij |closed integral of B.n over the boundary of cell ij|,
//            each edge by Simpson's rule: dy/6 ([R] - [L]) + dx/6 ([T] - [B]),
//            [.] = corner + 4 face centre + corner of B1 (R, L) or B2 (T, B).
//            Reading: the text defines this measure as the edge integral of
//            B.n; the printed sum carries a factor dx dy instead of the edge
//            lengths, which is the same only up to a factor h on a square
//            mesh, so the edge integral is taken.
int or_divb(const or_params *p, int nx, int ny, const double *const *U, double *out) {
  Ctx C;
  make_ctx(p, nx, ny, C);
  State S;
  load_state(C, U, S);
  for (int cls = 0; cls < 4; ++cls) ghost_fill_state(C, S.c[cls], cls);
  Work W;
  long long st[ST_NSTATS] = {0};
  compute_centers(C, S, W, st);
  const real w[3] = {real(1.0) / real(6.0), real(2.0) / real(3.0), real(1.0) / real(6.0)};
  real d1 = real(0.0), d2 = real(0.0);
  for (int j = 0; j < C.ny; ++j)
    for (int i = 0; i < C.nx; ++i) {
      // node values N[l][m] of B1 (q = 4) and B2 (q = 5), l along x, m along y
      real b[2][3][3];
      for (int q = 0; q < 2; ++q) {
        const int k = 4 + q;
        b[q][0][0] = S.c[3].at(C, k, i, j);     b[q][1][0] = S.c[2].at(C, k, i, j);     b[q][2][0] = S.c[3].at(C, k, i + 1, j);
        b[q][0][1] = S.c[1].at(C, k, i, j);     b[q][1][1] = W.Uc.at(C, k, i, j);      b[q][2][1] = S.c[1].at(C, k, i + 1, j);
        b[q][0][2] = S.c[3].at(C, k, i, j + 1); b[q][1][2] = S.c[2].at(C, k, i, j + 1); b[q][2][2] = S.c[3].at(C, k, i + 1, j + 1);
      }
      for (int l = 0; l < 3; ++l)
        for (int m = 0; m < 3; ++m) {
          real dB1, dB2;
          if (l == 0) dB1 = Dminus(b[0][0][m], b[0][1][m], b[0][2][m], C.dx);
          else if (l == 1) dB1 = Dcen(b[0][0][m], b[0][2][m], C.dx);
          else dB1 = Dplus(b[0][0][m], b[0][1][m], b[0][2][m], C.dx);
          if (m == 0) dB2 = Dminus(b[1][l][0], b[1][l][1], b[1][l][2], C.dy);
          else if (m == 1) dB2 = Dcen(b[1][l][0], b[1][l][2], C.dy);
          else dB2 = Dplus(b[1][l][0], b[1][l][1], b[1][l][2], C.dy);
          d1 = d1 + fabs(dB1 + dB2) * w[l] * w[m] * real(C.dx * C.dy);
        }
      const real right = b[0][2][0] + real(4.0) * b[0][2][1] + b[0][2][2];
      const real left = b[0][0][0] + real(4.0) * b[0][0][1] + b[0][0][2];
      const real top = b[1][0][2] + real(4.0) * b[1][1][2] + b[1][2][2];
      const real bottom = b[1][0][0] + real(4.0) * b[1][1][0] + b[1][2][0];
      d2 = d2 + fabs(real(C.dy) * (right - left) + real(C.dx) * (top - bottom)) / real(6.0);
    }
  out[0] = val(d1);
  out[1] = val(d2);
  return 0;
}

// ---- pointwise pieces, exported for the unit tests --------------------------
void or_flux(int l, const double *U, double gamma, double *F) {
  real u[8];
  for (int k = 0; k < 8; ++k) u[k] = U[k];
  PD d;
  point_data(u, gamma, d);
  for (int k = 0; k < 8; ++k) F[k] = val(d.F[l - 1][k]);
}
double or_pressure(const double *U, double gamma) {
  real u[8];
  for (int k = 0; k < 8; ++k) u[k] = U[k];
  return val(pressure(u, gamma));
}
double or_fast_speed(int l, const double *U, double gamma) {
  real u[8];
  for (int k = 0; k < 8; ++k) u[k] = U[k];
  PD d;
  point_data(u, gamma, d);
  return val(d.cf[l - 1]);
}
double or_spectral_radius(int l, const double *U, double gamma) {
  real u[8];
  for (int k = 0; k < 8; ++k) u[k] = U[k];
  PD d;
  point_data(u, gamma, d);
  return val(d.sr[l - 1]);
}
double or_llf_flux(int l, const double *U, const double *V, double gamma, double *F) {
  real u[8], v[8], f[8], al;
  for (int k = 0; k < 8; ++k) { u[k] = U[k]; v[k] = V[k]; }
  PD a, b;
  point_data(u, gamma, a);
  point_data(v, gamma, b);
  llf_flux(l - 1, a, b, f, &al);
  for (int k = 0; k < 8; ++k) F[k] = val(f[k]);
  return val(al);
}
// Bi-parabola centre value: faces[4][8] = L,R,D,U; corners[4][8] = DL,DR,UL,UR.
void or_center_value(const double *avg, const double *faces, const double *corners, double *out) {
  real a[8], f[4][8], c[4][8], o[8];
  for (int k = 0; k < 8; ++k) {
    a[k] = avg[k];
    for (int q = 0; q < 4; ++q) { f[q][k] = faces[q * 8 + k]; c[q][k] = corners[q * 8 + k]; }
  }
  center_value(a, f[0], f[1], f[2], f[3], c[0], c[1], c[2], c[3], o);
  for (int k = 0; k < 8; ++k) out[k] = val(o[k]);
}
// FD operators along a line (values a, b, c; spacing h): out = {D+, D-, D}.
void or_fd(double a, double b, double c, double h, double *out) {
  out[0] = val(Dplus(a, b, c, h));
  out[1] = val(Dminus(a, b, c, h));
  out[2] = val(Dcen(a, c, h));
}
// Step (2) of the flux limiter: Lambda[4] for one cell.  H is [4][8] (L,R,D,U).
int or_flux_limiter(const double *lim1, const double *H, double eps_rho, double eps_p, double gamma,
                    double *Lam, int *newton_maxit) {
  real L1[8], h[4][8], lam[4];
  for (int k = 0; k < 8; ++k) {
    L1[k] = lim1[k];
    for (int I = 0; I < 4; ++I) h[I][k] = H[I * 8 + k];
  }
  NewtonLog nl;
  flux_limiter_box(L1, h, eps_rho, eps_p, gamma, lam, nl);
  for (int I = 0; I < 4; ++I) Lam[I] = val(lam[I]);
  if (newton_maxit) *newton_maxit = nl.maxit;
  return (int)nl.solves;
}
// Scaling limiter (Sec. 3.3): theta[2] = {theta*, theta**}.
void or_scaling_limiter(const double *UH, const double *UL, double gamma, double *out, double *theta) {
  real h[8], l[8], o[8], t1, t2;
  for (int k = 0; k < 8; ++k) { h[k] = UH[k]; l[k] = UL[k]; }
  scaling_limiter(h, l, gamma, o, t1, t2);
  for (int k = 0; k < 8; ++k) out[k] = val(o[k]);
  theta[0] = val(t1);
  theta[1] = val(t2);
}

// Shock-sensor values of one cell (Sec. 3.4): phi[4] = phi_1 (x), phi_1 (y),
// phi_2, phi_3 from the cell average c and its east/west/north/south neighbours.
void or_sensor_phi(const double *c, const double *e, const double *w, const double *n, const double *s,
                   double gamma, double dx, double dy, double *phi) {
  const double *src[5] = {c, e, w, n, s};
  PD d[5];
  for (int q = 0; q < 5; ++q) {
    real u[8];
    for (int k = 0; k < 8; ++k) u[k] = src[q][k];
    point_data(u, gamma, d[q]);
  }
  real ph[4];
  sensor_phi(d[0], d[1], d[2], d[3], d[4], dx, dy, ph);
  for (int q = 0; q < 4; ++q) phi[q] = val(ph[q]);
}

// ---- the 1D scheme (see the block above) ----------------------------------
// U[0]: averages [8][n], U[1]: point values [8][nf], nf = n (periodic) or n+1.
double or1d_dt(const or_params *p, int n, const double *const *U) {
  Ctx1 C;
  make_ctx1(p, n, C);
  Arr1 A, P;
  load1(C, U, A, P);
  return val(compute_dt1(C, A, P));
}

int or1d_stage(const or_params *p, int n, const double *const *Un, const double *const *Us, double dt, double a,
               double b, double *const *out, long long *st) {
  Ctx1 C;
  make_ctx1(p, n, C);
  Arr1 An, Pn, As, Ps, Ao, Po;
  load1(C, Un, An, Pn);
  load1(C, Us, As, Ps);
  long long loc[ST_NSTATS] = {0};
  stage1(C, An, Pn, As, Ps, real(dt), real(a), real(b), Ao, Po, loc);
  store1(C, Ao, Po, out);
  if (st) for (int k = 0; k < ST_NSTATS; ++k) st[k] = (k == ST_NEWTON_MAXIT) ? std::max(st[k], loc[k]) : st[k] + loc[k];
  return 0;
}

int or1d_step(const or_params *p, int n, double *const *U, double dt_in, double *dt_used, long long *st) {
  Ctx1 C;
  make_ctx1(p, n, C);
  Arr1 An, Pn, A1, P1, A2, P2, A3, P3;
  load1(C, U, An, Pn);
  real dt = (dt_in > 0.0) ? real(dt_in) : compute_dt1(C, An, Pn);
  long long loc[ST_NSTATS] = {0};
  stage1(C, An, Pn, An, Pn, dt, real(0.0), real(1.0), A1, P1, loc);
  stage1(C, An, Pn, A1, P1, dt, real(3.0) / real(4.0), real(1.0) / real(4.0), A2, P2, loc);
  stage1(C, An, Pn, A2, P2, dt, real(1.0) / real(3.0), real(2.0) / real(3.0), A3, P3, loc);
  store1(C, A3, P3, U);
  if (dt_used) *dt_used = val(dt);
  if (st) for (int k = 0; k < ST_NSTATS; ++k) st[k] = (k == ST_NEWTON_MAXIT) ? std::max(st[k], loc[k]) : st[k] + loc[k];
  return 0;
}

#ifdef AF_ORACLE_COMPLEX
// One SSP-RK3 step of the complex state (re[cls], im[cls]) (complex-step
// differentiation).  dt > 0: that fixed, real time step; dt <= 0: the step's
// own dt of the complex state (the A16 formula in complex arithmetic, the
// maxima taken by real part), so that the derivative includes d(dt)/dU.
int or_step_cs(const or_params *p, int nx, int ny, double *const *re, double *const *im, double dt) {
  Ctx C;
  make_ctx(p, nx, ny, C);
  State Sn;
  Sn.init(C);
  for (int cls = 0; cls < 4; ++cls) {
    int ex = C.ext[cls][0], ey = C.ext[cls][1];
    for (int k = 0; k < 8; ++k)
      for (int j = 0; j < ey; ++j)
        for (int i = 0; i < ex; ++i) {
          const size_t o = ((size_t)k * ey + j) * ex + i;
          Sn.c[cls].at(C, k, i, j) = Cx(re[cls][o], im[cls][o]);
        }
  }
  long long loc[ST_NSTATS] = {0};
  State S1, S2, S3;
  const real h = dt > 0.0 ? real(dt) : compute_dt(C, Sn);
  stage(C, Sn, Sn, h, real(0.0), real(1.0), S1, loc);
  stage(C, Sn, S1, h, real(3.0) / real(4.0), real(1.0) / real(4.0), S2, loc);
  stage(C, Sn, S2, h, real(1.0) / real(3.0), real(2.0) / real(3.0), S3, loc);
  for (int cls = 0; cls < 4; ++cls) {
    int ex = C.ext[cls][0], ey = C.ext[cls][1];
    for (int k = 0; k < 8; ++k)
      for (int j = 0; j < ey; ++j)
        for (int i = 0; i < ex; ++i) {
          const size_t o = ((size_t)k * ey + j) * ex + i;
          re[cls][o] = S3.c[cls].at(C, k, i, j).re;
          im[cls][o] = S3.c[cls].at(C, k, i, j).im;
        }
  }
  // limiter activity (the derivative is that of the branch taken)
  long long act = 0;
  for (int k = 0; k < ST_NSTATS; ++k)
    if (k != ST_NEWTON_MAXIT && k != ST_SENSOR_LT099 && k != ST_CFL_VIOLATIONS) act += loc[k];
  return (int)act;
}
#endif

#ifdef AF_ORACLE_COMPLEX
// One forward-Euler stage out = a Un + b FE(Us, dt) of complex states
// (complex-step differentiation), with the limiter coefficients frozen at
// *frz (NULL: formed from the complex state, branches by real part).
int or_stage_cs(const or_params *p, int nx, int ny, const double *const *un_re, const double *const *un_im,
                const double *const *us_re, const double *const *us_im, double dt, double a, double b,
                double *const *out_re, double *const *out_im, const or_coeffs *frz) {
  Ctx C;
  make_ctx(p, nx, ny, C);
  C.frz = frz;
  State Sn, Ss, So;
  Sn.init(C);
  Ss.init(C);
  for (int cls = 0; cls < 4; ++cls) {
    int ex = C.ext[cls][0], ey = C.ext[cls][1];
    for (int k = 0; k < 8; ++k)
      for (int j = 0; j < ey; ++j)
        for (int i = 0; i < ex; ++i) {
          const size_t o = ((size_t)k * ey + j) * ex + i;
          Sn.c[cls].at(C, k, i, j) = Cx(un_re[cls][o], un_im[cls][o]);
          Ss.c[cls].at(C, k, i, j) = Cx(us_re[cls][o], us_im[cls][o]);
        }
  }
  long long loc[ST_NSTATS] = {0};
  stage(C, Sn, Ss, real(dt), real(a), real(b), So, loc);
  for (int cls = 0; cls < 4; ++cls) {
    int ex = C.ext[cls][0], ey = C.ext[cls][1];
    for (int k = 0; k < 8; ++k)
      for (int j = 0; j < ey; ++j)
        for (int i = 0; i < ex; ++i) {
          const size_t o = ((size_t)k * ey + j) * ex + i;
          out_re[cls][o] = So.c[cls].at(C, k, i, j).re;
          out_im[cls][o] = So.c[cls].at(C, k, i, j).im;
        }
  }
  return 0;
}
#endif

// Operation counts per phase since the last reset (counting build only).
// out[NPHASE][NKIND]: add(+sub), mul, div, sqrt, exp, min/max/|.|, comparisons.
int or_counts(long long *out, int reset) {
#ifdef AF_ORACLE_COUNT
  for (int p = 0; p < NPHASE; ++p)
    for (int k = 0; k < NKIND; ++k) out[p * NKIND + k] = g_cnt[p][k];
  if (reset) std::memset(g_cnt, 0, sizeof(g_cnt));
  return 1;
#else
  (void)out; (void)reset;
  return 0;
#endif
}

int or_nphase(void) { return NPHASE; }
int or_nstats(void) { return ST_NSTATS; }

}  // extern "C"
