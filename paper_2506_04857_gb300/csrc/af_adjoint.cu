// af_adjoint.cu -- transpose of the linearised semi-discrete operator L(U)
// (Sec. 2.1-2.3): out = (dL/dU)^T v, in gather form (every output element is
// written by exactly one thread, no atomics, deterministic).
//
// L is the high-order AF right-hand side: LLF flux-vector splitting on the
// point values (alpha = the largest spectral radius on the 5-point line,
// differentiated through the point that attains it), central divergence and
// Powell source for the points, Simpson fluxes and the 3x3 Powell source for
// the cell averages, and the bi-parabola cell-centre values.  On smooth data
// with the shock sensor off (kappa = 0) and every positivity limiter inactive,
// a limited forward-Euler stage is exactly U + dt L(U), so its transpose is
// v + dt (dL/dU)^T v.
//
// Three kernels, after the forward point-data pass at the linearisation state;
// each runs one grid slice (blockIdx.z) per DoF class, so that every thread
// does the work of one DoF with compile-time class and direction:
//   A1 (per output): line coefficients alpha, d(out)/d(alpha) and the argmax,
//      divergence and its cotangent of each point output; for each cell the
//      weighted node divergences and their cotangents.
//   A2 (per DoF): gathers, over every output whose stencil contains the DoF,
//      the cotangents of the DoF's fluxes F1, F2, spectral radii, Psi and B,
//      then applies the transposed pointwise Jacobians.  Cell centres too.
//   A3 (per DoF): distributes the cell-centre cotangents to the DoFs of the
//      bi-parabola, [36 Ubar - 4 (faces) - (corners)] / 16, and applies the
//      Runge-Kutta combination of the reverse sweep (AfAdjEpi).
//
// A 5-point FVS line of an output with index s holds points with indices
// s-1, s, s+1 along its direction (after the periodic wrap or the outflow
// mirror), so a DoF is gathered from the outputs at offsets -1, 0, +1.
//
// Frozen branch (limiter coefficients recorded by a forward stage, co != NULL):
// with theta^s, theta_ij, the face theta (Sec. 3.2, 3.4) and the scaling-limiter
// theta*, theta** (Sec. 3.3, Remark 3.2) held at their recorded values, a
// limited forward-Euler stage is FE(U) = U + dt L_w(U) with
//   cell averages: the face flux w_f F^ + (1 - w_f) F^LLF, w_f = theta_f theta^s_f,
//                  the source w_c S + (1 - w_c) S^LLF, w_c = theta_ij theta^s_ij;
//   point values:  m o L_pt(U) + (1 - m) o L^LLF_pt(U), m = (theta* theta**, theta**, ...);
//   cell centres:  m_c o U_c + (1 - m_c) o Ubar (Remark 3.2 toward the average).
// The kernels above then run on the weighted cotangents (A0 scales the point
// rows by m; A1, A2 weight the cell rows by w_f, w_c; A3 applies m_c), and AL
// adds the transposes of the first-order LLF terms (eq. 2d_llf_flux, S^LLF and
// the three point LLF schemes of Sec. 3.3), with alpha^LLF differentiated along
// the branch its maxima take.
#include "../../include/af.h"
#include "af_internal.h"
#include "af_math.cuh"
#include "af_device.cuh"

using namespace afm;

namespace {

// A1 slots (per index point)
enum {
  A_CX_AL = 0, A_CX_GA, A_CX_AM, A_CY_AL, A_CY_GA, A_CY_AM, A_C_DB, A_C_DBB,   // corner
  A_X_AL, A_X_GA, A_X_AM, A_X_DB, A_X_DBB,                                    // x-face
  A_Y_AL, A_Y_GA, A_Y_AM, A_Y_DB, A_Y_DBB,                                    // y-face
  A_WD = 18,      // 9: W_lm div_lm of the cell
  A_DIVB = 27,    // 9: cotangent of div_lm
  A_N = 36
};
enum { CX = 1, CY = 2, CC = 3, CZ = 4 };   // point classes (x-face, y-face, corner, cell centre)

struct PI {
  int c, i, j;
};
__device__ __forceinline__ bool same(const PI &a, const PI &b) { return a.c == b.c && a.i == b.i && a.j == b.j; }

__constant__ double kCoefF[5] = {1.0, -4.0, 0.0, 4.0, -1.0};   // (F0 - F4) + 4 (F3 - F1)
__constant__ double kCoefU[5] = {1.0, -4.0, 6.0, -4.0, 1.0};   // (U0 + U4) - 4 (U1 + U3) + 6 U2
// coefficient of the node value at position l (0,1,2) in the derivative at node lp
__constant__ double kD1[3][3] = {{-3.0, 4.0, -1.0}, {-1.0, 0.0, 1.0}, {1.0, -4.0, 3.0}};

struct Vec4 {
  const double *p[4];
};
struct OVec4 {
  double *p[4];
};

__device__ __forceinline__ bool valid_point(const AfGrid &g, const PI &q) {
  if (q.c == CZ) return q.i >= 0 && q.i < g.nx && q.j >= 0 && q.j < g.ny;
  return q.i >= 0 && q.i < g.ex[q.c] && q.j >= 0 && q.j < g.ey[q.c];
}

// value of component k of point q's state (cell centres from the centre array)
__device__ __forceinline__ double uval(const AfDev &d, const AfGrid &g, const PI &q, int k) {
  if (q.c == CZ) return __ldg(d.uc + (size_t)k * g.nxa * g.nya + (size_t)q.j * g.nxa + q.i);
  return __ldg(d.us[q.c] + (size_t)k * g.ex[q.c] * g.ey[q.c] + (size_t)q.j * g.ex[q.c] + q.i);
}
__device__ __forceinline__ double pval(const AfDev &d, const AfGrid &g, const PI &q, int slot) {
  return __ldg(d.pd[q.c] + (size_t)slot * g.nxa * g.nya + (size_t)q.j * g.nxa + q.i);
}
__device__ __forceinline__ double vval(const Vec4 &v, const AfGrid &g, int c, int i, int j, int k) {
  return __ldg(v.p[c] + (size_t)k * g.ex[c] * g.ey[c] + (size_t)j * g.ex[c] + i);
}
__device__ __forceinline__ double aval(const double *a, const AfGrid &g, int i, int j, int slot) {
  return __ldg(a + (size_t)slot * g.nxa * g.nya + (size_t)j * g.nxa + i);
}

// The 5-point FVS line of point output (cls, i, j) in direction dir, exactly
// as the forward point-update kernel builds it.
__device__ __forceinline__ void fvs_line(const AfGrid &g, int cls, int dir, int i, int j, PI *P) {
  const int im = mface(i - 1, g.nx, g.bc), ip = mface(i + 1, g.nx, g.bc);
  const int jm = mface(j - 1, g.ny, g.bc), jp = mface(j + 1, g.ny, g.bc);
  const int ci0 = mcell(i - 1, g.nx, g.bc), ci1 = mcell(i, g.nx, g.bc);
  const int cj0 = mcell(j - 1, g.ny, g.bc), cj1 = mcell(j, g.ny, g.bc);
  if (cls == CC && dir == 0) {
    P[0] = {CC, im, j}; P[1] = {CY, ci0, j}; P[2] = {CC, i, j}; P[3] = {CY, ci1, j}; P[4] = {CC, ip, j};
  } else if (cls == CC) {
    P[0] = {CC, i, jm}; P[1] = {CX, i, cj0}; P[2] = {CC, i, j}; P[3] = {CX, i, cj1}; P[4] = {CC, i, jp};
  } else if (cls == CX) {
    P[0] = {CX, im, j}; P[1] = {CZ, ci0, j}; P[2] = {CX, i, j}; P[3] = {CZ, ci1, j}; P[4] = {CX, ip, j};
  } else {
    P[0] = {CY, i, jm}; P[1] = {CZ, i, cj0}; P[2] = {CY, i, j}; P[3] = {CZ, i, cj1}; P[4] = {CY, i, jp};
  }
}

// the 3x3 Simpson nodes of cell (i, j): N[l + 3 m]
__device__ __forceinline__ void cell_nodes(const AfGrid &g, int i, int j, PI *N) {
  const int ip = mface(i + 1, g.nx, g.bc), jp = mface(j + 1, g.ny, g.bc);
  N[0] = {CC, i, j};  N[1] = {CY, i, j};  N[2] = {CC, ip, j};
  N[3] = {CX, i, j};  N[4] = {CZ, i, j};  N[5] = {CX, ip, j};
  N[6] = {CC, i, jp}; N[7] = {CY, i, jp}; N[8] = {CC, ip, jp};
}

// Psi = (0, B, v, v.B) of point q, component k >= 1
__device__ __forceinline__ double psi(const AfDev &d, const AfGrid &g, const PI &q, int k) {
  if (k <= 3) return uval(d, g, q, 3 + k);
  return pval(d, g, q, QP_V1 + (k - 4));
}

// ---- frozen limiter coefficients (co: one stage's AF_NCOEF arrays, or NULL) ----
__device__ __forceinline__ double cof(const double *co, const AfGrid &g, int slot, int i, int j) {
  return __ldg(co + (size_t)slot * g.nxa * g.nya + (size_t)j * g.nxa + i);
}
// weight of the high-order flux at x-face (fi, fj) (dir 0) or y-face (dir 1), stored indices
__device__ __forceinline__ double wface(const double *co, const AfGrid &g, int dir, int fi, int fj) {
  if (!co) return 1.0;
  return cof(co, g, dir ? AFC_THY : AFC_THX, fi, fj) * cof(co, g, dir ? AFC_TSY : AFC_TSX, fi, fj);
}
// weight of the high-order source of cell (i, j): theta_ij times the least theta^s of its faces
__device__ __forceinline__ double wcell(const double *co, const AfGrid &g, int i, int j) {
  if (!co) return 1.0;
  const int ip = mface(i + 1, g.nx, g.bc), jp = mface(j + 1, g.ny, g.bc);
  const double ts = fmin(fmin(cof(co, g, AFC_TSX, i, j), cof(co, g, AFC_TSX, ip, j)),
                         fmin(cof(co, g, AFC_TSY, i, j), cof(co, g, AFC_TSY, i, jp)));
  return cof(co, g, AFC_TSRC, i, j) * ts;
}
// scaling-limiter weight of component k: theta* theta** for the density, theta** otherwise
// (slot s1: theta* of the class or of the cell centre)
__device__ __forceinline__ double mweight(const double *co, const AfGrid &g, int s1, int i, int j, int k) {
  const double t2 = cof(co, g, s1 + 1, i, j);
  return k == 0 ? cof(co, g, s1, i, j) * t2 : t2;
}

// ---------------------------------------------------------------------------
// A1
// ---------------------------------------------------------------------------
template <int CLS, int DIR>
__device__ __forceinline__ void line_coefs(const AfDev &d, const AfGrid &g, const Vec4 &v, int i, int j, double rh,
                                           double *a, int sal, int sga, int sam) {
  PI P[5];
  fvs_line(g, CLS, DIR, i, j, P);
  constexpr int qsr = DIR == 0 ? QP_SR1 : QP_SR2;
  double al = pval(d, g, P[0], qsr);
  int am = 0;
#pragma unroll
  for (int p = 1; p < 5; ++p) {
    const double s = pval(d, g, P[p], qsr);
    if (s > al) { al = s; am = p; }
  }
  double ga = 0.0;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const double up = fma(6.0, uval(d, g, P[2], k),
                          fma(-4.0, uval(d, g, P[1], k) + uval(d, g, P[3], k), uval(d, g, P[0], k) + uval(d, g, P[4], k)));
    ga = fma(vval(v, g, CLS, i, j, k), up, ga);
  }
  const size_t PS = (size_t)g.nxa * g.nya, o = (size_t)j * g.nxa + i;
  a[sal * PS + o] = al;
  a[sga * PS + o] = -0.5 * rh * ga;
  a[sam * PS + o] = (double)am;
}

// (B_l(P0) - B_l(P4)) + 4 (B_l(P3) - B_l(P1)) along the FVS line
template <int CLS, int DIR>
__device__ __forceinline__ double line_db(const AfDev &d, const AfGrid &g, int i, int j) {
  PI P[5];
  fvs_line(g, CLS, DIR, i, j, P);
  constexpr int k = 4 + DIR;
  return fma(4.0, uval(d, g, P[3], k) - uval(d, g, P[1], k), uval(d, g, P[0], k) - uval(d, g, P[4], k));
}

template <int CLS>
__device__ __forceinline__ void point_div(const AfDev &d, const AfGrid &g, const Vec4 &v, int i, int j, double rdx,
                                          double rdy, double *a, int sdb, int sdbb) {
  double divB;
  if (CLS == CC) {
    divB = fma(line_db<CC, 0>(d, g, i, j), 0.5 * rdx, line_db<CC, 1>(d, g, i, j) * (0.5 * rdy));
  } else if (CLS == CX) {
    const int jp = mface(j + 1, g.ny, g.bc);
    const PI lo = {CC, i, j}, hi = {CC, i, jp};
    divB = fma(line_db<CX, 0>(d, g, i, j), 0.5 * rdx, (uval(d, g, hi, 5) - uval(d, g, lo, 5)) * rdy);
  } else {
    const int ip = mface(i + 1, g.nx, g.bc);
    const PI lo = {CC, i, j}, hi = {CC, ip, j};
    divB = fma(uval(d, g, hi, 4) - uval(d, g, lo, 4), rdx, line_db<CY, 1>(d, g, i, j) * (0.5 * rdy));
  }
  const PI q = {CLS, i, j};
  double dbb = 0.0;
  if (g.src_point_on)
#pragma unroll
    for (int k = 1; k < 8; ++k) dbb = fma(-vval(v, g, CLS, i, j, k), psi(d, g, q, k), dbb);
  const size_t PS = (size_t)g.nxa * g.nya, o = (size_t)j * g.nxa + i;
  a[sdb * PS + o] = divB;
  a[sdbb * PS + o] = dbb;
}

__device__ __forceinline__ void cell_terms(const AfDev &d, const AfGrid &g, const Vec4 &v, int i, int j, double rdx,
                                           double rdy, double *a, const double *co) {
  PI N[9];
  cell_nodes(g, i, j, N);
  constexpr double w1[3] = {1.0 / 6.0, 2.0 / 3.0, 1.0 / 6.0};
  const size_t PS = (size_t)g.nxa * g.nya, o = (size_t)j * g.nxa + i;
  const double wc = wcell(co, g, i, j);
  double vc[8];
#pragma unroll
  for (int k = 1; k < 8; ++k) vc[k] = vval(v, g, 0, i, j, k) * wc;
#pragma unroll
  for (int m = 0; m < 3; ++m)
#pragma unroll
    for (int l = 0; l < 3; ++l) {
      double dx1 = 0.0, dy2 = 0.0;
#pragma unroll
      for (int t = 0; t < 3; ++t) {
        dx1 = fma(kD1[l][t], uval(d, g, N[t + 3 * m], 4), dx1);
        dy2 = fma(kD1[m][t], uval(d, g, N[l + 3 * t], 5), dy2);
      }
      const double W = w1[l] * w1[m];
      const double div = fma(dx1, rdx, dy2 * rdy);
      double dd = 0.0;
      if (g.src_cell_on)
#pragma unroll
        for (int k = 1; k < 8; ++k) dd = fma(-vc[k], psi(d, g, N[l + 3 * m], k), dd);
      a[(A_WD + l + 3 * m) * PS + o] = g.src_cell_on ? W * div : 0.0;
      a[(A_DIVB + l + 3 * m) * PS + o] = W * dd;
    }
}

// blockIdx.z: 0 corners, 1 x-faces, 2 y-faces, 3 cells
__global__ void __launch_bounds__(128) k_adj1(const __grid_constant__ AfDev d, const __grid_constant__ AfGrid g,
                                              const __grid_constant__ Vec4 v, double *a, const double *co) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
  const double rdx = 1.0 / g.dx, rdy = 1.0 / g.dy;
  switch (blockIdx.z) {
    case 0:
      if (i < g.ex[CC] && j < g.ey[CC]) {
        line_coefs<CC, 0>(d, g, v, i, j, rdx, a, A_CX_AL, A_CX_GA, A_CX_AM);
        line_coefs<CC, 1>(d, g, v, i, j, rdy, a, A_CY_AL, A_CY_GA, A_CY_AM);
        point_div<CC>(d, g, v, i, j, rdx, rdy, a, A_C_DB, A_C_DBB);
      }
      break;
    case 1:
      if (i < g.ex[CX] && j < g.ey[CX]) {
        line_coefs<CX, 0>(d, g, v, i, j, rdx, a, A_X_AL, A_X_GA, A_X_AM);
        point_div<CX>(d, g, v, i, j, rdx, rdy, a, A_X_DB, A_X_DBB);
      }
      break;
    case 2:
      if (i < g.ex[CY] && j < g.ey[CY]) {
        line_coefs<CY, 1>(d, g, v, i, j, rdy, a, A_Y_AL, A_Y_GA, A_Y_AM);
        point_div<CY>(d, g, v, i, j, rdx, rdy, a, A_Y_DB, A_Y_DBB);
      }
      break;
    default:
      if (i < g.nx && j < g.ny) cell_terms(d, g, v, i, j, rdx, rdy, a, co);
  }
}

// ---------------------------------------------------------------------------
// A2
// ---------------------------------------------------------------------------
struct Acc {
  double F[2][8];   // cotangents of F1, F2
  double sr[2];     // of varrho_1, varrho_2
  double ps[8];     // of Psi
  double B[2];      // of B1, B2 through the divergence stencils
  double U[8];      // direct cotangent of U (the alpha (U0 + U4 - ...) terms)
  double av[2];     // of |v_1|, |v_2| (alpha^LLF)
  double cf[2];     // of c_f1, c_f2 (alpha^LLF)
  double srho;      // of sqrt(rho) (alpha^LLF)
};
__device__ __forceinline__ void acc_zero(Acc &a) {
#pragma unroll
  for (int k = 0; k < 8; ++k) a.F[0][k] = a.F[1][k] = a.ps[k] = a.U[k] = 0.0;
  a.sr[0] = a.sr[1] = a.B[0] = a.B[1] = a.av[0] = a.av[1] = a.cf[0] = a.cf[1] = a.srho = 0.0;
}


// output of class oc at offset o (-1..1) from q along dir, mapped into range;
// false when it does not exist
__device__ __forceinline__ bool candidate(const AfGrid &g, int oc, int dir, const PI &q, int o, PI &s) {
  int i = q.i, j = q.j;
  if (dir == 0) i += o; else j += o;
  if (g.bc == 0) {
    i = wrapi(wrapi(i, g.nx), g.nx);
    j = wrapi(wrapi(j, g.ny), g.ny);
  }
  s = {oc, i, j};
  return s.i >= 0 && s.j >= 0 && s.i < g.ex[oc] && s.j < g.ey[oc];
}

// FVS lines of outputs of class OC in direction DIR that contain q
template <int OC, int DIR>
__device__ __forceinline__ void gather_lines(const AfDev &d, const AfGrid &g, const Vec4 &v, const double *a,
                                             const PI &q, double rh, Acc &acc) {
  constexpr int sal = OC == CC ? (DIR == 0 ? A_CX_AL : A_CY_AL) : (OC == CX ? A_X_AL : A_Y_AL);
  constexpr int sdbb = OC == CC ? A_C_DBB : (OC == CX ? A_X_DBB : A_Y_DBB);
  const double c = 0.5 * rh;
#pragma unroll
  for (int o = -1; o <= 1; ++o) {
    PI s;
    if (!candidate(g, OC, DIR, q, o, s)) continue;
    PI P[5];
    fvs_line(g, OC, DIR, s.i, s.j, P);
    double cf = 0.0, cu = 0.0, csr = 0.0;
    int hits = 0;
    const int am = (int)aval(a, g, s.i, s.j, sal + 2);
#pragma unroll
    for (int p = 0; p < 5; ++p)
      if (same(P[p], q)) {
        cf += kCoefF[p];
        cu += kCoefU[p];
        if (p == am) csr += 1.0;
        ++hits;
      }
    if (!hits) continue;
    const double al = aval(a, g, s.i, s.j, sal);
    if (csr != 0.0) acc.sr[DIR] = fma(csr, aval(a, g, s.i, s.j, sal + 1), acc.sr[DIR]);
    acc.B[DIR] = fma(cf * c, aval(a, g, s.i, s.j, sdbb), acc.B[DIR]);
    const double cual = cu * al;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const double gk = -c * vval(v, g, OC, s.i, s.j, k);
      if (k != 4 + DIR) acc.F[DIR][k] = fma(cf, gk, acc.F[DIR][k]);
      acc.U[k] = fma(cual, gk, acc.U[k]);
    }
  }
}

// central differences: y-face outputs (F1 between corners, along x) and
// x-face outputs (F2 between corners, along y) that use corner q
template <int DIR>
__device__ __forceinline__ void gather_central(const AfGrid &g, const Vec4 &v, const double *a, const PI &q,
                                               double rh, Acc &acc) {
  constexpr int oc = DIR == 0 ? CY : CX;
  constexpr int sdbb = DIR == 0 ? A_Y_DBB : A_X_DBB;
#pragma unroll
  for (int o = -1; o <= 0; ++o) {
    PI s;
    if (!candidate(g, oc, DIR, q, o, s)) continue;
    PI lo = {CC, s.i, s.j}, hi = lo;
    if (DIR == 0) hi.i = mface(s.i + 1, g.nx, g.bc); else hi.j = mface(s.j + 1, g.ny, g.bc);
    const double sgn = (same(hi, q) ? 1.0 : 0.0) - (same(lo, q) ? 1.0 : 0.0);
    if (sgn == 0.0) continue;
    // L -= (F(hi) - F(lo))/h, divB += (B(hi) - B(lo))/h
    acc.B[DIR] = fma(sgn * rh, aval(a, g, s.i, s.j, sdbb), acc.B[DIR]);
#pragma unroll
    for (int k = 0; k < 8; ++k)
      if (k != 4 + DIR) acc.F[DIR][k] = fma(-sgn * rh, vval(v, g, oc, s.i, s.j, k), acc.F[DIR][k]);
  }
}

// cotangent of the Simpson flux of x-face (fi, fj) (DIR 0) or y-face (DIR 1),
// times wgt, added to acc: sum over the cells that use it as their
// left/lower (+) or right/upper (-) face
template <int DIR>
__device__ __forceinline__ void face_cot(const AfGrid &g, const Vec4 &v, int fi, int fj, double wgt, double rh,
                                         Acc &acc, const double *co) {
  wgt *= wface(co, g, DIR, fi, fj);
#pragma unroll
  for (int o = -1; o <= 0; ++o) {
    int ci = fi, cj = fj;
    if (DIR == 0) ci += o; else cj += o;
    if (g.bc == 0) { ci = wrapi(ci, g.nx); cj = wrapi(cj, g.ny); }
    if (ci < 0 || cj < 0 || ci >= g.nx || cj >= g.ny) continue;
    double sgn = 0.0;
    if (DIR == 0) {
      if (ci == fi && cj == fj) sgn += 1.0;                                   // left face of the cell
      if (mface(ci + 1, g.nx, g.bc) == fi && cj == fj) sgn -= 1.0;            // right face
    } else {
      if (ci == fi && cj == fj) sgn += 1.0;
      if (mface(cj + 1, g.ny, g.bc) == fj && ci == fi) sgn -= 1.0;
    }
    if (sgn == 0.0) continue;
    const double w = sgn * wgt * rh;
#pragma unroll
    for (int k = 0; k < 8; ++k)
      if (k != 4 + DIR) acc.F[DIR][k] = fma(w, vval(v, g, 0, ci, cj, k), acc.F[DIR][k]);
  }
}

template <int C>
__device__ __forceinline__ void gather_simpson(const AfGrid &g, const Vec4 &v, const PI &q, double rdx, double rdy,
                                               Acc &acc, const double *co) {
  if constexpr (C == CX) face_cot<0>(g, v, q.i, q.j, 4.0 / 6.0, rdx, acc, co);   // middle node of its own face
  if constexpr (C == CY) face_cot<1>(g, v, q.i, q.j, 4.0 / 6.0, rdy, acc, co);
  if constexpr (C == CC) {
    // corner: end node (weight 1/6) of the x-faces below/above and the y-faces left/right
#pragma unroll
    for (int o = -1; o <= 0; ++o) {
      PI s;
      if (candidate(g, CX, 1, q, o, s)) {
        const int hj = mface(s.j + 1, g.ny, g.bc);
        const double wgt = (s.j == q.j ? 1.0 : 0.0) + (hj == q.j ? 1.0 : 0.0);
        if (wgt != 0.0) face_cot<0>(g, v, s.i, s.j, wgt / 6.0, rdx, acc, co);
      }
      if (candidate(g, CY, 0, q, o, s)) {
        const int hi = mface(s.i + 1, g.nx, g.bc);
        const double wgt = (s.i == q.i ? 1.0 : 0.0) + (hi == q.i ? 1.0 : 0.0);
        if (wgt != 0.0) face_cot<1>(g, v, s.i, s.j, wgt / 6.0, rdy, acc, co);
      }
    }
  }
}

// the 3x3 source nodes of the cells that have q as a node (node n = l + 3 m)
template <int C>
__device__ __forceinline__ void gather_source(const AfGrid &g, const Vec4 &v, const double *a, const PI &q, double rdx,
                                              double rdy, Acc &acc, const double *co) {
  constexpr int na = C == CC ? 4 : (C == CZ ? 1 : 2);
  constexpr int nodes[4] = {C == CC ? 0 : (C == CX ? 3 : (C == CY ? 1 : 4)), C == CC ? 2 : (C == CX ? 5 : 7),
                            6, 8};
#pragma unroll
  for (int b = 0; b <= 1; ++b)
#pragma unroll
    for (int aa = 0; aa <= 1; ++aa) {
      if (C == CZ && (aa || b)) continue;
      if (C == CX && b) continue;    // x-face (i, j) is a node of cells (i-1, j) and (i, j) only
      if (C == CY && aa) continue;
      int ci = q.i - aa, cj = q.j - b;
      if (g.bc == 0) { ci = wrapi(ci, g.nx); cj = wrapi(cj, g.ny); }
      if (ci < 0 || cj < 0 || ci >= g.nx || cj >= g.ny) continue;
      PI N[9];
      cell_nodes(g, ci, cj, N);
#pragma unroll
      for (int t = 0; t < na; ++t) {
        const int n = nodes[t];
        if (!same(N[n], q)) continue;
        const int l = n % 3, m = n / 3;
        const double wd = aval(a, g, ci, cj, A_WD + n) * wcell(co, g, ci, cj);
#pragma unroll
        for (int k = 1; k < 8; ++k) acc.ps[k] = fma(-wd, vval(v, g, 0, ci, cj, k), acc.ps[k]);
        double s1 = 0.0, s2 = 0.0;
#pragma unroll
        for (int r = 0; r < 3; ++r) {
          s1 = fma(aval(a, g, ci, cj, A_DIVB + r + 3 * m), kD1[r][l], s1);   // d/dx at node (r, m) uses node (l, m)
          s2 = fma(aval(a, g, ci, cj, A_DIVB + l + 3 * r), kD1[r][m], s2);   // d/dy at node (l, r) uses node (l, m)
        }
        acc.B[0] = fma(s1, rdx, acc.B[0]);
        acc.B[1] = fma(s2, rdy, acc.B[1]);
      }
    }
}

// Transpose of the point data of one state: F1, F2, varrho_1, varrho_2 and
// Psi = (0, B, v, v.B) as computed by the forward point-data pass.
__device__ __forceinline__ void pointwise_transpose(const double *U, const AfGrid &g, const Acc &acc, double *out) {
  const double rho = U[0], r = rcp(rho);
  const double m1 = U[1], m2 = U[2], m3 = U[3];
  const double v1 = mul_i(m1, r), v2 = mul_i(m2, r), v3 = mul_i(m3, r);
  const double B1 = U[4], B2 = U[5], B3 = U[6], E = U[7];
  const double BB = fma(B3, B3, fma(B2, B2, mul_i(B1, B1)));
  const double mv = fma(m3, v3, fma(m2, v2, mul_i(m1, v1)));
  const double p = mul_i(g.gm1, fma(-0.5, mv + BB, E));
  const double pt = fma(0.5, BB, p);
  const double vB = fma(v3, B3, fma(v2, B2, mul_i(v1, B1)));
  const double Ept = E + pt;
  double mb1 = 0, mb2 = 0, mb3 = 0, Bb1 = acc.B[0], Bb2 = acc.B[1], Bb3 = 0, Eb = 0;
  double vb1 = 0, vb2 = 0, vb3 = 0, ptb = 0, vBb = 0, Eptb = 0, pb = 0;
  const double *F1 = acc.F[0], *F2 = acc.F[1];
  // F1
  mb1 += F1[0];
  mb1 += F1[1] * v1; vb1 += F1[1] * m1; ptb += F1[1]; Bb1 -= 2.0 * B1 * F1[1];
  mb1 += F1[2] * v2; vb2 += F1[2] * m1; Bb1 -= F1[2] * B2; Bb2 -= F1[2] * B1;
  mb1 += F1[3] * v3; vb3 += F1[3] * m1; Bb1 -= F1[3] * B3; Bb3 -= F1[3] * B1;
  vb1 += F1[5] * B2; Bb2 += F1[5] * v1; Bb1 -= F1[5] * v2; vb2 -= F1[5] * B1;
  vb1 += F1[6] * B3; Bb3 += F1[6] * v1; Bb1 -= F1[6] * v3; vb3 -= F1[6] * B1;
  Eptb += F1[7] * v1; vb1 += F1[7] * Ept; Bb1 -= F1[7] * vB; vBb -= F1[7] * B1;
  // F2
  mb2 += F2[0];
  mb1 += F2[1] * v2; vb2 += F2[1] * m1; Bb1 -= F2[1] * B2; Bb2 -= F2[1] * B1;
  mb2 += F2[2] * v2; vb2 += F2[2] * m2; ptb += F2[2]; Bb2 -= 2.0 * B2 * F2[2];
  mb2 += F2[3] * v3; vb3 += F2[3] * m2; Bb2 -= F2[3] * B3; Bb3 -= F2[3] * B2;
  Bb1 += F2[4] * v2; vb2 += F2[4] * B1; vb1 -= F2[4] * B2; Bb2 -= F2[4] * v1;
  vb2 += F2[6] * B3; Bb3 += F2[6] * v2; Bb2 -= F2[6] * v3; vb3 -= F2[6] * B2;
  Eptb += F2[7] * v2; vb2 += F2[7] * Ept; Bb2 -= F2[7] * vB; vBb -= F2[7] * B2;
  // Psi
  Bb1 += acc.ps[1]; Bb2 += acc.ps[2]; Bb3 += acc.ps[3];
  vb1 += acc.ps[4]; vb2 += acc.ps[5]; vb3 += acc.ps[6]; vBb += acc.ps[7];
  // spectral radii varrho_l = |v_l| + c_{f,l}
  const double c2 = mul_i(mul_i(g.gamma, p), r);
  const double a = fma(BB, r, c2);
  const double k4 = ldexp_i<2>(mul_i(c2, r));
  double ab = 0, c2b = 0, k4b = 0;
#pragma unroll
  for (int l = 0; l < 2; ++l) {
    const double avb = acc.sr[l] + acc.av[l], srb = acc.sr[l] + acc.cf[l];   // of |v_l| and of c_f,l
    const double vl = l == 0 ? v1 : v2, Bl = l == 0 ? B1 : B2;
    if (l == 0) vb1 += vl >= 0.0 ? avb : -avb; else vb2 += vl >= 0.0 ? avb : -avb;
    if (srb == 0.0) continue;
    const double k4B = mul_i(k4, Bl);
    double dd = fma(-k4B, Bl, mul_i(a, a));
    if (!gt_zero(dd)) dd = 0.0;
    const double sd = dsqrt(dd);
    const double s = fma(0.5, sd, ldexp_i<-1>(a));
    const double cf = dsqrt(s);
    const double sb = gt_zero(cf) ? mul_i(ldexp_i<-1>(srb), rcp(cf)) : 0.0;
    ab = fma(0.5, sb, ab);
    const double ddb = gt_zero(sd) ? mul_i(ldexp_i<-2>(sb), rcp(sd)) : 0.0;
    ab = fma(ldexp_i<1>(a), ddb, ab);
    k4b = fma(-mul_i(Bl, Bl), ddb, k4b);
    if (l == 0) Bb1 = fma(-ldexp_i<1>(k4B), ddb, Bb1); else Bb2 = fma(-ldexp_i<1>(k4B), ddb, Bb2);
  }
  double rbar = 0.0;
  c2b = fma(ldexp_i<2>(r), k4b, c2b);
  rbar = fma(ldexp_i<2>(c2), k4b, rbar);
  const double rab2 = ldexp_i<1>(mul_i(r, ab));
  Bb1 = fma(B1, rab2, Bb1); Bb2 = fma(B2, rab2, Bb2); Bb3 = fma(B3, rab2, Bb3);
  rbar = fma(BB, ab, rbar);
  c2b += ab;
  pb = fma(mul_i(g.gamma, r), c2b, pb);
  rbar = fma(mul_i(g.gamma, p), c2b, rbar);
  // Ept = E + pt; vB = v.B; pt = p + BB/2; p = (gamma-1)(E - (mv + BB)/2)
  Eb += Eptb; ptb += Eptb;
  vb1 += vBb * B1; vb2 += vBb * B2; vb3 += vBb * B3;
  Bb1 += vBb * v1; Bb2 += vBb * v2; Bb3 += vBb * v3;
  pb += ptb;
  Bb1 += ptb * B1; Bb2 += ptb * B2; Bb3 += ptb * B3;
  const double gpb = mul_i(g.gm1, pb);
  Eb += gpb;
  const double mvb = ldexp_i<-1>(neg_i(gpb));
  Bb1 = fma(-gpb, B1, Bb1); Bb2 = fma(-gpb, B2, Bb2); Bb3 = fma(-gpb, B3, Bb3);
  mb1 += mvb * v1; mb2 += mvb * v2; mb3 += mvb * v3;
  vb1 += mvb * m1; vb2 += mvb * m2; vb3 += mvb * m3;
  // v_k = m_k r, r = 1/rho
  mb1 += vb1 * r; mb2 += vb2 * r; mb3 += vb3 * r;
  rbar += vb1 * m1 + vb2 * m2 + vb3 * m3;
  out[0] = fma(-mul_i(r, r), rbar, acc.U[0]);
  if (!is_zero(acc.srho)) out[0] = fma(ldexp_i<-1>(acc.srho), rcp(dsqrt(rho)), out[0]);   // d sqrt(rho) / d rho
  out[1] = mb1 + acc.U[1];
  out[2] = mb2 + acc.U[2];
  out[3] = mb3 + acc.U[3];
  out[4] = Bb1 + acc.U[4];
  out[5] = Bb2 + acc.U[5];
  out[6] = Bb3 + acc.U[6];
  out[7] = Eb + acc.U[7];
}

template <int C>
__device__ __forceinline__ void adj_point(const AfDev &d, const AfGrid &g, const Vec4 &v, const double *a, int i,
                                          int j, double rdx, double rdy, double *const *tp, double *zc,
                                          const double *co) {
  const PI q = {C, i, j};
  if (!valid_point(g, q)) return;
  Acc acc;
  acc_zero(acc);
  if (C == CC || C == CY) gather_lines<CC, 0>(d, g, v, a, q, rdx, acc);
  if (C == CC || C == CX) gather_lines<CC, 1>(d, g, v, a, q, rdy, acc);
  if (C == CX || C == CZ) gather_lines<CX, 0>(d, g, v, a, q, rdx, acc);
  if (C == CY || C == CZ) gather_lines<CY, 1>(d, g, v, a, q, rdy, acc);
  if (C == CC) {
    gather_central<0>(g, v, a, q, rdx, acc);
    gather_central<1>(g, v, a, q, rdy, acc);
  }
  gather_simpson<C>(g, v, q, rdx, rdy, acc, co);
  gather_source<C>(g, v, a, q, rdx, rdy, acc, co);
  if (C != CZ && g.src_point_on) {   // own Powell term -(div B) Psi
    constexpr int sdb = C == CC ? A_C_DB : (C == CX ? A_X_DB : A_Y_DB);
    const double divB = aval(a, g, i, j, sdb);
#pragma unroll
    for (int k = 1; k < 8; ++k) acc.ps[k] = fma(-divB, vval(v, g, C, i, j, k), acc.ps[k]);
  }
  double U[8], o[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) U[k] = uval(d, g, q, k);
  pointwise_transpose(U, g, acc, o);
  if (C == CZ) {
    const size_t PS = (size_t)g.nxa * g.nya, oo = (size_t)j * g.nxa + i;
#pragma unroll
    for (int k = 0; k < 8; ++k) zc[k * PS + oo] = o[k];
  } else {
    const size_t cs = (size_t)g.ex[C] * g.ey[C], oo = (size_t)j * g.ex[C] + i;
#pragma unroll
    for (int k = 0; k < 8; ++k) tp[C][k * cs + oo] = o[k];
  }
}

// blockIdx.z: 0 x-faces, 1 y-faces, 2 corners, 3 cell centres
// A2 compiled for 4 resident blocks of 128 threads (128 registers): 3 % faster than
// the compiler's 166 registers on the 256x256 adjoint workload
#ifndef AF_MINB_ADJ2
#define AF_MINB_ADJ2 4
#endif
#define AF_LB_ADJ2 __launch_bounds__(128, AF_MINB_ADJ2)
__global__ void AF_LB_ADJ2 k_adj2(const __grid_constant__ AfDev d, const __grid_constant__ AfGrid g,
                                              const __grid_constant__ Vec4 v, const double *a,
                                              const __grid_constant__ OVec4 tp, double *zc, const double *co) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
  const double rdx = 1.0 / g.dx, rdy = 1.0 / g.dy;
  switch (blockIdx.z) {
    case 0: adj_point<CX>(d, g, v, a, i, j, rdx, rdy, tp.p, zc, co); break;
    case 1: adj_point<CY>(d, g, v, a, i, j, rdx, rdy, tp.p, zc, co); break;
    case 2: adj_point<CC>(d, g, v, a, i, j, rdx, rdy, tp.p, zc, co); break;
    default: adj_point<CZ>(d, g, v, a, i, j, rdx, rdy, tp.p, zc, co);
  }
}

// ---------------------------------------------------------------------------
// A3: U_c = 2.25 Ubar - 0.25 (faces) - 0.0625 (corners), then the epilogue
// ---------------------------------------------------------------------------
template <int C>
__device__ __forceinline__ void adj_final(const AfGrid &g, const double *zc, const double *const *tp,
                                          const AfAdjEpi &e, int i, int j, const double *co) {
  if (i >= g.ex[C] || j >= g.ey[C]) return;
  const size_t PS = (size_t)g.nxa * g.nya;
  const size_t cs = (size_t)g.ex[C] * g.ey[C], oo = (size_t)j * g.ex[C] + i;
  double T[8];
  if (C == 0) {
    if (co) {   // frozen branch: Remark 3.2 blend m_c o U_c + (1 - m_c) o Ubar, plus the LLF part (AL)
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const double z = __ldg(zc + k * PS + (size_t)j * g.nxa + i), m = mweight(co, g, AFC_C1, i, j, k);
        T[k] = fma(2.25 * m, z, fma(1.0 - m, z, __ldg(tp[0] + k * cs + oo)));
      }
    } else {
#pragma unroll
      for (int k = 0; k < 8; ++k) T[k] = 2.25 * __ldg(zc + k * PS + (size_t)j * g.nxa + i);
    }
  } else {
#pragma unroll
    for (int k = 0; k < 8; ++k) T[k] = __ldg(tp[C] + k * cs + oo);
    const PI q = {C, i, j};
#pragma unroll
    for (int b = 0; b <= 1; ++b)
#pragma unroll
      for (int aa = 0; aa <= 1; ++aa) {
        if (C == 1 && b) continue;
        if (C == 2 && aa) continue;
        int ci = i - aa, cj = j - b;
        if (g.bc == 0) { ci = wrapi(ci, g.nx); cj = wrapi(cj, g.ny); }
        if (ci < 0 || cj < 0 || ci >= g.nx || cj >= g.ny) continue;
        PI N[9];
        cell_nodes(g, ci, cj, N);
        double wgt = 0.0;
#pragma unroll
        for (int n = 0; n < 9; ++n)
          if (n != 4 && same(N[n], q)) wgt += (n == 1 || n == 3 || n == 5 || n == 7) ? -0.25 : -0.0625;
        if (wgt == 0.0) continue;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const double m = co ? mweight(co, g, AFC_C1, ci, cj, k) : 1.0;
          T[k] = fma(wgt * m, __ldg(zc + k * PS + (size_t)cj * g.nxa + ci), T[k]);
        }
      }
  }
  const double bs = e.dt ? e.b * __ldg(e.dt) : e.b;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const size_t o = k * cs + oo;
    const double vk = e.v[C][o];
    double r = fma(bs, T[k], e.a * vk);
    if (e.z1[0]) r = fma(e.c, e.z1[C][o], r);
    if (e.out2[0]) e.out2[C][o] = fma(e.f, e.z2[C][o], e.e * vk);
    e.out1[C][o] = r;
  }
}

// blockIdx.z: DoF class 0..3
__global__ void __launch_bounds__(128) k_adj3(const __grid_constant__ AfGrid g, const double *zc,
                                              const __grid_constant__ OVec4 tp, const __grid_constant__ AfAdjEpi e,
                                              const double *co) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
  switch (blockIdx.z) {
    case 0: adj_final<0>(g, zc, tp.p, e, i, j, co); break;
    case 1: adj_final<1>(g, zc, tp.p, e, i, j, co); break;
    case 2: adj_final<2>(g, zc, tp.p, e, i, j, co); break;
    default: adj_final<3>(g, zc, tp.p, e, i, j, co);
  }
}

// ---------------------------------------------------------------------------
// Frozen branch: A0 (point rows scaled by the scaling-limiter weights m) and AL
// (transposes of the first-order LLF terms)
// ---------------------------------------------------------------------------
// blockIdx.z: point class 1..3 (z = 0 idle); vp = m o v for that class
__global__ void __launch_bounds__(128) k_adj0(const __grid_constant__ AfGrid g, const __grid_constant__ Vec4 v,
                                              const __grid_constant__ OVec4 vp, const double *co) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y, c = blockIdx.z;
  if (c == 0 || i >= g.ex[c] || j >= g.ey[c]) return;
  const size_t cs = (size_t)g.ex[c] * g.ey[c], oo = (size_t)j * g.ex[c] + i;
  const int s1 = AFC_P1 + 2 * (c - 1);
#pragma unroll
  for (int k = 0; k < 8; ++k) vp.p[c][k * cs + oo] = mweight(co, g, s1, i, j, k) * __ldg(v.p[c] + k * cs + oo);
}

// What alpha^LLF along direction l and Psi need of one state
struct LS {
  double U[8], v[3], B[3], vB, cf, srho;
};
__device__ __forceinline__ void lstate(const AfDev &d, const AfGrid &g, int c, int i, int j, int l, LS &s) {
  const size_t cs = (size_t)g.ex[c] * g.ey[c], oo = (size_t)j * g.ex[c] + i;
#pragma unroll
  for (int k = 0; k < 8; ++k) s.U[k] = __ldg(d.us[c] + k * cs + oo);
  const double rho = s.U[0], r = rcp(rho);
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    s.v[k] = s.U[1 + k] * r;
    s.B[k] = s.U[4 + k];
  }
  s.vB = fma(s.v[0], s.B[0], fma(s.v[1], s.B[1], s.v[2] * s.B[2]));
  const double BB = fma(s.B[0], s.B[0], fma(s.B[1], s.B[1], s.B[2] * s.B[2]));
  const double mv = fma(s.U[1], s.v[0], fma(s.U[2], s.v[1], s.U[3] * s.v[2]));
  const double p = g.gm1 * fma(-0.5, mv + BB, s.U[7]);
  const double c2 = g.gamma * p * r, a = fma(BB, r, c2);
  double dd = fma(-4.0 * (c2 * r), s.B[l] * s.B[l], a * a);
  dd = dd > 0.0 ? dd : 0.0;
  s.cf = dsqrt(fma(0.5, dsqrt(dd), 0.5 * a));
  s.srho = dsqrt(rho);
}

// Cotangent c of F^LLF_l(Ua, Ub) = (F_l(Ua) + F_l(Ub) - alpha (Ub - Ua)) / 2 (eq. 2d_llf_flux)
// taken back to state a (which = 0) or b (which = 1) of that flux.  alpha^LLF =
// max(|v_a|, |v_b|) + max(c_f,a, c_f,b) + |B_a - B_b| / (sqrt(rho_a) + sqrt(rho_b))
// (Lemma 3.1 with equality), differentiated through the terms its maxima take
// (ties: state a).
__device__ __forceinline__ void llf_vjp(int l, int which, const LS &a, const LS &b, const double *c, Acc &acc) {
  const double va = absd(a.v[l]), vb = absd(b.v[l]);
  const double d0 = a.B[0] - b.B[0], d1 = a.B[1] - b.B[1], d2 = a.B[2] - b.B[2];
  const double n = dsqrt(fma(d0, d0, fma(d1, d1, d2 * d2))), den = a.srho + b.srho;
  const double al = fmax(va, vb) + fmax(a.cf, b.cf) + n / den;
  double T = 0.0;
#pragma unroll
  for (int k = 0; k < 8; ++k) T = fma(c[k], b.U[k] - a.U[k], T);
  const double h = -0.5 * T, sal = which == 0 ? 0.5 * al : -0.5 * al;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    acc.F[l][k] = fma(0.5, c[k], acc.F[l][k]);
    acc.U[k] = fma(sal, c[k], acc.U[k]);
  }
  if (which == 0 ? va >= vb : vb > va) acc.av[l] += h;
  if (which == 0 ? a.cf >= b.cf : b.cf > a.cf) acc.cf[l] += h;
  if (n > 0.0) {
    const double sb = (which == 0 ? h : -h) / (n * den);
    acc.U[4] = fma(sb, d0, acc.U[4]);
    acc.U[5] = fma(sb, d1, acc.U[5]);
    acc.U[6] = fma(sb, d2, acc.U[6]);
    acc.srho -= h * n / (den * den);
  }
}

// Psi(U) . w over the components 1..7 (Psi = (0, B, v, v.B))
__device__ __forceinline__ double psi_dot(const LS &s, const double *w) {
  return fma(w[1], s.B[0], fma(w[2], s.B[1], fma(w[3], s.B[2],
             fma(w[4], s.v[0], fma(w[5], s.v[1], fma(w[6], s.v[2], w[7] * s.vB))))));
}

// The four LLF neighbours (left/right along x, low/high along y) of point value
// (c, i, j), mapped as the forward point limiter maps them (Sec. 3.3).
__device__ __forceinline__ void llf_nbrs(const AfGrid &g, int c, int i, int j, PI *nb) {
  if (c == CC) {
    nb[0] = {CC, mface(i - 1, g.nx, g.bc), j}; nb[1] = {CC, mface(i + 1, g.nx, g.bc), j};
    nb[2] = {CC, i, mface(j - 1, g.ny, g.bc)}; nb[3] = {CC, i, mface(j + 1, g.ny, g.bc)};
  } else if (c == CX) {
    nb[0] = {CX, mface(i - 1, g.nx, g.bc), j}; nb[1] = {CX, mface(i + 1, g.nx, g.bc), j};
    nb[2] = {CC, i, j}; nb[3] = {CC, i, mface(j + 1, g.ny, g.bc)};
  } else {
    nb[0] = {CC, i, j}; nb[1] = {CC, mface(i + 1, g.nx, g.bc), j};
    nb[2] = {CY, i, mface(j - 1, g.ny, g.bc)}; nb[3] = {CY, i, mface(j + 1, g.ny, g.bc)};
  }
}

// (1 - m) o v of point p, false when m = 1 (the point limiter took theta* = theta** = 1)
__device__ __forceinline__ bool llf_cot(const AfGrid &g, const Vec4 &v, const double *co, const PI &p, double *gp) {
  const int s1 = AFC_P1 + 2 * (p.c - 1);
  const double t1 = cof(co, g, s1, p.i, p.j), t2 = cof(co, g, s1 + 1, p.i, p.j);
  if (t1 == 1.0 && t2 == 1.0) return false;
#pragma unroll
  for (int k = 0; k < 8; ++k) gp[k] = (1.0 - (k == 0 ? t1 * t2 : t2)) * vval(v, g, p.c, p.i, p.j, k);
  return true;
}

// candidate point values whose LLF stencil may hold point q
__device__ __forceinline__ int llf_candidates(const AfGrid &g, const PI &q, PI *cand) {
  int n = 0;
  auto add = [&](int c, int i, int j) {
    if (g.bc == 0) {
      i = wrapi(i, g.ex[c]);
      j = wrapi(j, g.ey[c]);
    }
    if (i >= 0 && j >= 0 && i < g.ex[c] && j < g.ey[c]) cand[n++] = {c, i, j};
  };
  if (q.c == CC) {
    add(CC, q.i - 1, q.j); add(CC, q.i + 1, q.j); add(CC, q.i, q.j - 1); add(CC, q.i, q.j + 1);
    add(CX, q.i, q.j); add(CX, q.i, q.j - 1); add(CY, q.i, q.j); add(CY, q.i - 1, q.j);
  } else if (q.c == CX) {
    add(CX, q.i - 1, q.j); add(CX, q.i + 1, q.j);
  } else {
    add(CY, q.i, q.j - 1); add(CY, q.i, q.j + 1);
  }
  return n;
}

template <int C>
__device__ __forceinline__ void adj_llf(const AfDev &d, const AfGrid &g, const Vec4 &v, const double *co, int i,
                                        int j, double *const *tp) {
  const double rdx = g.rdx, rdy = g.rdy;
  Acc acc;
  acc_zero(acc);
  bool touched = false;
  LS me, ot;
  if constexpr (C == 0) {
    if (i >= g.nx || j >= g.ny) return;
    // face fluxes F^LLF of the cell's four faces (weight 1 - w_f)
#pragma unroll
    for (int dir = 0; dir < 2; ++dir) {
      const int n = dir ? g.ny : g.nx, io = dir ? j : i;
      const double rh = dir ? rdy : rdx;
      lstate(d, g, 0, i, j, dir, me);
#pragma unroll
      for (int side = 0; side < 2; ++side) {
        const int f = io + side, fs = mface(f, n, g.bc);
        const double w = wface(co, g, dir, dir ? i : fs, dir ? fs : j);
        if (w == 1.0) continue;
        double cv[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) cv[k] = 0.0;
        // the real cells on either side: -F/h for the left/lower one, +F/h for the right/upper one
#pragma unroll
        for (int t = 0; t < 2; ++t) {
          int ci = f - 1 + t;
          if (g.bc == 0) ci = wrapi(ci, n);
          else if (ci < 0 || ci >= n) continue;
          const double sg = (t ? 1.0 : -1.0) * (1.0 - w) * rh;
#pragma unroll
          for (int k = 0; k < 8; ++k) cv[k] = fma(sg, vval(v, g, 0, dir ? i : ci, dir ? ci : j, k), cv[k]);
        }
        const int ma = mcell(f - 1, n, g.bc), mb = mcell(f, n, g.bc);
        if (ma == io) {
          lstate(d, g, 0, dir ? i : mb, dir ? mb : j, dir, ot);
          llf_vjp(dir, 0, me, ot, cv, acc);
        }
        if (mb == io) {
          lstate(d, g, 0, dir ? i : ma, dir ? ma : j, dir, ot);
          llf_vjp(dir, 1, ot, me, cv, acc);
        }
        touched = true;
      }
    }
    // S^LLF = (central div Bbar) Psi(Ubar) of the cell and of its neighbours (weight 1 - w_c)
    if (g.src_cell_on) {
      const int cc[5][2] = {{i, j}, {i - 1, j}, {i + 1, j}, {i, j - 1}, {i, j + 1}};
#pragma unroll
      for (int t = 0; t < 5; ++t) {
        int ci = cc[t][0], cj = cc[t][1];
        if (g.bc == 0) {
          ci = wrapi(ci, g.nx);
          cj = wrapi(cj, g.ny);
        } else if (ci < 0 || cj < 0 || ci >= g.nx || cj >= g.ny) {
          continue;
        }
        const double wc = wcell(co, g, ci, cj);
        if (wc == 1.0) continue;
        const int e = mcell(ci + 1, g.nx, g.bc), wv = mcell(ci - 1, g.nx, g.bc);
        const int nn = mcell(cj + 1, g.ny, g.bc), sv = mcell(cj - 1, g.ny, g.bc);
        double gc[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) gc[k] = -(1.0 - wc) * vval(v, g, 0, ci, cj, k);
        lstate(d, g, 0, ci, cj, 0, ot);
        const double sc = psi_dot(ot, gc);
        const double c1 = ((cj == j && e == i) ? 1.0 : 0.0) - ((cj == j && wv == i) ? 1.0 : 0.0);
        const double c2 = ((ci == i && nn == j) ? 1.0 : 0.0) - ((ci == i && sv == j) ? 1.0 : 0.0);
        acc.U[4] = fma(c1 * 0.5 * rdx, sc, acc.U[4]);
        acc.U[5] = fma(c2 * 0.5 * rdy, sc, acc.U[5]);
        if (t == 0) {   // its own Psi, times its central div Bbar
          const SV A = sview(d.us[0], g, 0);
          const double divB = fma(A(e, cj, 4) - A(wv, cj, 4), 0.5 * rdx, (A(ci, nn, 5) - A(ci, sv, 5)) * (0.5 * rdy));
#pragma unroll
          for (int k = 1; k < 8; ++k) acc.ps[k] = fma(divB, gc[k], acc.ps[k]);
        }
        touched = true;
      }
    }
    const size_t cs = (size_t)g.nx * g.ny, oo = (size_t)j * g.nx + i;
    double o[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    if (touched) {
      lstate(d, g, 0, i, j, 0, me);
      pointwise_transpose(me.U, g, acc, o);
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) tp[0][k * cs + oo] = o[k];
  } else {
    const PI q = {C, i, j};
    if (!valid_point(g, q)) return;
    double gq[8];
    PI nb[4];
    // its own LLF state: -(F1(q, xr) - F1(xl, q))/dx - (F2(q, yr) - F2(yl, q))/dy - div B Psi(q)
    if (llf_cot(g, v, co, q, gq)) {
      llf_nbrs(g, C, i, j, nb);
      double cp[8], cm[8];
#pragma unroll
      for (int l = 0; l < 2; ++l) {
        const double rh = l ? rdy : rdx;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          cp[k] = rh * gq[k];
          cm[k] = -rh * gq[k];
        }
        lstate(d, g, C, i, j, l, me);
        lstate(d, g, nb[2 * l].c, nb[2 * l].i, nb[2 * l].j, l, ot);
        llf_vjp(l, 1, ot, me, cp, acc);
        lstate(d, g, nb[2 * l + 1].c, nb[2 * l + 1].i, nb[2 * l + 1].j, l, ot);
        llf_vjp(l, 0, me, ot, cm, acc);
      }
      if (g.src_point_on) {
        const double divB = fma(uval(d, g, nb[1], 4) - uval(d, g, nb[0], 4), 0.5 * rdx,
                                (uval(d, g, nb[3], 5) - uval(d, g, nb[2], 5)) * (0.5 * rdy));
#pragma unroll
        for (int k = 1; k < 8; ++k) acc.ps[k] = fma(-divB, gq[k], acc.ps[k]);
      }
      touched = true;
    }
    // as a neighbour in the LLF states of other points
    PI cand[8];
    const int nc = llf_candidates(g, q, cand);
    for (int t = 0; t < nc; ++t) {
      const PI p = cand[t];
      double gp[8];
      if (!llf_cot(g, v, co, p, gp)) continue;
      llf_nbrs(g, p.c, p.i, p.j, nb);
      for (int r = 0; r < 4; ++r) {
        if (!same(nb[r], q)) continue;
        const int l = r >> 1;
        const double rh = l ? rdy : rdx;
        double cv[8];
        lstate(d, g, C, i, j, l, me);
        lstate(d, g, p.c, p.i, p.j, l, ot);
        if (r & 1) {   // q is the right/high neighbour: flux F(p, q), cotangent -g_p/h
#pragma unroll
          for (int k = 0; k < 8; ++k) cv[k] = -rh * gp[k];
          llf_vjp(l, 1, ot, me, cv, acc);
        } else {       // left/low neighbour: flux F(q, p), cotangent +g_p/h
#pragma unroll
          for (int k = 0; k < 8; ++k) cv[k] = rh * gp[k];
          llf_vjp(l, 0, me, ot, cv, acc);
        }
        if (g.src_point_on) {   // div B of p: +-B_l(q) / (2 h)
          const double sp = psi_dot(ot, gp) * 0.5 * rh;
          acc.U[4 + l] += (r & 1) ? -sp : sp;
        }
        touched = true;
      }
    }
    if (!touched) return;
    double U[8], o[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) U[k] = uval(d, g, q, k);
    pointwise_transpose(U, g, acc, o);
    const size_t cs = (size_t)g.ex[C] * g.ey[C], oo = (size_t)j * g.ex[C] + i;
#pragma unroll
    for (int k = 0; k < 8; ++k) tp[C][k * cs + oo] += o[k];
  }
}

// blockIdx.z: DoF class 0..3; after A2 (adds into its point outputs, writes tp[0])
__global__ void __launch_bounds__(128) k_adjl(const __grid_constant__ AfDev d, const __grid_constant__ AfGrid g,
                                              const __grid_constant__ Vec4 v, const __grid_constant__ OVec4 tp,
                                              const double *co) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
  switch (blockIdx.z) {
    case 0: adj_llf<0>(d, g, v, co, i, j, tp.p); break;
    case 1: adj_llf<CX>(d, g, v, co, i, j, tp.p); break;
    case 2: adj_llf<CY>(d, g, v, co, i, j, tp.p); break;
    default: adj_llf<CC>(d, g, v, co, i, j, tp.p);
  }
}

inline dim3 grid3(int nx, int ny) { return dim3((nx + 31) / 32, (ny + 3) / 4, 4); }

// ---------------------------------------------------------------------------
// Sensitivity to dt.  dt = cfl / (M1/dx + M2/dy), M_l = max varrho_l over the
// DoFs of U^n, so dJ/dU^n gains mu * d(dt)/dU^n with mu = dJ/d(dt) and
// d(dt)/dU = -(dt^2/cfl) (dM1/dU / dx + dM2/dU / dy), dM_l/dU = d varrho_l / dU
// at the DoF attaining the maximum (a subgradient where it is not unique: the
// first such DoF in class-then-index order).  On the smooth branch FE(U) =
// U + dt L(U), so with the reverse-sweep variables
//   mu dt = 2/3 L3.(FE(U2) - U2) + 1/4 L2.(FE(U1) - U1) + L1.(FE(U0) - U0),
//   FE(U0) = U1,  FE(U1) = 4 U2 - 3 U0,  FE(U2) = (3 U3 - U0)/2.
// ---------------------------------------------------------------------------
struct DtVec {
  const double *L3[4], *L2[4], *L1[4], *U0[4], *U1[4], *U2[4], *U3[4];
  long long len[4];
};

__global__ void __launch_bounds__(256) k_dt_dot(const __grid_constant__ DtVec v, double *partials) {
  double acc = 0.0;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (int c = 0; c < 4; ++c)
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < v.len[c]; t += stride) {
      const double u0 = v.U0[c][t], u1 = v.U1[c][t], u2 = v.U2[c][t], u3 = v.U3[c][t];
      const double fe2 = fma(1.5, u3, -0.5 * u0) - u2;
      const double fe1 = fma(4.0, u2, fma(-3.0, u0, -u1));
      const double fe0 = u1 - u0;
      acc = fma(2.0 / 3.0, v.L3[c][t] * fe2, acc);
      acc = fma(0.25, v.L2[c][t] * fe1, acc);
      acc = fma(v.L1[c][t], fe0, acc);
    }
  __shared__ double sh[256];
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if (threadIdx.x < h) sh[threadIdx.x] += sh[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) partials[blockIdx.x] = sh[0];
}

// the larger varrho wins; equal values: the smaller DoF id (class << 28 | index)
__device__ __forceinline__ void better(double &bv, long long &bi, double v, long long i) {
  if (v > bv || (v == bv && i < bi)) { bv = v; bi = i; }
}

// per block: the DoF of U^n with the largest varrho_1 and varrho_2 (point data set of U^n bound in d)
__global__ void __launch_bounds__(256) k_dt_argmax(const __grid_constant__ AfDev d, const __grid_constant__ AfGrid g,
                                                   double *pv, long long *pi) {
  double b1 = -1.0, b2 = -1.0;
  long long i1 = 1LL << 62, i2 = 1LL << 62;
  const long long PS = (long long)g.nxa * g.nya, stride = (long long)gridDim.x * blockDim.x;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < PS; t += stride) {
    const int i = (int)(t % g.nxa), j = (int)(t / g.nxa);
    for (int c = 0; c < 4; ++c) {
      if (i >= g.ex[c] || j >= g.ey[c]) continue;
      const long long id = ((long long)c << 28) | ((long long)j * g.ex[c] + i);
      double s1, s2;
      const double *w = d.pd[c];
      if (c == 0) {
        s1 = absd(w[QA_V1 * PS + t]) + w[QA_CF1 * PS + t];
        s2 = absd(w[QA_V2 * PS + t]) + w[QA_CF2 * PS + t];
      } else {
        s1 = w[QP_SR1 * PS + t];
        s2 = w[QP_SR2 * PS + t];
      }
      better(b1, i1, s1, id);
      better(b2, i2, s2, id);
    }
  }
  __shared__ double sv[2][256];
  __shared__ long long si[2][256];
  sv[0][threadIdx.x] = b1; si[0][threadIdx.x] = i1;
  sv[1][threadIdx.x] = b2; si[1][threadIdx.x] = i2;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if (threadIdx.x < h)
      for (int l = 0; l < 2; ++l) better(sv[l][threadIdx.x], si[l][threadIdx.x], sv[l][threadIdx.x + h], si[l][threadIdx.x + h]);
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int l = 0; l < 2; ++l) {
      pv[2 * blockIdx.x + l] = sv[l][0];
      pi[2 * blockIdx.x + l] = si[l][0];
    }
}

// one block: sums the dot partials, reduces the argmax partials, and adds
// mu * d(dt)/dU at the two maximising DoFs to lambda (class pointers)
__global__ void __launch_bounds__(256) k_dt_apply(const __grid_constant__ AfDev d, const __grid_constant__ AfGrid g,
                                                  const double *dpart, const double *pv, const long long *pi, int nb,
                                                  const __grid_constant__ OVec4 lam, double *mu_out) {
  __shared__ double sd[256], sv[2][256];
  __shared__ long long si[2][256];
  double a = 0.0, b1 = -1.0, b2 = -1.0;
  long long i1 = 1LL << 62, i2 = 1LL << 62;
  for (int k = threadIdx.x; k < nb; k += 256) {
    a += dpart[k];
    better(b1, i1, pv[2 * k], pi[2 * k]);
    better(b2, i2, pv[2 * k + 1], pi[2 * k + 1]);
  }
  sd[threadIdx.x] = a;
  sv[0][threadIdx.x] = b1; si[0][threadIdx.x] = i1;
  sv[1][threadIdx.x] = b2; si[1][threadIdx.x] = i2;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if (threadIdx.x < h) {
      sd[threadIdx.x] += sd[threadIdx.x + h];
      for (int l = 0; l < 2; ++l) better(sv[l][threadIdx.x], si[l][threadIdx.x], sv[l][threadIdx.x + h], si[l][threadIdx.x + h]);
    }
    __syncthreads();
  }
  if (threadIdx.x != 0) return;
  const double dt = d.sc->dt, mudt = sd[0];
  if (mu_out) *mu_out = mudt / dt;
  for (int l = 0; l < 2; ++l) {
    const long long id = si[l][0];
    const int c = (int)(id >> 28);
    const long long o = id & ((1LL << 28) - 1);
    const size_t cs = (size_t)g.ex[c] * g.ey[c];
    double U[8], grad[8];
    for (int k = 0; k < 8; ++k) U[k] = d.un[c][k * cs + o];
    Acc acc;
    acc_zero(acc);
    acc.sr[l] = 1.0;
    pointwise_transpose(U, g, acc, grad);                       // d varrho_l / dU at that DoF
    const double coef = -mudt * dt / g.cfl * (l == 0 ? g.rdx : g.rdy);   // mu * (-dt^2/cfl) / h_l
    for (int k = 0; k < 8; ++k) lam.p[c][k * cs + o] = fma(coef, grad[k], lam.p[c][k * cs + o]);
  }
}

}  // namespace

int af_adj_nslots() { return A_N; }

int af_dt_sens_nblocks() { return 152 * 4; }

void af_launch_dt_dot(const AfGrid &g, const double *const *L3, const double *const *L2, const double *const *L1,
                      const double *const *U0, const double *const *U1, const double *const *U2,
                      const double *const *U3, double *work, cudaStream_t s) {
  DtVec v;
  for (int c = 0; c < 4; ++c) {
    v.L3[c] = L3[c]; v.L2[c] = L2[c]; v.L1[c] = L1[c];
    v.U0[c] = U0[c]; v.U1[c] = U1[c]; v.U2[c] = U2[c]; v.U3[c] = U3[c];
    v.len[c] = 8LL * g.ex[c] * g.ey[c];
  }
  k_dt_dot<<<af_dt_sens_nblocks(), 256, 0, s>>>(v, work);
}

void af_launch_dt_apply(const AfDev &d, const AfGrid &g, double *const *lam, double *work, double *mu_out,
                        cudaStream_t s) {
  const int nb = af_dt_sens_nblocks();
  OVec4 lo;
  for (int c = 0; c < 4; ++c) lo.p[c] = lam[c];
  double *dpart = work, *pv = work + nb;
  long long *pi = reinterpret_cast<long long *>(work + 3 * nb);
  k_dt_argmax<<<nb, 256, 0, s>>>(d, g, pv, pi);
  k_dt_apply<<<1, 256, 0, s>>>(d, g, dpart, pv, pi, nb, lo, mu_out);
}
void af_launch_vjp(const AfDev &d, const AfGrid &g, const AfAdjEpi &e, double *a, double *zc, double *const *tpart,
                   cudaStream_t s, const double *co, double *const *vscaled) {
  Vec4 vv, vr;
  OVec4 tp, vs;
  for (int c = 0; c < 4; ++c) {
    vv.p[c] = e.v[c];
    vr.p[c] = e.v[c];
    tp.p[c] = tpart[c];
    vs.p[c] = co ? vscaled[c] : nullptr;
  }
  if (co) {   // frozen branch: point rows weighted by m (A0), then A1, A2 on those
    k_adj0<<<grid3(g.nxa, g.nya), dim3(32, 4), 0, s>>>(g, vr, vs, co);
    for (int c = 1; c < 4; ++c) vv.p[c] = vscaled[c];
  }
  k_adj1<<<grid3(g.nxa, g.nya), dim3(32, 4), 0, s>>>(d, g, vv, a, co);
  k_adj2<<<grid3(g.nxa, g.nya), dim3(32, 4), 0, s>>>(d, g, vv, a, tp, zc, co);
  if (co) k_adjl<<<grid3(g.nxa, g.nya), dim3(32, 4), 0, s>>>(d, g, vr, tp, co);
  k_adj3<<<grid3(g.nxa, g.nya), dim3(32, 4), 0, s>>>(g, zc, tp, e, co);
}
