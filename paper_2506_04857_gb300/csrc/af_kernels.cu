// af_kernels.cu -- sm_103a kernels of one SSP-RK3 stage of the positivity-
// preserving Active Flux scheme for 2D ideal MHD with the Godunov-Powell
// source term (Duan, Chandrashekar, Klingenberg, arXiv:2506.04857).
//
// The stage is split into five passes so that every FP64 quantity is formed
// exactly once (the FP64 pipe is the bound on GB300; the intermediates cost
// HBM traffic, of which there is plenty):
//   P1 k_pointdata : per DoF: primitives, F1, F2, spectral radii (Sec. 1, eq. cf);
//                    per cell: bi-parabola centre value + its limiter (Sec. 2.1,
//                    Remark 3.2); the running max of varrho for dt.
//   P2 k_points    : per x-face / y-face / corner: LLF-FVS update with the
//                    central Powell source (Sec. 2.3), first-order LLF point
//                    schemes and scaling limiter (Sec. 3.3), round-off shrink
//                    (Remark 4.1), RK combination; per cell: shock-sensor phi
//                    (Sec. 3.4).
//   P3 k_faces     : per face: Simpson flux (Sec. 2.2), LLF flux between the
//                    adjacent cell averages (eq. 2d_llf_flux), theta^s (Sec. 3.4).
//   P4 k_cells     : per cell: Powell source on the 3x3 Simpson nodes
//                    (eq. semi_av_src), S^LLF, the sensor blend, steps (1)-(2)
//                    of the parametrized flux limiter (Sec. 3.2) -> Lambda.
//   P5 k_final     : per cell: unique face coefficients (step (3)), limited
//                    update, round-off check, RK combination.
// A one-thread repair kernel applies the round-off shrink of Remark 4.1 to
// the (rare) cell averages that leave the admissible set.
//
// Limiter fast paths: where the paper's limiter provably returns theta = 1
// (all tested quantities clear 1e-13 by a wide margin) the blend is skipped;
// everywhere else the full procedure runs.  Results are identical.
#include "../../include/af.h"
#include "af_internal.h"
#include "af_math.cuh"
#include "af_device.cuh"

using namespace afm;

namespace {

// ---------------------------------------------------------------------------
// indexing helpers: af_device.cuh

// warp-aggregated event counters
__device__ __forceinline__ void count(AfStatus *st, int slot, bool pred) {
  unsigned act = __activemask();
  unsigned m = __ballot_sync(act, pred);
  if (m && (threadIdx.x & 31) == (__ffs(act) - 1)) atomicAdd(&st->cnt[slot], (unsigned long long)__popc(m));
}

// Slot of this thread in a work list (warp-aggregated; every active thread enqueues
// one entry), or -1 with the overflow bit set when the list is full.
__device__ __forceinline__ int enqueue(AfStatus *st, int *counter, int cap) {
  const unsigned act = __activemask();
  const int lane = threadIdx.x & 31, leader = __ffs(act) - 1;
  int base = 0;
  if (lane == leader) base = atomicAdd(counter, __popc(act));
  base = __shfl_sync(act, base, leader);
  const int slot = base + __popc(act & ((1u << lane) - 1u));
  if (slot >= cap) {
    atomicOr(&st->err, AFE_LIST_OVERFLOW);
    return -1;
  }
  return slot;
}

// ---------------------------------------------------------------------------
// L0 physics (Sec. 1)
// ---------------------------------------------------------------------------
__device__ __forceinline__ double pressure(const double *U, double gm1) {
  double m2 = fma(U[1], U[1], fma(U[2], U[2], U[3] * U[3]));
  double b2 = fma(U[4], U[4], fma(U[5], U[5], U[6] * U[6]));
  return gm1 * (U[7] - 0.5 * ddiv(m2, U[0]) - 0.5 * b2);
}
// q = rho E - |m|^2/2 - rho |B|^2/2 - rho c; q >= 0 <=> p >= (gamma-1) c for rho > 0
__device__ __forceinline__ double qform(const double *U, double c) {
  double m2 = fma(U[1], U[1], fma(U[2], U[2], mul_i(U[3], U[3])));
  double b2 = fma(U[4], U[4], fma(U[5], U[5], mul_i(U[6], U[6])));
  double t = fma(0.5, b2, c);
  return fma(-U[0], t, fma(U[0], U[7], ldexp_i<-1>(neg_i(m2))));
}
// A double as a float truncated toward zero (integer operations).  In range:
// 2^-60 <= |x| < 2^61 (every product of two such floats is a normal float) or x = 0.
// With small = true a value below 2^-60 is taken as 0 (and stays in range).
template <bool SMALL>
__device__ __forceinline__ float trunc_f32(double x, bool &ok) {
  const unsigned long long b = bits(x);
  const unsigned hi = (unsigned)(b >> 32), e = (hi >> 20) & 0x7ffu;
  const bool zero = SMALL ? e < 963u : (b << 1) == 0;
  ok = ok && (zero || e - 963u <= 120u);
  const unsigned fb = ((((hi & 0x7fffffffu) - (896u << 20)) << 3) | ((unsigned)b >> 29)) | (hi & 0x80000000u);
  return zero ? 0.0f : __uint_as_float(fb);
}
// True when q(U) = rho E - |m|^2/2 - rho (|B|^2/2 + c), c >= 0, is certainly > 0, from
// q and the sum S of the magnitudes of its terms evaluated in FP32 on the truncated
// inputs: each term then carries a relative error below 8 * 2^-23 and the combination
// two more roundings, so |q32 - q| < 10 * 2^-23 S < 1.3e-6 S.  Components of m and B
// below 2^-60 are taken as 0: they enter squared, |m|^2/2 then errs by < 2^-119 and
// rho |B|^2/2 by < rho 2^-119; with S >= rho (|E| + c), |E| + c > 2^-96 and S > 2^-96
// required, both stay below 2^-22 S (which also keeps negligible the absolute error
// of a product of three inputs below the normal FP32 range).  So q32 > 2^-16 S32
// implies q > 0 (and the FP64 qform > 0, whose error is about 1e-15 S).  An overflow
// makes S32 infinite.  False means undecided: the FP64 form decides.
__device__ __forceinline__ bool qform_cert32(const double *U, double c) {
  bool ok = true;
  float f[8];
  f[0] = trunc_f32<false>(U[0], ok);
  f[7] = trunc_f32<false>(U[7], ok);
#pragma unroll
  for (int k = 1; k < 7; ++k) f[k] = trunc_f32<true>(U[k], ok);
  const float cf = trunc_f32<false>(c, ok);
  const float m2 = fmaf(f[1], f[1], fmaf(f[2], f[2], f[3] * f[3]));
  const float b2 = fmaf(f[4], f[4], fmaf(f[5], f[5], f[6] * f[6]));
  const float t = fmaf(0.5f, b2, cf);
  const float q = fmaf(-f[0], t, fmaf(f[0], f[7], -0.5f * m2));
  const float S = fmaf(fabsf(f[0]), fabsf(f[7]), fmaf(0.5f, m2, fabsf(f[0]) * fabsf(t)));
  return ok && fabsf(f[7]) + cf > 0x1p-96f && S > 0x1p-96f && q > 0x1p-16f * S;
}
// qform(U, c) >= 0 in FP64, in a function that is not inlined (values by value): an
// inlined one is evaluated whether or not the FP32 certificate decided
__device__ __noinline__ bool qform_ge0(double u0, double u1, double u2, double u3, double u4, double u5, double u6,
                                       double u7, double c) {
  const double U[8] = {u0, u1, u2, u3, u4, u5, u6, u7};
  return ge_zero(qform(U, c));
}
// qform(U, 0) > 0 and finite in FP64 (not inlined, as above)
__device__ __noinline__ bool qform_gt0(double u0, double u1, double u2, double u3, double u4, double u5, double u6,
                                       double u7) {
  const double U[8] = {u0, u1, u2, u3, u4, u5, u6, u7};
  const double q = qform(U, 0.0);
  return (long long)bits(q) > 0 && finite_bits(q);
}
// rho >= 1e-13 and p >= 1e-13 (so every limiter of Sec. 3 leaves the state alone)
__device__ __forceinline__ bool clear_of_floor(const double *U, const AfGrid &g) {
  if (!ge_pos(U[0], 1e-13)) return false;
  if (qform_cert32(U, g.c13)) return true;
  return qform_ge0(U[0], U[1], U[2], U[3], U[4], U[5], U[6], U[7], g.c13);
}
__device__ __forceinline__ bool in_G(const double *U, double gm1) {
  for (int k = 0; k < 8; ++k)
    if (!isfinite(U[k])) return false;
  if (!(U[0] > 0.0)) return false;
  return pressure(U, gm1) > 0.0;
}

// Point data of one DoF (see QP_* / QA_* slots).  Returns varrho_1, varrho_2.
// avg = true stores the cell-average layout.
__device__ __forceinline__ void point_data(const double *U, const AfGrid &g, double *out, size_t PS, bool avg,
                                           double &sr1, double &sr2) {
  // The standalone products run on the integer pipes (mul_i, bitwise those of
  // DMUL), beside the FMAs and sums on the FP64 pipe.
  const double rho = U[0], r = rcp(rho);
  const double v1 = mul_i(U[1], r), v2 = mul_i(U[2], r), v3 = mul_i(U[3], r);
  const double B1 = U[4], B2 = U[5], B3 = U[6], E = U[7];
  const double b1s = mul_i(B1, B1), b2s = mul_i(B2, B2);
  const double BB = fma(B3, B3, b1s + b2s);
  const double mv = fma(U[1], v1, fma(U[2], v2, mul_i(U[3], v3)));
  const double p = mul_i(g.gm1, fma(-0.5, mv + BB, E));
  const double pt = fma(0.5, BB, p);
  const double vB = fma(v1, B1, fma(v2, B2, mul_i(v3, B3)));
  const double Ept = E + pt;
  const double f12 = fma(U[1], v2, -mul_i(B1, B2));   // rho v1 v2 - B1 B2 (F1[2] = F2[1])
  const double f15 = fma(v1, B2, -mul_i(B1, v2));     // v1 B2 - B1 v2    (F1[5] = -F2[4])
  double F1[7], F2[7];
  F1[0] = U[1];
  F1[1] = fma(U[1], v1, pt) - b1s;
  F1[2] = f12;
  F1[3] = fma(U[1], v3, -mul_i(B1, B3));
  F1[4] = f15;
  F1[5] = fma(v1, B3, -mul_i(B1, v3));
  F1[6] = fma(Ept, v1, -mul_i(B1, vB));
  F2[0] = U[2];
  F2[1] = f12;
  F2[2] = fma(U[2], v2, pt) - b2s;
  F2[3] = fma(U[2], v3, -mul_i(B2, B3));
  F2[4] = -f15;
  F2[5] = fma(v2, B3, -mul_i(B2, v3));
  F2[6] = fma(Ept, v2, -mul_i(B2, vB));
  // eq. (cf)
  const double c2 = mul_i(mul_i(g.gamma, p), r);
  const double a = fma(BB, r, c2);
  const double k4 = ldexp_i<2>(mul_i(c2, r));
  const double aa = mul_i(a, a), ha = ldexp_i<-1>(a);
  double d1 = fma(-k4, b1s, aa), d2 = fma(-k4, b2s, aa);
  d1 = gt_zero(d1) ? d1 : 0.0;
  d2 = gt_zero(d2) ? d2 : 0.0;
  const double cf1 = dsqrt(fma(0.5, dsqrt(d1), ha));
  const double cf2 = dsqrt(fma(0.5, dsqrt(d2), ha));
  sr1 = absd(v1) + cf1;
  sr2 = absd(v2) + cf2;
#pragma unroll
  for (int q = 0; q < 7; ++q) {
    out[(QP_F1 + q) * PS] = F1[q];
    out[(QP_F2 + q) * PS] = F2[q];
  }
  out[QP_V1 * PS] = v1;
  out[QP_V2 * PS] = v2;
  out[QP_V3 * PS] = v3;
  if (avg) {
    out[QA_CF1 * PS] = cf1;
    out[QA_CF2 * PS] = cf2;
    out[QA_PT * PS] = pt;
    out[QA_SRHO * PS] = dsqrt(rho);
  } else {
    out[QP_SR1 * PS] = sr1;
    out[QP_SR2 * PS] = sr2;
    out[QP_VB * PS] = vB;
  }
}

// Everything about one state needed by the LLF fluxes of the slow paths.
struct Full {
  double U[8], v[3], B[3], vB;
  double F[2][8];
  double cf[2], sr[2], srho;
};
__device__ __noinline__ void full_data(const double *U, const AfGrid &g, Full &d) {
  for (int k = 0; k < 8; ++k) d.U[k] = U[k];
  const double rho = U[0], r = rcp(rho);
  for (int k = 0; k < 3; ++k) d.v[k] = U[1 + k] * r;
  for (int k = 0; k < 3; ++k) d.B[k] = U[4 + k];
  const double B1 = d.B[0], B2 = d.B[1], B3 = d.B[2], E = U[7];
  const double v1 = d.v[0], v2 = d.v[1], v3 = d.v[2];
  const double BB = fma(B1, B1, fma(B2, B2, B3 * B3));
  const double mv = fma(U[1], v1, fma(U[2], v2, U[3] * v3));
  const double p = g.gm1 * fma(-0.5, mv + BB, E);
  const double pt = fma(0.5, BB, p);
  d.vB = fma(v1, B1, fma(v2, B2, v3 * B3));
  const double Ept = E + pt;
  d.F[0][0] = U[1];
  d.F[0][1] = fma(U[1], v1, pt) - B1 * B1;
  d.F[0][2] = fma(U[1], v2, -B1 * B2);
  d.F[0][3] = fma(U[1], v3, -B1 * B3);
  d.F[0][4] = 0.0;
  d.F[0][5] = fma(v1, B2, -B1 * v2);
  d.F[0][6] = fma(v1, B3, -B1 * v3);
  d.F[0][7] = fma(Ept, v1, -B1 * d.vB);
  d.F[1][0] = U[2];
  d.F[1][1] = d.F[0][2];
  d.F[1][2] = fma(U[2], v2, pt) - B2 * B2;
  d.F[1][3] = fma(U[2], v3, -B2 * B3);
  d.F[1][4] = -d.F[0][5];
  d.F[1][5] = 0.0;
  d.F[1][6] = fma(v2, B3, -B2 * v3);
  d.F[1][7] = fma(Ept, v2, -B2 * d.vB);
  const double c2 = g.gamma * p * r;
  const double a = fma(BB, r, c2);
  const double k4 = 4.0 * (c2 * r);
  for (int l = 0; l < 2; ++l) {
    double dd = fma(-k4, d.B[l] * d.B[l], a * a);
    dd = dd > 0.0 ? dd : 0.0;
    d.cf[l] = dsqrt(fma(0.5, dsqrt(dd), 0.5 * a));
    d.sr[l] = absd(d.v[l]) + d.cf[l];
  }
  d.srho = dsqrt(rho);
}

// Lemma 3.1 with equality: alpha^LLF = max{varrho, varrho~, alpha*(U,U~), alpha*(U~,U)}
// = max(|v|, |v~|, |sqrt(rho) v + sqrt(rho~) v~|/(sqrt(rho)+sqrt(rho~)))
//   + max(c_f, c_f~) + |B - B~|/(sqrt(rho)+sqrt(rho~)),
// which dominates both spectral radii.
__device__ __forceinline__ double alpha_llf(double va, double vb, double cfa, double cfb, double sra, double srb,
                                            const double *Ba, const double *Bb) {
  const double rden = rcp(sra + srb);
  const double roe = mul_i(absd(fma(sra, va, mul_i(srb, vb))), rden);
  const double d0 = Ba[0] - Bb[0], d1 = Ba[1] - Bb[1], d2 = Ba[2] - Bb[2];
  const double nb = dsqrt(fma(d0, d0, fma(d1, d1, mul_i(d2, d2))));
  const double mv = maxnn(maxnn(absd(va), absd(vb)), roe);
  return mv + maxnn(cfa, cfb) + nb * rden;
}

__device__ void llf_flux_full(int l, const Full &u, const Full &w, double *F) {
  const double al = alpha_llf(u.v[l], w.v[l], u.cf[l], w.cf[l], u.srho, w.srho, u.B, w.B);
  for (int k = 0; k < 8; ++k) F[k] = 0.5 * (fma(-al, w.U[k] - u.U[k], u.F[l][k] + w.F[l][k]));
}

// Sec. 3.3 scaling limiter toward the safe state UL (theta*, then theta**).
__device__ void scaling_limiter(const double *UH, const double *UL, double gm1, double *out, double &t1, double &t2) {
  const double rhoL = UL[0], pL = pressure(UL, gm1);
  const double eps_rho = fmin(1e-13, rhoL), eps_p = fmin(1e-13, pL);
  t1 = 1.0;
  if (UH[0] < eps_rho) t1 = ddiv(rhoL - eps_rho, rhoL - UH[0]);
  double Us[8];
  for (int k = 0; k < 8; ++k) Us[k] = UH[k];
  Us[0] = fma(t1, UH[0], (1.0 - t1) * rhoL);
  const double ps = pressure(Us, gm1);
  t2 = 1.0;
  if (ps < eps_p) t2 = ddiv(pL - eps_p, pL - ps);
  for (int k = 0; k < 8; ++k) out[k] = fma(t2, Us[k], (1.0 - t2) * UL[k]);
}

// The scaling limiter's result for given theta*, theta** (frozen branch).
__device__ void scaling_blend(const double *UH, const double *UL, double t1, double t2, double *out) {
  double Us[8];
  for (int k = 0; k < 8; ++k) Us[k] = UH[k];
  Us[0] = fma(t1, UH[0], (1.0 - t1) * UL[0]);
  for (int k = 0; k < 8; ++k) out[k] = fma(t2, Us[k], (1.0 - t2) * UL[k]);
}

// ---------------------------------------------------------------------------
// P1: point data, cell-centre values, dt reduction
// ---------------------------------------------------------------------------
__device__ __forceinline__ void load8(const SV &v, int i, int j, double *U) {
#pragma unroll
  for (int k = 0; k < 8; ++k) U[k] = v(i, j, k);
}

// Sec. 2.1 centre value [36 Ubar - 4 (faces) - (corners)] / 16 of cell (i, j),
// limited toward the cell average A by Remark 3.2; true when the limiter acted.
__device__ __forceinline__ bool centre_value(const AfDev &d, const AfGrid &g, int i, int j, const double *A,
                                             double *uc) {
  const SV X = sview(d.us[1], g, 1), Y = sview(d.us[2], g, 2), C = sview(d.us[3], g, 3);
  const int ip = mface(i + 1, g.nx, g.bc), jp = mface(j + 1, g.ny, g.bc);
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const double faces = (X(i, j, k) + X(ip, j, k)) + (Y(i, j, k) + Y(i, jp, k));
    const double corners = (C(i, j, k) + C(ip, j, k)) + (C(i, jp, k) + C(ip, jp, k));
    uc[k] = fma(2.25, A[k], fma(-0.25, faces, ldexp_i<-4>(neg_i(corners))));
  }
  const size_t PS = (size_t)g.nxa * g.nya, o = (size_t)j * g.nxa + i;
  double t1 = 1.0, t2 = 1.0;
  if (d.frz) {   // frozen branch: the recorded theta*, theta**
    t1 = d.frz[AFC_C1 * PS + o];
    t2 = d.frz[AFC_C2 * PS + o];
    if (!(t1 == 1.0 && t2 == 1.0)) {
      double out[8];
      scaling_blend(uc, A, t1, t2, out);
      for (int k = 0; k < 8; ++k) uc[k] = out[k];
    }
  } else if (!clear_of_floor(uc, g)) {
    double out[8];
    scaling_limiter(uc, A, g.gm1, out, t1, t2);
    for (int k = 0; k < 8; ++k) uc[k] = out[k];
  }
  if (d.rec) {
    d.rec[AFC_C1 * PS + o] = t1;
    d.rec[AFC_C2 * PS + o] = t2;
  }
  return lt_one(t1) || lt_one(t2);   // theta in [0, 1]
}

__device__ __forceinline__ void b_pointdata(const AfDev &d, const AfGrid &g, const int i, const int j, int reduce_dt) {
  const size_t PS = (size_t)g.nxa * g.nya;
  const size_t o = (size_t)j * g.nxa + i;
  double m1 = 0.0, m2 = 0.0;
  bool clim = false;
  if (i < g.nxa && j < g.nya) {
    // the five points of index (i, j) -- x-face, y-face, corner, cell average, cell
    // centre -- through one instance of point_data (one copy of its code)
    double A[8];
#pragma unroll 1
    for (int c = 1; c <= 5; ++c) {
      double U[8];
      if (c <= 3) {
        if (!(i < g.ex[c] && j < g.ey[c])) continue;
        load8(sview(d.us[c], g, c), i, j, U);
      } else {
        if (!(i < g.nx && j < g.ny)) break;
        if (c == 4) {
          load8(sview(d.us[0], g, 0), i, j, A);
#pragma unroll
          for (int k = 0; k < 8; ++k) U[k] = A[k];
        } else {
          clim = centre_value(d, g, i, j, A, U);
#pragma unroll
          for (int k = 0; k < 8; ++k) d.uc[k * PS + o] = U[k];
        }
      }
      double s1, s2;
      point_data(U, g, d.pd[c == 5 ? 4 : (c == 4 ? 0 : c)] + o, PS, c == 4, s1, s2);
      if (c <= 4) {   // the centre is not a DoF: not in the time-step bound
        m1 = maxnn(m1, s1);
        m2 = maxnn(m2, s2);
      }
    }
  }
  count(d.st, ST_CENTER_LIMITED, clim);
  if (reduce_dt) {
    unsigned long long b1 = (unsigned long long)__double_as_longlong(m1);
    unsigned long long b2 = (unsigned long long)__double_as_longlong(m2);
    for (int off = 16; off > 0; off >>= 1) {
      unsigned long long o1 = __shfl_down_sync(0xffffffffu, b1, off);
      unsigned long long o2 = __shfl_down_sync(0xffffffffu, b2, off);
      b1 = o1 > b1 ? o1 : b1;
      b2 = o2 > b2 ? o2 : b2;
    }
    if ((threadIdx.x & 31) == 0) {
      atomicMax(&d.sc->smax[0], b1);
      atomicMax(&d.sc->smax[1], b2);
    }
  }
}

// dt = cfl / (max varrho_1 / dx + max varrho_2 / dy) over the four DoF classes of U^n.
__device__ void b_dt(const AfDev &d, const AfGrid &g) {
  const double m1 = __longlong_as_double((long long)d.sc->smax[0]);
  const double m2 = __longlong_as_double((long long)d.sc->smax[1]);
  const double dt = g.cfl / (m1 / g.dx + m2 / g.dy);
  d.sc->dt = dt;
  d.sc->smax[0] = 0ull;
  d.sc->smax[1] = 0ull;
  if (!isfinite(dt) || !(dt > 0.0)) atomicOr(&d.st->err, AFE_NONFINITE_DT);
}

// ---------------------------------------------------------------------------
// P2: point values (Sec. 2.3, 3.3) and the sensor (Sec. 3.4)
// ---------------------------------------------------------------------------
// A point on an FVS line: state view + work view + index (cls 4 = cell centre).
struct PP {
  const double *u;   // state base (class array or centre array)
  size_t ucs;        // component stride of u
  int uex;           // row length of u
  const double *w;   // point data base
  int i, j;
};

__device__ __forceinline__ PP pref(const AfDev &d, const AfGrid &g, int c, int i, int j) {
  PP p;
  if (c == 4) {
    p.u = d.uc;
    p.ucs = (size_t)g.nxa * g.nya;
    p.uex = g.nxa;
  } else {
    p.u = d.us[c];
    p.ucs = (size_t)g.ex[c] * g.ey[c];
    p.uex = g.ex[c];
  }
  p.w = d.pd[c];
  p.i = i;
  p.j = j;
  return p;
}
__device__ __forceinline__ double pu(const PP &p, int k) { return __ldg(p.u + (size_t)k * p.ucs + (size_t)p.j * p.uex + p.i); }
__device__ __forceinline__ double pw(const PP &p, size_t PS, int nxa, int q) {
  return __ldg(p.w + (size_t)q * PS + (size_t)p.j * nxa + p.i);
}

// ---- reflective and inflow sides -------------------------------------------
// Kernels are instantiated twice: GB = false (periodic or mirror outflow on all
// sides: ghost indices map onto interior DoFs) and GB = true (some side
// reflective or inflow).  With GB a ghost index is mapped along x first
// (mirror; a reflective side negates m1, B1 and the point-data slots that
// change sign with them), then along y (mirror; reflective: m2, B2; inflow:
// the inflow state where the x coordinate of the x-mapped index lies inside
// the inflow range).  Reading: the paper names the conditions only (Example 4.8).
constexpr unsigned kFlipUx = (1u << 1) | (1u << 4), kFlipUy = (1u << 2) | (1u << 5);
// point-data slots (QP and QA share the positions that change sign): F1 and F2
// without their B_l component, v1 / v2
constexpr unsigned kFlipWx = (1u << 0) | (1u << 2) | (1u << 3) | (1u << 4) | (1u << 5) | (1u << 6) | (1u << 8) |
                             (1u << 11) | (1u << 16);
constexpr unsigned kFlipWy = (1u << 2) | (1u << 4) | (1u << 7) | (1u << 8) | (1u << 10) | (1u << 11) | (1u << 12) |
                             (1u << 13) | (1u << 17);

struct GR {
  int i, j;        // mapped index
  unsigned um, wm; // sign masks of the state components and of the point-data slots
  bool in;         // the inflow state
};
// cls 0 average, 1 x-face, 2 y-face, 3 corner, 4 cell centre; (i, j) unmapped
__device__ __forceinline__ GR gres(const AfGrid &g, int cls, int i, int j) {
  const bool xf = cls == 1 || cls == 3, yf = cls == 2 || cls == 3;
  const int nxe = xf ? g.nx + 1 : g.nx, nye = yf ? g.ny + 1 : g.ny;
  GR r;
  r.um = r.wm = 0u;
  r.in = false;
  r.i = xf ? mface(i, g.nx, g.bc) : mcell(i, g.nx, g.bc);
  r.j = yf ? mface(j, g.ny, g.bc) : mcell(j, g.ny, g.bc);
  if ((i < 0 || i >= nxe) && g.side[i < 0 ? 0 : 1] == 1) {
    r.um ^= kFlipUx;
    r.wm ^= kFlipWx;
  }
  if (j < 0 || j >= nye) {
    const int sd = g.side[j < 0 ? 2 : 3];
    if (sd == 1) {
      r.um ^= kFlipUy;
      r.wm ^= kFlipWy;
    } else if (sd == 2) {
      const double x = g.x0 + (r.i + (xf ? 0.0 : 0.5)) * g.dx;
      r.in = x > g.in_lo && x < g.in_hi;
    }
  }
  return r;
}
__device__ __forceinline__ double flipv(double v, unsigned mask, int k) { return ((mask >> k) & 1u) ? -v : v; }

// a point on an FVS line with its own point-data strides and sign masks
struct PPG {
  PP p;
  size_t wps;
  int wnx;
  unsigned um, wm;
};
__device__ __forceinline__ PPG prefg(const AfDev &d, const AfGrid &g, int c, int i, int j) {
  const GR r = gres(g, c, i, j);
  PPG q;
  if (r.in) {
    q.p.u = d.inflow;
    q.p.ucs = 1;
    q.p.uex = 0;
    q.p.w = d.inflow + 8 + (c == 0 ? AF_NQP : 0);
    q.p.i = q.p.j = 0;
    q.wps = 1;
    q.wnx = 0;
    q.um = q.wm = 0u;
  } else {
    q.p = pref(d, g, c, r.i, r.j);
    q.wps = (size_t)g.nxa * g.nya;
    q.wnx = g.nxa;
    q.um = r.um;
    q.wm = r.wm;
  }
  return q;
}
__device__ __forceinline__ double pug(const PPG &q, int k) { return flipv(pu(q.p, k), q.um, k); }
__device__ __forceinline__ double pwg(const PPG &q, int s) {
  return flipv(__ldg(q.p.w + (size_t)s * q.wps + (size_t)q.p.j * q.wnx + q.p.i), q.wm, s);
}
// the 8 state values of DoF (cls, i, j) (unmapped; cls 0..3)
template <bool GB>
__device__ __forceinline__ void gload8(const AfDev &d, const AfGrid &g, int cls, int i, int j, double *U) {
  if constexpr (GB) {
    const PPG q = prefg(d, g, cls, i, j);
#pragma unroll
    for (int k = 0; k < 8; ++k) U[k] = pug(q, k);
  } else {
    const int mi = (cls == 1 || cls == 3) ? mface(i, g.nx, g.bc) : mcell(i, g.nx, g.bc);
    const int mj = (cls == 2 || cls == 3) ? mface(j, g.ny, g.bc) : mcell(j, g.ny, g.bc);
    const SV v = sview(d.us[cls], g, cls);
#pragma unroll
    for (int k = 0; k < 8; ++k) U[k] = v(mi, mj, k);
  }
}

// 2h times the derivative of B_l at the middle point of a line (spacing h/2)
// for the point source: the central (D+ B + D- B)/2 of Sec. 2.3 gives
// (B0 - B4) + 4 (B3 - B1); the velocity-upwind variant of Example 4.2 takes
// D+ B = (B0 - 4 B1 + 3 B2)/h for upw > 0 and D- B = (4 B3 - B4 - 3 B2)/h for upw < 0.
__device__ __forceinline__ double b_line(double u0, double u1, double u2, double u3, double u4, int upw) {
  if (upw > 0) return 2.0 * fma(3.0, u2, fma(-4.0, u1, u0));
  if (upw < 0) return 2.0 * fma(-3.0, u2, fma(4.0, u3, -u4));
  return fma(4.0, u3 - u1, u0 - u4);
}

// Upwind selector of the Example 4.2 variant: the sign of v_l at the point, or 0.
__device__ __forceinline__ int upwind_sign(const AfGrid &g, double vl) {
  if (!g.upwind) return 0;
  return vl > 0.0 ? 1 : (vl < 0.0 ? -1 : 0);
}

// Accumulate -c * [ (D+ F+ + D- F-) * h ] of direction l along the line P[0..4]
// into acc (per component), with F^pm = (F +- alpha U)/2.  Writing out D+ and D-:
// (D+F+ + D-F-) h = ((F0 - F4) + 4 (F3 - F1) + alpha ((U0 + U4) - 4 (U1 + U3) + 6 U2)) / 2.
// Also returns 2h times the derivative of B_l for the point source in dBl (b_line).
template <int L>
__device__ __forceinline__ void fvs_line(const PP *P, size_t PS, int nxa, double c, double *acc, double &dBl,
                                         int upw) {
  const int qsr = L == 0 ? QP_SR1 : QP_SR2;
  double al = pw(P[0], PS, nxa, qsr);
#pragma unroll
  for (int q = 1; q < 5; ++q) al = maxnn(al, pw(P[q], PS, nxa, qsr));
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const double u0 = pu(P[0], k), u1 = pu(P[1], k), u2 = pu(P[2], k), u3 = pu(P[3], k), u4 = pu(P[4], k);
    const double up = fma(6.0, u2, fma(-4.0, u1 + u3, u0 + u4));
    double dk;
    if (k == 4 + L) {
      dk = mul_i(al, up);
      dBl = b_line(u0, u1, u2, u3, u4, upw);
    } else {
      const int s = (L == 0 ? QP_F1 : QP_F2) + fslot(L, k);
      const double f0 = pw(P[0], PS, nxa, s), f1 = pw(P[1], PS, nxa, s), f3 = pw(P[3], PS, nxa, s),
                   f4 = pw(P[4], PS, nxa, s);
      dk = fma(al, up, fma(4.0, f3 - f1, f0 - f4));
    }
    acc[k] = fma(-c, dk, acc[k]);
  }
}

// fvs_line on ghost-aware points (reflective / inflow sides)
template <int L>
__device__ __forceinline__ void fvs_line_g(const PPG *P, double c, double *acc, double &dBl, int upw) {
  const int qsr = L == 0 ? QP_SR1 : QP_SR2;
  double al = pwg(P[0], qsr);
#pragma unroll
  for (int q = 1; q < 5; ++q) al = maxnn(al, pwg(P[q], qsr));
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const double u0 = pug(P[0], k), u1 = pug(P[1], k), u2 = pug(P[2], k), u3 = pug(P[3], k), u4 = pug(P[4], k);
    const double up = fma(6.0, u2, fma(-4.0, u1 + u3, u0 + u4));
    double dk;
    if (k == 4 + L) {
      dk = al * up;
      dBl = b_line(u0, u1, u2, u3, u4, upw);
    } else {
      const int s = (L == 0 ? QP_F1 : QP_F2) + fslot(L, k);
      dk = fma(al, up, fma(4.0, pwg(P[3], s) - pwg(P[1], s), pwg(P[0], s) - pwg(P[4], s)));
    }
    acc[k] = fma(-c, dk, acc[k]);
  }
}

// Central derivative of F_l between two points lo, hi: acc -= c (F(hi) - F(lo)).
template <int L>
__device__ __forceinline__ void central_line(const PP &lo, const PP &hi, size_t PS, int nxa, double c, double *acc,
                                             double &dBl) {
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    if (k == 4 + L) {
      dBl = pu(hi, k) - pu(lo, k);
      continue;
    }
    const int s = (L == 0 ? QP_F1 : QP_F2) + fslot(L, k);
    acc[k] = fma(-c, pw(hi, PS, nxa, s) - pw(lo, PS, nxa, s), acc[k]);
  }
}

// First-order LLF state of Sec. 3.3 for one point value (cls 1, 2, 3 at (i,j)).
template <bool GB>
__device__ __noinline__ void point_llf_state(const AfDev &d, const AfGrid &g, int cls, int i, int j, double dt,
                                             double *UL) {
  // neighbours (class, unmapped index) for the x and y fluxes (left/low, right/high)
  int cx[2], ix[2], jx[2], cy[2], iy[2], jy[2];
  if (cls == 3) {
    cx[0] = cx[1] = 3; ix[0] = i - 1; ix[1] = i + 1; jx[0] = jx[1] = j;
    cy[0] = cy[1] = 3; iy[0] = iy[1] = i; jy[0] = j - 1; jy[1] = j + 1;
  } else if (cls == 1) {
    cx[0] = cx[1] = 1; ix[0] = i - 1; ix[1] = i + 1; jx[0] = jx[1] = j;
    cy[0] = cy[1] = 3; iy[0] = iy[1] = i; jy[0] = j; jy[1] = j + 1;
  } else {
    cx[0] = cx[1] = 3; ix[0] = i; ix[1] = i + 1; jx[0] = jx[1] = j;
    cy[0] = cy[1] = 2; iy[0] = iy[1] = i; jy[0] = j - 1; jy[1] = j + 1;
  }
  double U[8];
  load8(sview(d.us[cls], g, cls), i, j, U);
  Full me, nb;
  full_data(U, g, me);
  double Fxl[8], Fxr[8], Fyl[8], Fyr[8];
  gload8<GB>(d, g, cx[0], ix[0], jx[0], U);
  full_data(U, g, nb);
  llf_flux_full(0, nb, me, Fxl);
  const double b1l = nb.B[0];
  gload8<GB>(d, g, cx[1], ix[1], jx[1], U);
  full_data(U, g, nb);
  llf_flux_full(0, me, nb, Fxr);
  const double b1r = nb.B[0];
  gload8<GB>(d, g, cy[0], iy[0], jy[0], U);
  full_data(U, g, nb);
  llf_flux_full(1, nb, me, Fyl);
  const double b2l = nb.B[1];
  gload8<GB>(d, g, cy[1], iy[1], jy[1], U);
  full_data(U, g, nb);
  llf_flux_full(1, me, nb, Fyr);
  const double b2r = nb.B[1];
  // Reading: the printed stencils are used literally (fluxes between values
  // half a cell apart are still divided by dx or dy; divergence over 2 dx, 2 dy).
  const double divB = (b1r - b1l) * (0.5 * g.rdx) + (b2r - b2l) * (0.5 * g.rdy);
  const double Ps[8] = {0.0, me.B[0], me.B[1], me.B[2], me.v[0], me.v[1], me.v[2], me.vB};
  const double cxf = dt * g.rdx, cyf = dt * g.rdy;
  for (int k = 0; k < 8; ++k) {
    double u = me.U[k] - cxf * (Fxr[k] - Fxl[k]) - cyf * (Fyr[k] - Fyl[k]);
    if (g.src_point_on) u -= dt * divB * Ps[k];
    UL[k] = u;
  }
}

// Slow path of Sec. 3.3 for one point value: its first-order LLF state, the
// scaling limiter and the round-off shrink.  t1o, t2o: the theta*, theta** taken
// (theta** after the shrink; 0 for the fall-back to the LLF state).
template <bool GB>
__device__ __noinline__ void point_pp(const AfDev &d, const AfGrid &g, int cls, int i, int j, const double *UH,
                                      double dt, double *out, int &limited, int &shrunk, int &bad, double &t1o,
                                      double &t2o) {
  double UL[8];
  point_llf_state<GB>(d, g, cls, i, j, dt, UL);
  double t1, t2;
  scaling_limiter(UH, UL, g.gm1, out, t1, t2);
  t1o = t1;
  t2o = t2;
  limited = (t1 < 1.0 || t2 < 1.0);
  shrunk = 0;
  bad = 0;
  if (!in_G(out, g.gm1)) {
    // Remark 4.1: theta** lowered by 2^m 1e-8, m = 0..9, else the LLF state
    shrunk = 1;
    double Us[8];
    for (int k = 0; k < 8; ++k) Us[k] = UH[k];
    Us[0] = fma(t1, UH[0], (1.0 - t1) * UL[0]);
    bool ok = false;
    for (int m = 0; m < 10 && !ok; ++m) {
      const double th = fmax(0.0, t2 - ldexp(1e-8, m));
      for (int k = 0; k < 8; ++k) out[k] = fma(th, Us[k], (1.0 - th) * UL[k]);
      ok = in_G(out, g.gm1);
      t2o = th;
    }
    if (!ok) {
      for (int k = 0; k < 8; ++k) out[k] = UL[k];
      t2o = 0.0;
    }
    bad = !in_G(out, g.gm1);
  }
}

// Shock-sensor values of cell (ci, cj) (ghost cells allowed) from the cell
// averages around it, with boundary-mapped neighbour indices (Sec. 3.4).
// Reading: phi_1 is differenced along x for x-faces and along y for y-faces.
template <bool GB>
__device__ void sensor_phi(const AfDev &d, const AfGrid &g, int ci, int cj, double *phi) {
  // slot q of the average's point data and component k of the average, cell (a, b) unmapped
  auto A = [&](int a, int b, int q) -> double {
    if constexpr (GB) {
      return pwg(prefg(d, g, 0, a, b), q);
    } else {
      return __ldg(d.pd[0] + (size_t)q * g.nxa * g.nya + (size_t)mcell(b, g.ny, g.bc) * g.nxa + mcell(a, g.nx, g.bc));
    }
  };
  auto Ub = [&](int a, int b, int k) -> double {
    if constexpr (GB) {
      return pug(prefg(d, g, 0, a, b), k);
    } else {
      return __ldg(d.us[0] + (size_t)k * g.nx * g.ny + (size_t)mcell(b, g.ny, g.bc) * g.nx + mcell(a, g.nx, g.bc));
    }
  };
  const int e = ci + 1, w = ci - 1, n = cj + 1, s = cj - 1;
  const double ptc = A(ci, cj, QA_PT), pte = A(e, cj, QA_PT), ptw = A(w, cj, QA_PT);
  const double ptn = A(ci, n, QA_PT), pts = A(ci, s, QA_PT);
  const double sx = pte + ptw, sy = ptn + pts;
  phi[0] = ddiv(absd(fma(-2.0, ptc, sx)), absd(fma(2.0, ptc, sx)));
  phi[1] = ddiv(absd(fma(-2.0, ptc, sy)), absd(fma(2.0, ptc, sy)));
  const double hx = 0.5 * g.rdx, hy = 0.5 * g.rdy;
  const double divv = fma(A(e, cj, QA_V1) - A(w, cj, QA_V1), hx, mul_i(A(ci, n, QA_V2) - A(ci, s, QA_V2), hy));
  const double curl = fma(A(e, cj, QA_V2) - A(w, cj, QA_V2), hx, -mul_i(A(ci, n, QA_V1) - A(ci, s, QA_V1), hy));
  if (is_zero(divv)) {   // -0 / den gives 0: no square root or quotient needed
    phi[2] = 0.0;
  } else {
    const double den = dsqrt(fma(divv, divv, fma(curl, curl, 1e-40)));
    const double ph2 = ddiv(-divv, den);
    phi[2] = gt_zero(ph2) ? ph2 : 0.0;
  }
  const double num = (Ub(e, cj, 4) - Ub(w, cj, 4)) + (Ub(ci, n, 5) - Ub(ci, s, 5));
  phi[3] = ddiv(absd(num), absd(Ub(ci, cj, 4) + Ub(ci, cj, 5)) + 1e-40);
}

template <bool GB, bool UP>
__device__ __forceinline__ void b_points(const AfDev &d, const AfGrid &g, const int i, const int j, double a, double b,
                                         int mode) {
  const size_t PS = (size_t)g.nxa * g.nya;
  const double dt = mode == 1 ? 1.0 : d.sc->dt;
  const double cxc = mul_i(dt, g.rdx), cyc = mul_i(dt, g.rdy);   // central differences
  const double cx = ldexp_i<-1>(cxc), cy = ldexp_i<-1>(cyc);      // the FVS lines carry a factor 1/2
  int nlim = 0, nshr = 0, nbad = 0;
  if (i < g.nxa && j < g.nya) {
    const int im = mface(i - 1, g.nx, g.bc), ip = mface(i + 1, g.nx, g.bc);
    const int jm = mface(j - 1, g.ny, g.bc), jp = mface(j + 1, g.ny, g.bc);
    const int ci0 = mcell(i - 1, g.nx, g.bc), ci1 = mcell(i, g.nx, g.bc);
    const int cj0 = mcell(j - 1, g.ny, g.bc), cj1 = mcell(j, g.ny, g.bc);
#pragma unroll 1
    for (int cls = 1; cls <= 3; ++cls) {
      if (mode == 2 || !(i < g.ex[cls] && j < g.ey[cls])) continue;   // mode 2: sensor only
      const PP me = pref(d, g, cls, i, j);
      double acc[8];   // U + dt L(U) for a stage, L(U) itself for the rhs (mode 1)
#pragma unroll
      for (int k = 0; k < 8; ++k) acc[k] = mode == 1 ? 0.0 : pu(me, k);
      double dBx, dBy, divB;
      if constexpr (GB) {   // lines through reflective / inflow ghosts (unmapped indices)
        const PPG mg = prefg(d, g, cls, i, j);
        if (cls == 3) {
          const PPG Px[5] = {prefg(d, g, 3, i - 1, j), prefg(d, g, 2, i - 1, j), mg, prefg(d, g, 2, i, j),
                             prefg(d, g, 3, i + 1, j)};
          const PPG Py[5] = {prefg(d, g, 3, i, j - 1), prefg(d, g, 1, i, j - 1), mg, prefg(d, g, 1, i, j),
                             prefg(d, g, 3, i, j + 1)};
          fvs_line_g<0>(Px, cx, acc, dBx, (UP ? upwind_sign(g, pw(me, PS, g.nxa, QP_V1)) : 0));
          fvs_line_g<1>(Py, cy, acc, dBy, (UP ? upwind_sign(g, pw(me, PS, g.nxa, QP_V2)) : 0));
          divB = fma(dBx, 0.5 * g.rdx, mul_i(dBy, 0.5 * g.rdy));
        } else if (cls == 1) {
          const PPG Px[5] = {prefg(d, g, 1, i - 1, j), prefg(d, g, 4, i - 1, j), mg, prefg(d, g, 4, i, j),
                             prefg(d, g, 1, i + 1, j)};
          fvs_line_g<0>(Px, cx, acc, dBx, (UP ? upwind_sign(g, pw(me, PS, g.nxa, QP_V1)) : 0));
          central_line<1>(pref(d, g, 3, i, j), pref(d, g, 3, i, jp), PS, g.nxa, cyc, acc, dBy);
          divB = fma(dBx, 0.5 * g.rdx, mul_i(dBy, g.rdy));
        } else {
          central_line<0>(pref(d, g, 3, i, j), pref(d, g, 3, ip, j), PS, g.nxa, cxc, acc, dBx);
          const PPG Py[5] = {prefg(d, g, 2, i, j - 1), prefg(d, g, 4, i, j - 1), mg, prefg(d, g, 4, i, j),
                             prefg(d, g, 2, i, j + 1)};
          fvs_line_g<1>(Py, cy, acc, dBy, (UP ? upwind_sign(g, pw(me, PS, g.nxa, QP_V2)) : 0));
          divB = fma(dBx, g.rdx, mul_i(dBy, 0.5 * g.rdy));
        }
      } else {
        // the x line, then the y line of the point (one instance of each form): an FVS
        // line through points half a cell apart, or, for the other direction of a face
        // point, the central difference between the corners at its ends
        if (cls == 2) {
          central_line<0>(pref(d, g, 3, i, j), pref(d, g, 3, ip, j), PS, g.nxa, cxc, acc, dBx);
        } else {
          const int cm = cls == 3 ? 2 : 4;   // between the points: y-faces (corner), centres (x-face)
          const PP Px[5] = {pref(d, g, cls, im, j), pref(d, g, cm, ci0, j), me, pref(d, g, cm, ci1, j),
                            pref(d, g, cls, ip, j)};
          fvs_line<0>(Px, PS, g.nxa, cx, acc, dBx, (UP ? upwind_sign(g, pw(me, PS, g.nxa, QP_V1)) : 0));
        }
        if (cls == 1) {
          central_line<1>(pref(d, g, 3, i, j), pref(d, g, 3, i, jp), PS, g.nxa, cyc, acc, dBy);
        } else {
          const int cm = cls == 3 ? 1 : 4;   // x-faces (corner), centres (y-face)
          const PP Py[5] = {pref(d, g, cls, i, jm), pref(d, g, cm, i, cj0), me, pref(d, g, cm, i, cj1),
                            pref(d, g, cls, i, jp)};
          fvs_line<1>(Py, PS, g.nxa, cy, acc, dBy, (UP ? upwind_sign(g, pw(me, PS, g.nxa, QP_V2)) : 0));
        }
        divB = fma(dBx, cls == 2 ? g.rdx : 0.5 * g.rdx, mul_i(dBy, cls == 1 ? g.rdy : 0.5 * g.rdy));
      }
      if (g.src_point_on) {
        // -(div B) Psi(U), Psi = (0, B, v, v.B)
        const double sdt = mul_i(dt, divB);
        acc[1] = fma(-sdt, pu(me, 4), acc[1]);
        acc[2] = fma(-sdt, pu(me, 5), acc[2]);
        acc[3] = fma(-sdt, pu(me, 6), acc[3]);
        acc[4] = fma(-sdt, pw(me, PS, g.nxa, QP_V1), acc[4]);
        acc[5] = fma(-sdt, pw(me, PS, g.nxa, QP_V2), acc[5]);
        acc[6] = fma(-sdt, pw(me, PS, g.nxa, QP_V3), acc[6]);
        acc[7] = fma(-sdt, pw(me, PS, g.nxa, QP_VB), acc[7]);
      }
      double *uo = d.uo[cls];
      const size_t cs = (size_t)g.ex[cls] * g.ey[cls], oo = (size_t)j * g.ex[cls] + i;
      if (mode == 1) {   // semi-discrete right-hand side
#pragma unroll
        for (int k = 0; k < 8; ++k) uo[k * cs + oo] = acc[k];
        continue;
      }
      if (g.pp_on) {
        const size_t op = (size_t)j * g.nxa + i, s1 = (size_t)(AFC_P1 + 2 * (cls - 1)) * PS + op;
        double t1 = 1.0, t2 = 1.0;
        if (d.frz) {   // frozen branch: the recorded theta*, theta**
          t1 = d.frz[s1];
          t2 = d.frz[s1 + PS];
          if (!(t1 == 1.0 && t2 == 1.0)) {
            double UL[8], out[8];
            point_llf_state<GB>(d, g, cls, i, j, dt, UL);
            scaling_blend(acc, UL, t1, t2, out);
            nlim += 1;
            for (int k = 0; k < 8; ++k) acc[k] = out[k];
          }
        } else if (!clear_of_floor(acc, g)) {
          if (d.pq) {   // slow path in k_points_slow, over a dense list (the warp does not wait here)
            const int slot = enqueue(d.st, &d.st->npq, d.pq_cap);
            if (slot >= 0) {
              d.pq[slot] = (cls << 28) | (int)op;
#pragma unroll
              for (int k = 0; k < 8; ++k) d.pqu[(size_t)k * d.pq_cap + slot] = acc[k];
            }
            continue;
          }
          double out[8];
          int lim, shr, bad;
          point_pp<GB>(d, g, cls, i, j, acc, dt, out, lim, shr, bad, t1, t2);
          nlim += lim;
          nshr += shr;
          nbad += bad;
          for (int k = 0; k < 8; ++k) acc[k] = out[k];
        }
        if (d.rec) {
          d.rec[s1] = t1;
          d.rec[s1 + PS] = t2;
        }
      }
      if (is_zero(a)) {
#pragma unroll
        for (int k = 0; k < 8; ++k) uo[k * cs + oo] = acc[k];
      } else {
        const double *un = d.un[cls];
#pragma unroll
        for (int k = 0; k < 8; ++k) uo[k * cs + oo] = fma(a, __ldg(un + k * cs + oo), mul_i(b, acc[k]));
      }
    }
    if (mode != 1 && i < g.nx && j < g.ny && !is_zero(g.kappa)) {
      double phi[4];
      sensor_phi<GB>(d, g, i, j, phi);
      const size_t o = (size_t)j * g.nxa + i;
#pragma unroll
      for (int q = 0; q < 4; ++q) d.phi[q * PS + o] = phi[q];
    }
  }
  if (nlim) atomicAdd(&d.st->cnt[ST_POINT_LIMITED], (unsigned long long)nlim);
  if (nshr) atomicAdd(&d.st->cnt[ST_SHRINK], (unsigned long long)nshr);
  if (nbad) {
    atomicAdd(&d.st->cnt[ST_NONADMISSIBLE], (unsigned long long)nbad);
    atomicOr(&d.st->err, AFE_NONADMISSIBLE);
  }
}

// ---------------------------------------------------------------------------
// P3: faces
// ---------------------------------------------------------------------------
// phi of cell (ci, cj): stored for interior cells, recomputed for ghost cells
template <bool GB>
__device__ __forceinline__ void get_phi(const AfDev &d, const AfGrid &g, int ci, int cj, double *phi) {
  if (ci >= 0 && ci < g.nx && cj >= 0 && cj < g.ny) {
    const WV P = wview(d.phi, g);
#pragma unroll
    for (int q = 0; q < 4; ++q) phi[q] = P(ci, cj, q);
  } else if (g.bc == 0) {
    const WV P = wview(d.phi, g);
    const int a = wrapi(ci, g.nx), b2 = wrapi(cj, g.ny);
#pragma unroll
    for (int q = 0; q < 4; ++q) phi[q] = P(a, b2, q);
  } else {
    sensor_phi<GB>(d, g, ci, cj, phi);
  }
}

// theta^s = exp(-kappa [phi_1 phi_2 + phi_3]) with each phi maxed over the two cells
template <bool GB>
__device__ __forceinline__ double theta_s(const AfDev &d, const AfGrid &g, int dir, int ia, int ja, int ib, int jb) {
  if (is_zero(g.kappa)) return 1.0;
  double pa[4], pb[4];
  get_phi<GB>(d, g, ia, ja, pa);
  get_phi<GB>(d, g, ib, jb, pb);
  const double p1 = maxnn(pa[dir], pb[dir]), p2 = maxnn(pa[2], pb[2]), p3 = maxnn(pa[3], pb[3]);
  const double arg = mul_i(-g.kappa, fma(p1, p2, p3));
  return is_zero(arg) ? 1.0 : exp(arg);   // quiet data: exp(-0) = 1 without the call
}

// One face in direction L between cell averages ca, cb (mapped indices),
// Simpson nodes lo, mid, hi.  Writes F^LLF, G = theta^s (F - F^LLF), theta^s, alpha.
// GB: the cell indices are unmapped and resolved through reflective / inflow sides.
template <int L, bool GB>
__device__ __forceinline__ void face(const AfDev &d, const AfGrid &g, double *out, size_t PS, const PP &lo, const PP &mid,
                                     const PP &hi, int cai, int caj, int cbi, int cbj, double ts, bool llf, int &nsens) {
  const WV Aw = wview(d.pd[0], g);
  const SV Uw = sview(d.us[0], g, 0);
  PPG ga, gb;
  if constexpr (GB) {
    ga = prefg(d, g, 0, cai, caj);
    gb = prefg(d, g, 0, cbi, cbj);
  }
  auto A = [&](int a, int b, int q) -> double {
    if constexpr (GB) return pwg(a == cai && b == caj ? ga : gb, q);
    else return Aw(a, b, q);
  };
  auto Ub = [&](int a, int b, int k) -> double {
    if constexpr (GB) return pug(a == cai && b == caj ? ga : gb, k);
    else return Uw(a, b, k);
  };
  double al = 0.0;
  if (llf) {
    const int qv = L == 0 ? QA_V1 : QA_V2, qc = L == 0 ? QA_CF1 : QA_CF2;
    const double Ba[3] = {Ub(cai, caj, 4), Ub(cai, caj, 5), Ub(cai, caj, 6)};
    const double Bb[3] = {Ub(cbi, cbj, 4), Ub(cbi, cbj, 5), Ub(cbi, cbj, 6)};
    al = alpha_llf(A(cai, caj, qv), A(cbi, cbj, qv), A(cai, caj, qc), A(cbi, cbj, qc), A(cai, caj, QA_SRHO),
                   A(cbi, cbj, QA_SRHO), Ba, Bb);
  }
  const int f0 = L == 0 ? QP_F1 : QP_F2;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    double Fh = 0.0, Fl = 0.0;
    if (k != 4 + L) {
      const int s = f0 + fslot(L, k);
      Fh = mul_i(fma(4.0, pw(mid, PS, g.nxa, s), pw(lo, PS, g.nxa, s) + pw(hi, PS, g.nxa, s)), 1.0 / 6.0);
      if (llf) Fl = ldexp_i<-1>(fma(-al, Ub(cbi, cbj, k) - Ub(cai, caj, k), A(cai, caj, s) + A(cbi, cbj, s)));
    } else if (llf) {
      Fl = mul_i(ldexp_i<-1>(neg_i(al)), Ub(cbi, cbj, k) - Ub(cai, caj, k));
    }
    out[(QF_FLLF + k) * PS] = Fl;
    out[(QF_G + k) * PS] = is_one(ts) ? Fh - Fl : mul_i(ts, Fh - Fl);
  }
  out[QF_TS * PS] = ts;
  out[QF_AL * PS] = al;
  nsens += (long long)bits(ts) < (long long)bits(0.99);   // ts in [0, 1]
}

template <bool GB>
__device__ __forceinline__ void b_faces(const AfDev &d, const AfGrid &g, const int i, const int j, int mode) {
  const size_t PS = (size_t)g.nxa * g.nya;
  const size_t o = (size_t)j * g.nxa + i;
  const bool llf = mode == 0 && (g.pp_on || !is_zero(g.kappa));
  const bool sens = mode != 1;   // theta^s for stages (mode 0) and af_sensor (mode 2)
  int nsens = 0;
  if (i < g.nxa && j < g.nya) {
    // x-face (f = i, row j): cells i-1 | i; Simpson nodes: corners (i,j), (i,j+1), x-face (i,j)
    if (i < g.ex[1] && j < g.ey[1]) {
      const int jp = mface(j + 1, g.ny, g.bc);
      double ts;
      if (d.frz && mode == 0) ts = d.frz[AFC_TSX * PS + o];   // frozen branch
      else ts = sens ? theta_s<GB>(d, g, 0, i - 1, j, i, j) : 1.0;
      if (d.rec && mode == 0) d.rec[AFC_TSX * PS + o] = ts;
      if constexpr (GB)
        face<0, true>(d, g, d.fx + o, PS, pref(d, g, 3, i, j), pref(d, g, 1, i, j), pref(d, g, 3, i, jp), i - 1, j, i, j,
                      ts, llf, nsens);
      else
        face<0, false>(d, g, d.fx + o, PS, pref(d, g, 3, i, j), pref(d, g, 1, i, j), pref(d, g, 3, i, jp),
                       mcell(i - 1, g.nx, g.bc), j, mcell(i, g.nx, g.bc), j, ts, llf, nsens);
    }
    // y-face (i, g = j): cells j-1 | j; Simpson nodes: corners (i,j), (i+1,j), y-face (i,j)
    if (i < g.ex[2] && j < g.ey[2]) {
      const int ip = mface(i + 1, g.nx, g.bc);
      double ts;
      if (d.frz && mode == 0) ts = d.frz[AFC_TSY * PS + o];
      else ts = sens ? theta_s<GB>(d, g, 1, i, j - 1, i, j) : 1.0;
      if (d.rec && mode == 0) d.rec[AFC_TSY * PS + o] = ts;
      if constexpr (GB)
        face<1, true>(d, g, d.fy + o, PS, pref(d, g, 3, i, j), pref(d, g, 2, i, j), pref(d, g, 3, ip, j), i, j - 1, i, j,
                      ts, llf, nsens);
      else
        face<1, false>(d, g, d.fy + o, PS, pref(d, g, 3, i, j), pref(d, g, 2, i, j), pref(d, g, 3, ip, j), i,
                       mcell(j - 1, g.ny, g.bc), i, mcell(j, g.ny, g.bc), ts, llf, nsens);
    }
  }
  if (sens && !is_zero(g.kappa)) {
    const unsigned act = __activemask();
    const int tot = __reduce_add_sync(act, nsens);
    if (tot && (threadIdx.x & 31) == (__ffs(act) - 1)) atomicAdd(&d.st->cnt[ST_SENSOR_LT099], (unsigned long long)tot);
  }
}

// ---------------------------------------------------------------------------
// P4: cells -- source, sensor blend, flux limiter steps (1)-(2)
// ---------------------------------------------------------------------------
struct NewtonLog { int solves, maxit; };

// Newton on the vertex cubic q(r) = rho E - |m|^2/2 - rho|B|^2/2 - rho eps_p/(gamma-1)
// along V(r) = L1 + r D, from r = 1, with a sign bracket and the Newton step
// from the other bracket end as fallback, then bisection (Sec. 3.2 step (2)).
__device__ void cubic_eval(const double *L1, const double *D, double ce, double r, double &q, double &dq) {
  const double rho = fma(r, D[0], L1[0]);
  const double m0 = fma(r, D[1], L1[1]), m1 = fma(r, D[2], L1[2]), m2 = fma(r, D[3], L1[3]);
  const double b0 = fma(r, D[4], L1[4]), b1 = fma(r, D[5], L1[5]), b2 = fma(r, D[6], L1[6]);
  const double E = fma(r, D[7], L1[7]);
  const double mm = fma(m0, m0, fma(m1, m1, m2 * m2));
  const double bb = fma(b0, b0, fma(b1, b1, b2 * b2));
  q = fma(rho, E, -0.5 * mm) - rho * fma(0.5, bb, ce);
  const double mdm = fma(m0, D[1], fma(m1, D[2], m2 * D[3]));
  const double bdb = fma(b0, D[4], fma(b1, D[5], b2 * D[6]));
  dq = fma(D[0], E, rho * D[7]) - mdm - D[0] * fma(0.5, bb, ce) - rho * bdb;
}

__device__ double newton_root(const double *L1, const double *D, double eps_p, double gm1, NewtonLog &nl) {
  const double ce = eps_p / gm1;
  double lo = 0.0, hi = 1.0, r = 1.0, qlo, dqlo, qhi, dqhi, q, dq;
  cubic_eval(L1, D, ce, lo, qlo, dqlo);
  cubic_eval(L1, D, ce, hi, qhi, dqhi);
  q = qhi;
  dq = dqhi;
  bool at_hi = true;
  int it = 0;
  for (; it < 40; ++it) {
    double rn = r - q / dq;
    if (fabs(rn - r) <= 1e-14) { r = rn; ++it; break; }
    if (!(rn > lo && rn < hi)) {
      const double ro = at_hi ? lo - qlo / dqlo : hi - qhi / dqhi;
      rn = (ro > lo && ro < hi) ? ro : 0.5 * (lo + hi);
    }
    const double dr = rn - r;
    r = rn;
    cubic_eval(L1, D, ce, r, q, dq);
    at_hi = !(q >= 0.0);
    if (!at_hi) { lo = r; qlo = q; dqlo = dq; } else { hi = r; qhi = q; dqhi = dq; }
    if (fabs(dr) <= 1e-14 || hi - lo <= 1e-14) { ++it; break; }
  }
  nl.solves++;
  nl.maxit = max(nl.maxit, it);
  return r;
}

__device__ __noinline__ void flux_limiter_box(const double *L1, const double (*H)[8], double eps_rho, double eps_p,
                                              double gm1, double *Lam, NewtonLog &nl) {
  double negsum = 0.0;
  for (int J = 0; J < 4; ++J)
    if (H[J][0] < 0.0) negsum = negsum + H[J][0];
  double LamRho[4];
  for (int I = 0; I < 4; ++I) {
    LamRho[I] = 1.0;
    if (H[I][0] < 0.0) LamRho[I] = fmin(1.0, (L1[0] - eps_rho) / (1e-12 - negsum));
    Lam[I] = LamRho[I];
  }
  for (int kk = 0; kk < 16; ++kk) {
    double A[4], V[8], D[8];
    for (int I = 0; I < 4; ++I) A[I] = ((kk >> I) & 1) ? LamRho[I] : 0.0;
    for (int k = 0; k < 8; ++k) {
      double s = 0.0;
      for (int I = 0; I < 4; ++I) s = fma(A[I], H[I][k], s);
      D[k] = s;
      V[k] = L1[k] + s;
    }
    double r = 1.0;
    if (pressure(V, gm1) < eps_p) r = newton_root(L1, D, eps_p, gm1, nl);
    for (int I = 0; I < 4; ++I)
      if ((kk >> I) & 1) Lam[I] = fmin(Lam[I], r * A[I]);
  }
}

// Certificate that every vertex of the Sec. 3.2 box around L1 is in S_p with
// room to spare and needs no density scaling, so that the full procedure
// would return Lambda = 1 exactly: with V = L1 + d, |d_k| <= D_k = sum_I
// |H_I,k|, q(V) >= q(L1) - T, T bounding the linear, quadratic and cubic terms.
__device__ __forceinline__ bool box_certified(const double *L1, const double *D, const AfGrid &g) {
  const double rho = L1[0], E = L1[7];
  const double bb = fma(L1[4], L1[4], fma(L1[5], L1[5], mul_i(L1[6], L1[6])));
  const double mm = fma(L1[1], L1[1], fma(L1[2], L1[2], mul_i(L1[3], L1[3])));
  const double q0 = fma(rho, E, ldexp_i<-1>(neg_i(mm))) - rho * fma(0.5, bb, g.c13);
  const double bD = fma(absd(L1[4]), D[4], fma(absd(L1[5]), D[5], mul_i(absd(L1[6]), D[6])));
  const double mD = fma(absd(L1[1]), D[1], fma(absd(L1[2]), D[2], mul_i(absd(L1[3]), D[3])));
  const double DB2 = fma(D[4], D[4], fma(D[5], D[5], mul_i(D[6], D[6])));
  const double DM2 = fma(D[1], D[1], fma(D[2], D[2], mul_i(D[3], D[3])));
  const double hrho = ldexp_i<-1>(rho);
  const double T1 = fma(absd(E - fma(0.5, bb, g.c13)), D[0], fma(rho, D[7], fma(rho, bD, mD)));
  const double T2 = fma(D[0], D[7], fma(0.5, DM2, fma(hrho, DB2, mul_i(D[0], bD))));
  const double T3 = mul_i(ldexp_i<-1>(D[0]), DB2);
  const double T = T1 + T2 + T3;
  const double scale = fma(rho, absd(E), fma(0.5, mm, fma(hrho, bb, T)));
  // density rectangle: Lambda^rho = 1 when rho(L1) - 1e-13 >= 1e-12 + sum |rho(H)|
  return ge_i(q0 - T, mul_i(1e-12, scale)) && ge_i(rho - 1e-13, mul_i(1e-12 + D[0], 1.0 + 1e-10));
}

// |x| as a float, rounded up to 2^-60 when 0 < |x| < 2^-60 (an upper bound; 0 stays 0)
// and truncated toward zero above; ok false from 2^61 on
__device__ __forceinline__ float abs_f32_bound(double x, bool &ok) {
  const unsigned long long b = bits(x) & 0x7fffffffffffffffULL;
  const unsigned hi = (unsigned)(b >> 32), e = hi >> 20;
  ok = ok && e < 1084u;
  const float f = __uint_as_float(((hi - (896u << 20)) << 3) | ((unsigned)b >> 29));
  return b == 0 ? 0.0f : (e < 963u ? 0x1p-60f : f);
}
// FP32 certificate of the box: true when box_certified(L1, D) holds for the bounds
// D_k = cxf (|G0k| + |G1k|) + cyf (|G2k| + |G3k|), formed here in FP32 and rounded up
// (truncated inputs, three roundings: relative error < 2^-21, covered by the factor
// 1 + 2^-19), so that T, which grows with every D_k, is bounded above.  Components
// of m and B of L1 below 2^-60 are taken as 0 in |m|^2 and |B|^2 (an error below
// 2^-119 there, below 2^-77 rho c <= 2^-77 S in q0 and T, c > 0) and as 2^-60 in the
// terms linear in them (bD, mD: an upper bound).  Each computed term then errs by
// less than eps = 8 * 2^-23 of S, the sum of the magnitudes of every term of q0,
// T and scale, so q0_32 - T_32 > 2^-14 S_32 implies q0 - T > (2^-14 - 3 eps) S >
// 1e-12 scale, and the FP64 certificate (error about 1e-15 S) holds too.  The
// density condition rho - 1e-13 >= (1e-12 + D0)(1 + 1e-10) follows from rho_32 >=
// 1.0001 (1e-12 + D0_32 + 1e-13).  S_32 > 2^-100 keeps the absolute errors of
// products below the normal FP32 range negligible; an overflow makes S_32 infinite.
__device__ __forceinline__ bool box_cert32(const double *L1, const double (*Gf)[8], double cxf, double cyf,
                                           double c13) {
  bool ok = true;
  float L[8], La[8], D[8];   // L: for the squares (small m, B flushed); La: |L|, small ones as 2^-60
  L[0] = trunc_f32<false>(L1[0], ok);
  L[7] = trunc_f32<false>(L1[7], ok);
#pragma unroll
  for (int k = 1; k < 7; ++k) {
    L[k] = trunc_f32<true>(L1[k], ok);
    La[k] = abs_f32_bound(L1[k], ok);
  }
  const float cx = trunc_f32<false>(cxf, ok), cy = trunc_f32<false>(cyf, ok), c = trunc_f32<false>(c13, ok);
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const float gx = abs_f32_bound(Gf[0][k], ok) + abs_f32_bound(Gf[1][k], ok);
    const float gy = abs_f32_bound(Gf[2][k], ok) + abs_f32_bound(Gf[3][k], ok);
    D[k] = fmaf(cx, gx, cy * gy) * (1.0f + 0x1p-19f);
  }
  const float rho = L[0], E = L[7];
  const float bb = fmaf(L[4], L[4], fmaf(L[5], L[5], L[6] * L[6]));
  const float mm = fmaf(L[1], L[1], fmaf(L[2], L[2], L[3] * L[3]));
  const float eb = fmaf(0.5f, bb, c);
  const float q0 = fmaf(-rho, eb, fmaf(rho, E, -0.5f * mm));
  const float bD = fmaf(La[4], D[4], fmaf(La[5], D[5], La[6] * D[6]));
  const float mD = fmaf(La[1], D[1], fmaf(La[2], D[2], La[3] * D[3]));
  const float DB2 = fmaf(D[4], D[4], fmaf(D[5], D[5], D[6] * D[6]));
  const float DM2 = fmaf(D[1], D[1], fmaf(D[2], D[2], D[3] * D[3]));
  const float ar = fabsf(rho);
  const float T1 = fmaf(fabsf(E - eb), D[0], fmaf(ar, D[7], fmaf(ar, bD, mD)));
  const float T2 = fmaf(D[0], D[7], fmaf(0.5f, DM2, fmaf(0.5f * ar, DB2, D[0] * bD)));
  const float T3 = 0.5f * D[0] * DB2;
  const float T = T1 + T2 + T3;
  const float S = fmaf(ar, fabsf(E), fmaf(0.5f, mm, fmaf(ar, eb, fmaf(fabsf(E) + eb, D[0], T))));
  return ok && c > 0.0f && S > 0x1p-100f && q0 - T > 0x1p-14f * S && rho >= 1.0001f * (1e-12f + D[0] + 1e-13f);
}

// The FP64 bounds D and certificate for a cell that box_cert32 left undecided (not
// inlined: the rare case; Lim1 by value, the face values G reloaded)
__device__ __noinline__ bool box_cert64(const AfDev &d, const AfGrid &g, int i, int j, int ip, int jp, double l0,
                                        double l1, double l2, double l3, double l4, double l5, double l6, double l7,
                                        double cxf, double cyf) {
  const WV FX = wview(d.fx, g), FY = wview(d.fy, g);
  const double L1[8] = {l0, l1, l2, l3, l4, l5, l6, l7};
  double D[8];
#pragma unroll
  for (int k = 0; k < 8; ++k)
    D[k] = fma(cxf, absd(FX(i, j, QF_G + k)) + absd(FX(ip, j, QF_G + k)),
               mul_i(cyf, absd(FY(i, j, QF_G + k)) + absd(FY(i, jp, QF_G + k))));
  return box_certified(L1, D, g);
}

// Sec. 3.2 step (1) for one cell: theta_ij and Lim1, with the floors eps_rho, eps_p.
__device__ __forceinline__ void cell_source_limit(const double *Ullf, const double *dS, double dtts, const AfGrid &g,
                                                  double *L1, int &srclim, double &th_out, double &eps_rho,
                                                  double &eps_p) {
  double Usrc[8];
  for (int k = 0; k < 8; ++k) Usrc[k] = fma(-dtts, dS[k], Ullf[k]);
  eps_rho = fmin(1e-13, Ullf[0]);
  const double pllf = pressure(Ullf, g.gm1);
  eps_p = fmin(1e-13, pllf);
  double th = 1.0;
  const double psrc = pressure(Usrc, g.gm1);
  srclim = 0;
  if (psrc < eps_p) {
    th = fmin(1.0, ddiv(pllf - eps_p, pllf - psrc));
    srclim = 1;
  }
  for (int k = 0; k < 8; ++k) L1[k] = fma(th, Usrc[k] - Ullf[k], Ullf[k]);
  th_out = th;
}

// Full Sec. 3.2 steps (1)-(2) for one cell (slow path).
__device__ __noinline__ void cell_limiter_full(const double *Ullf, const double *dS, double dtts, const double (*H)[8],
                                               const AfGrid &g, double *L1, double *Lam, int &srclim, NewtonLog &nl,
                                               double &th_out) {
  double eps_rho, eps_p;
  cell_source_limit(Ullf, dS, dtts, g, L1, srclim, th_out, eps_rho, eps_p);
  flux_limiter_box(L1, H, eps_rho, eps_p, g.gm1, Lam, nl);
}

// The anti-diffusive fluxes H_L, H_R, H_D, H_U of cell (i, j) (Sec. 3.2 step 2)
// from the stored G = theta^s (F - F^LLF) of its faces.
__device__ __forceinline__ void cell_H(const AfDev &d, const AfGrid &g, int i, int j, double cxf, double cyf,
                                       double (*H)[8]) {
  const WV FX = wview(d.fx, g), FY = wview(d.fy, g);
  const int ip = mface(i + 1, g.nx, g.bc), jp = mface(j + 1, g.ny, g.bc);
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    H[0][k] = cxf * FX(i, j, QF_G + k);
    H[1][k] = -(cxf * FX(ip, j, QF_G + k));
    H[2][k] = cyf * FY(i, j, QF_G + k);
    H[3][k] = -(cyf * FY(i, jp, QF_G + k));
  }
}

template <bool GB>
__device__ __forceinline__ void b_cells(const AfDev &d, const AfGrid &g, const int i, const int j, double a, double b,
                                        int mode) {
  const size_t PS = (size_t)g.nxa * g.nya;
  const size_t o = (size_t)j * g.nxa + i;
  int nsrc = 0, nlam = 0, ncfl = 0;
  NewtonLog nl = {0, 0};
  if (i < g.nx && j < g.ny) {
    const double dt = mode == 1 ? 1.0 : d.sc->dt;
    const int ip = mface(i + 1, g.nx, g.bc), jp = mface(j + 1, g.ny, g.bc);
    const SV X = sview(d.us[1], g, 1), Y = sview(d.us[2], g, 2), C = sview(d.us[3], g, 3);
    const WV PX = wview(d.pd[1], g), PY = wview(d.pd[2], g), PC = wview(d.pd[3], g), PZ = wview(d.pd[4], g);
    const WV ZU = wview(d.uc, g);
    // ---- eq. (semi_av_src): 3x3 Simpson nodes (l along x, m along y; 1 = centre)
    double S[8];
    {
      double b1[3][3], b2[3][3];
      b1[0][0] = C(i, j, 4); b1[1][0] = Y(i, j, 4); b1[2][0] = C(ip, j, 4);
      b1[0][1] = X(i, j, 4); b1[1][1] = ZU(i, j, 4); b1[2][1] = X(ip, j, 4);
      b1[0][2] = C(i, jp, 4); b1[1][2] = Y(i, jp, 4); b1[2][2] = C(ip, jp, 4);
      b2[0][0] = C(i, j, 5); b2[1][0] = Y(i, j, 5); b2[2][0] = C(ip, j, 5);
      b2[0][1] = X(i, j, 5); b2[1][1] = ZU(i, j, 5); b2[2][1] = X(ip, j, 5);
      b2[0][2] = C(i, jp, 5); b2[1][2] = Y(i, jp, 5); b2[2][2] = C(ip, jp, 5);
      const double rdx = g.rdx, rdy = g.rdy;
      const double w[3] = {1.0 / 6.0, 2.0 / 3.0, 1.0 / 6.0};
      double wd[3][3];
#pragma unroll
      for (int l = 0; l < 3; ++l)
#pragma unroll
        for (int m = 0; m < 3; ++m) {
          double dx1, dy2;
          // D^-, D, D^+ of B1 along row m and of B2 along column l (Sec. 2.1), the
          // one-sided ones as 3 (b1 - b0) - (b2 - b1): exactly 0 on constant data
          if (l == 0) dx1 = fma(3.0, b1[1][m] - b1[0][m], -(b1[2][m] - b1[1][m]));
          else if (l == 1) dx1 = b1[2][m] - b1[0][m];
          else dx1 = fma(3.0, b1[2][m] - b1[1][m], -(b1[1][m] - b1[0][m]));
          if (m == 0) dy2 = fma(3.0, b2[l][1] - b2[l][0], -(b2[l][2] - b2[l][1]));
          else if (m == 1) dy2 = b2[l][2] - b2[l][0];
          else dy2 = fma(3.0, b2[l][2] - b2[l][1], -(b2[l][1] - b2[l][0]));
          wd[l][m] = mul_i(w[l] * w[m], fma(dx1, rdx, mul_i(dy2, rdy)));
        }
      // Psi at the nodes: B from the DoFs, v and v.B from the point data
      // node (l,m): corners (l,m even), x-faces (l even, m = 1), y-faces (l = 1, m even), centre (1,1)
      S[0] = 0.0;
      const int ni[3] = {i, i, ip}, nj[3] = {j, j, jp};
      // quiet data: every node divergence exactly 0 gives S = +0 exactly (each
      // fma(+-0, Psi, +0) of the sum is +0), without the Psi loads
      unsigned long long nz = 0;
#pragma unroll
      for (int l = 0; l < 3; ++l)
#pragma unroll
        for (int m = 0; m < 3; ++m) nz |= bits(wd[l][m]) << 1;
      if (nz == 0) {
#pragma unroll
        for (int k = 1; k < 8; ++k) S[k] = 0.0;
      } else {
#pragma unroll
        for (int k = 1; k < 8; ++k) {
          double s = 0.0;
#pragma unroll
          for (int l = 0; l < 3; ++l)
#pragma unroll
            for (int m = 0; m < 3; ++m) {
              double psi;
              if (k == 1) psi = b1[l][m];
              else if (k == 2) psi = b2[l][m];
              else {
                const int q = k == 3 ? -1 : QP_V1 + (k - 4);
                if (l == 1 && m == 1) psi = q < 0 ? ZU(i, j, 6) : PZ(i, j, q);
                else if (l == 1) psi = q < 0 ? Y(i, nj[m], 6) : PY(i, nj[m], q);
                else if (m == 1) psi = q < 0 ? X(ni[l], j, 6) : PX(ni[l], j, q);
                else psi = q < 0 ? C(ni[l], nj[m], 6) : PC(ni[l], nj[m], q);
              }
              s = fma(wd[l][m], psi, s);
            }
          S[k] = s;
        }
      }
      if (!g.src_cell_on)
        for (int k = 0; k < 8; ++k) S[k] = 0.0;
    }
    const SV Ub = sview(d.us[0], g, 0);
    const WV A = wview(d.pd[0], g);
    const WV FX = wview(d.fx, g), FY = wview(d.fy, g);
    const double cxf = mul_i(dt, g.rdx), cyf = mul_i(dt, g.rdy);
    double *uo = d.uo[0];
    const size_t cs0 = (size_t)g.nx * g.ny, o0 = (size_t)j * g.nx + i;
    if (mode == 1) {
      // semi-discrete rhs: -(F_R - F_L)/dx - (F_U - F_D)/dy - S (G holds the Simpson flux here)
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const double fl = FX(i, j, QF_G + k), fr = FX(ip, j, QF_G + k);
        const double fd = FY(i, j, QF_G + k), fu = FY(i, jp, QF_G + k);
        uo[k * cs0 + o0] = -(fr - fl) * g.rdx - (fu - fd) * g.rdy - S[k];
      }
    } else {
      // S^LLF = (central div Bbar) Psi(Ubar)
      double be, bw, bn, bs;
      if constexpr (GB) {
        be = pug(prefg(d, g, 0, i + 1, j), 4);
        bw = pug(prefg(d, g, 0, i - 1, j), 4);
        bn = pug(prefg(d, g, 0, i, j + 1), 5);
        bs = pug(prefg(d, g, 0, i, j - 1), 5);
      } else {
        const int ie = mcell(i + 1, g.nx, g.bc), iw = mcell(i - 1, g.nx, g.bc);
        const int jn = mcell(j + 1, g.ny, g.bc), js = mcell(j - 1, g.ny, g.bc);
        be = Ub(ie, j, 4);
        bw = Ub(iw, j, 4);
        bn = Ub(i, jn, 5);
        bs = Ub(i, js, 5);
      }
      const double divBb = fma(be - bw, 0.5 * g.rdx, mul_i(bn - bs, 0.5 * g.rdy));
      double Ubar[8];
      load8(Ub, i, j, Ubar);
      const double vb1 = A(i, j, QA_V1), vb2 = A(i, j, QA_V2), vb3 = A(i, j, QA_V3);
      double SL[8];
      SL[0] = 0.0;
      SL[1] = mul_i(divBb, Ubar[4]);
      SL[2] = mul_i(divBb, Ubar[5]);
      SL[3] = mul_i(divBb, Ubar[6]);
      SL[4] = mul_i(divBb, vb1);
      SL[5] = mul_i(divBb, vb2);
      SL[6] = mul_i(divBb, vb3);
      SL[7] = mul_i(divBb, fma(vb1, Ubar[4], fma(vb2, Ubar[5], mul_i(vb3, Ubar[6]))));
      if (!g.src_cell_on)
        for (int k = 0; k < 8; ++k) SL[k] = 0.0;
      // theta^s_ij = min over the four faces
      const double tsL = FX(i, j, QF_TS), tsR = FX(ip, j, QF_TS), tsD = FY(i, j, QF_TS), tsU = FY(i, jp, QF_TS);
      const double tsc = minnn(minnn(tsL, tsR), minnn(tsD, tsU));
      if (!g.pp_on) {
        // sensor-blended high-order update: F^ss = F^LLF + G, S^ss = S^LLF + theta^s (S - S^LLF)
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const double fl = FX(i, j, QF_FLLF + k) + FX(i, j, QF_G + k), fr = FX(ip, j, QF_FLLF + k) + FX(ip, j, QF_G + k);
          const double fd = FY(i, j, QF_FLLF + k) + FY(i, j, QF_G + k), fu = FY(i, jp, QF_FLLF + k) + FY(i, jp, QF_G + k);
          const double sss = fma(tsc, S[k] - SL[k], SL[k]);
          const double fe = Ubar[k] - cxf * (fr - fl) - cyf * (fu - fd) - dt * sss;
          uo[k * cs0 + o0] = a == 0.0 ? fe : fma(a, __ldg(d.un[0] + k * cs0 + o0), b * fe);
        }
      } else {
        // eq. (2d_llf): U^LLF; U^src - U^LLF = -dt theta^s_ij (S - S^LLF)
        double Ullf[8], dS[8], Gf[4][8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const double fl = FX(i, j, QF_FLLF + k), fr = FX(ip, j, QF_FLLF + k);
          const double fd = FY(i, j, QF_FLLF + k), fu = FY(i, jp, QF_FLLF + k);
          Ullf[k] = fma(-dt, SL[k], fma(-cyf, fu - fd, fma(-cxf, fr - fl, Ubar[k])));
          dS[k] = S[k] - SL[k];
          Gf[0][k] = FX(i, j, QF_G + k);
          Gf[1][k] = FX(ip, j, QF_G + k);
          Gf[2][k] = FY(i, j, QF_G + k);
          Gf[3][k] = FY(i, jp, QF_G + k);
        }
        // Lemma 3.1 CFL condition (diagnostic count only)
        {
          const double lhs = mul_i(dt, (FX(i, j, QF_AL) + FX(ip, j, QF_AL)) * g.rdx + (FY(i, j, QF_AL) + FY(i, jp, QF_AL)) * g.rdy +
                                   ddiv(absd(divBb), A(i, j, QA_SRHO)));
          ncfl += gt_pos(lhs, 1.0 + 1e-12);
        }
        const double dtts = mul_i(dt, tsc);
        double L1[8], Lam[4];
        double th_src = 1.0;
        if (d.frz) {   // frozen branch: Lim1 with the recorded theta_ij; face theta are recorded too
          th_src = d.frz[AFC_TSRC * PS + o];
#pragma unroll
          for (int k = 0; k < 8; ++k) L1[k] = fma(th_src, fma(-dtts, dS[k], Ullf[k]) - Ullf[k], Ullf[k]);
          Lam[0] = Lam[1] = Lam[2] = Lam[3] = 1.0;
          nsrc += th_src < 1.0;
        }
        bool fast = !d.frz && clear_of_floor(Ullf, g);
        if (fast) {
#pragma unroll
          for (int k = 0; k < 8; ++k) L1[k] = fma(-dtts, dS[k], Ullf[k]);
          fast = clear_of_floor(L1, g);
        }
        if (fast)
          fast = box_cert32(L1, Gf, cxf, cyf, g.c13) ||
                 box_cert64(d, g, i, j, ip, jp, L1[0], L1[1], L1[2], L1[3], L1[4], L1[5], L1[6], L1[7], cxf, cyf);
        bool listed = false;
        if (d.frz) {
        } else if (fast) {
          Lam[0] = Lam[1] = Lam[2] = Lam[3] = 1.0;
        } else if (d.cq) {   // step (1) here, the box of step (2) in k_cells_slow over a dense list
          int sl = 0;
          double eps_rho, eps_p;
          cell_source_limit(Ullf, dS, dtts, g, L1, sl, th_src, eps_rho, eps_p);
          nsrc += sl;
          const int slot = enqueue(d.st, &d.st->ncq, d.cq_cap);
          if (slot >= 0) {
            d.cq[slot] = (int)o;
            d.cqe[2 * slot] = eps_rho;
            d.cqe[2 * slot + 1] = eps_p;
          }
          listed = true;
        } else {
          double H[4][8];
#pragma unroll
          for (int k = 0; k < 8; ++k) {
            H[0][k] = cxf * Gf[0][k];
            H[1][k] = -(cxf * Gf[1][k]);
            H[2][k] = cyf * Gf[2][k];
            H[3][k] = -(cyf * Gf[3][k]);
          }
          int sl = 0;
          cell_limiter_full(Ullf, dS, dtts, H, g, L1, Lam, sl, nl, th_src);
          nsrc += sl;
          nlam += (Lam[0] < 1.0 || Lam[1] < 1.0 || Lam[2] < 1.0 || Lam[3] < 1.0);
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) d.lim1[k * PS + o] = L1[k];
        if (!listed)
#pragma unroll
          for (int I = 0; I < 4; ++I) d.lam[I * PS + o] = Lam[I];
        if (d.rec) d.rec[AFC_TSRC * PS + o] = th_src;
      }
    }
  }
  if (nsrc) atomicAdd(&d.st->cnt[ST_SRC_LIMITED], (unsigned long long)nsrc);
  if (nlam) atomicAdd(&d.st->cnt[ST_LAMBDA_LT1], (unsigned long long)nlam);
  if (ncfl) atomicAdd(&d.st->cnt[ST_CFL_VIOLATIONS], (unsigned long long)ncfl);
  if (nl.solves) {
    atomicAdd(&d.st->cnt[ST_NEWTON_SOLVES], (unsigned long long)nl.solves);
    atomicMax(&d.st->cnt[ST_NEWTON_MAXIT], (unsigned long long)nl.maxit);
  }
}

// ---------------------------------------------------------------------------
// P5: unique face coefficients, limited update, round-off check
// ---------------------------------------------------------------------------
// Reading (outflow): a boundary face takes the Lambda of its one interior cell.
__device__ __forceinline__ double theta_x(const AfGrid &g, const WV &L, int f, int j) {
  if (g.bc == 1) {
    if (f == 0) return L(0, j, 0);
    if (f == g.nx) return L(g.nx - 1, j, 1);
    return minnn(L(f - 1, j, 1), L(f, j, 0));
  }
  return minnn(L(wrapi(f - 1, g.nx), j, 1), L(wrapi(f, g.nx), j, 0));
}
__device__ __forceinline__ double theta_y(const AfGrid &g, const WV &L, int i, int gg) {
  if (g.bc == 1) {
    if (gg == 0) return L(i, 0, 2);
    if (gg == g.ny) return L(i, g.ny - 1, 3);
    return minnn(L(i, gg - 1, 3), L(i, gg, 2));
  }
  return minnn(L(i, wrapi(gg - 1, g.ny), 3), L(i, wrapi(gg, g.ny), 2));
}

__device__ __forceinline__ void limited_value(const AfDev &d, const AfGrid &g, int i, int j, const double *th, double dt,
                                              double *out) {
  const WV FX = wview(d.fx, g), FY = wview(d.fy, g), L1 = wview(d.lim1, g);
  const int ip = mface(i + 1, g.nx, g.bc), jp = mface(j + 1, g.ny, g.bc);
  const double cxf = mul_i(dt, g.rdx), cyf = mul_i(dt, g.rdy);
  const bool ones = is_one(th[0]) && is_one(th[1]) && is_one(th[2]) && is_one(th[3]);
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const double gl = FX(i, j, QF_G + k), gr = FX(ip, j, QF_G + k), gd = FY(i, j, QF_G + k), gu = FY(i, jp, QF_G + k);
    double tx, ty;
    if (ones) {
      tx = sub_i(gl, gr);
      ty = sub_i(gd, gu);
    } else {
      tx = fma(-th[1], gr, th[0] * gl);
      ty = fma(-th[3], gu, th[2] * gd);
    }
    out[k] = fma(cyf, ty, fma(cxf, tx, L1(i, j, k)));
  }
}

__device__ __forceinline__ void b_final(const AfDev &d, const AfGrid &g, const int i, const int j, double a, double b) {
  int nface = 0, nlam = 0;
  if (i < g.nx && j < g.ny) {
    const double dt = d.sc->dt;
    const WV L = wview(d.lam, g);
    const size_t o = (size_t)j * g.nxa + i;
    // with the work lists the box of Sec. 3.2 ran in its own passes: count its cells
    // with some Lambda_I < 1 here (Lambda >= 0: bit-pattern compares on the integer pipe)
    if (d.cq && !d.frz)
      nlam = lt_one(L(i, j, 0)) || lt_one(L(i, j, 1)) || lt_one(L(i, j, 2)) || lt_one(L(i, j, 3));
    double th[4];
    if (d.frz) {   // frozen branch: the recorded face coefficients (after Remark 4.1)
      const size_t PS = (size_t)g.nxa * g.nya;
      const int ip = (g.bc == 0) ? wrapi(i + 1, g.nx) : i + 1, jp = (g.bc == 0) ? wrapi(j + 1, g.ny) : j + 1;
      th[0] = d.frz[AFC_THX * PS + o];
      th[1] = d.frz[AFC_THX * PS + (size_t)j * g.nxa + ip];
      th[2] = d.frz[AFC_THY * PS + o];
      th[3] = d.frz[AFC_THY * PS + (size_t)jp * g.nxa + i];
    } else {
      th[0] = theta_x(g, L, i, j);
      th[1] = theta_x(g, L, i + 1, j);
      th[2] = theta_y(g, L, i, j);
      th[3] = theta_y(g, L, i, j + 1);
    }
    d.thx[o] = th[0];
    d.thy[o] = th[2];
    nface += lt_one(th[0]) + lt_one(th[2]);
    if (g.bc == 1 && i == g.nx - 1) {
      d.thx[o + 1] = th[1];
      nface += lt_one(th[1]);
    }
    if (g.bc == 1 && j == g.ny - 1) {
      d.thy[o + g.nxa] = th[3];
      nface += lt_one(th[3]);
    }
    double fe[8];
    limited_value(d, g, i, j, th, dt, fe);
    // rho > 0 and p > 0 and all finite, on the integer pipe: for finite doubles
    // x > 0 exactly when the bit pattern, read as a signed integer, is > 0
    bool ok = (long long)bits(fe[0]) > 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) ok = ok && finite_bits(fe[k]);
    ok = ok && (qform_cert32(fe, 0.0) || qform_gt0(fe[0], fe[1], fe[2], fe[3], fe[4], fe[5], fe[6], fe[7]));
    if (!ok && !d.frz) {
      const int slot = atomicAdd(&d.st->nrepair, 1);
      if (slot < AF_MAX_REPAIR) d.st->repair[slot] = j * g.nx + i;
      else atomicOr(&d.st->err, AFE_REPAIR_OVERFLOW);
    }
    const size_t cs0 = (size_t)g.nx * g.ny, o0 = (size_t)j * g.nx + i;
    if (is_zero(a)) {
#pragma unroll
      for (int k = 0; k < 8; ++k) d.uo[0][k * cs0 + o0] = fe[k];
    } else {
#pragma unroll
      for (int k = 0; k < 8; ++k) d.uo[0][k * cs0 + o0] = fma(a, __ldg(d.un[0] + k * cs0 + o0), mul_i(b, fe[k]));
    }
  }
  if (nface) atomicAdd(&d.st->cnt[ST_FACE_THETA_LT1], (unsigned long long)nface);
  if (nlam) atomicAdd(&d.st->cnt[ST_LAMBDA_LT1], (unsigned long long)nlam);
}

// Remark 4.1 round-off shrink for the flagged cells, one thread, in cell order.
// Reading: the four face coefficients of a non-admissible cell are lowered to
// max(0, theta - 2^m 1e-8), m = 0..9, else to 0; the cells sharing a lowered
// face are recomputed (and repaired in turn if they come later in the order).
__device__ void fe_of(const AfDev &d, const AfGrid &g, int i, int j, double dt, double *fe) {
  const size_t o = (size_t)j * g.nxa + i;
  const int ip = (g.bc == 0) ? wrapi(i + 1, g.nx) : i + 1;
  const int jp = (g.bc == 0) ? wrapi(j + 1, g.ny) : j + 1;
  double th[4];
  th[0] = d.thx[o];
  th[1] = d.thx[(size_t)j * g.nxa + ip];
  th[2] = d.thy[o];
  th[3] = d.thy[(size_t)jp * g.nxa + i];
  limited_value(d, g, i, j, th, dt, fe);
}

__device__ void b_repair(const AfDev &d, const AfGrid &g, double a, double b) {
  int n = d.st->nrepair;
  if (n <= 0) return;
  if (n > AF_MAX_REPAIR) n = AF_MAX_REPAIR;
  int *list = d.st->repair;
  for (int p = 1; p < n; ++p) {   // insertion sort (the list is tiny)
    int v = list[p], q = p - 1;
    while (q >= 0 && list[q] > v) { list[q + 1] = list[q]; --q; }
    list[q + 1] = v;
  }
  const double dt = d.sc->dt;
  const size_t cs0 = (size_t)g.nx * g.ny;
  unsigned long long nshr = 0, nbad = 0;
  for (int p = 0; p < n; ++p) {
    const int cell = list[p], i = cell % g.nx, j = cell / g.nx;
    double fe[8];
    fe_of(d, g, i, j, dt, fe);
    if (in_G(fe, g.gm1)) continue;
    nshr++;
    const size_t o = (size_t)j * g.nxa + i;
    const int ip = (g.bc == 0) ? wrapi(i + 1, g.nx) : i + 1;
    const int jp = (g.bc == 0) ? wrapi(j + 1, g.ny) : j + 1;
    double *t[4] = {&d.thx[o], &d.thx[(size_t)j * g.nxa + ip], &d.thy[o], &d.thy[(size_t)jp * g.nxa + i]};
    const double th0[4] = {*t[0], *t[1], *t[2], *t[3]};
    bool ok = false;
    for (int m = 0; m <= 10 && !ok; ++m) {
      for (int I = 0; I < 4; ++I) *t[I] = (m < 10) ? fmax(0.0, th0[I] - ldexp(1e-8, m)) : 0.0;
      fe_of(d, g, i, j, dt, fe);
      ok = in_G(fe, g.gm1) || m == 10;
    }
    if (!in_G(fe, g.gm1)) nbad++;
    for (int k = 0; k < 8; ++k) {
      const size_t oo = k * cs0 + (size_t)j * g.nx + i;
      d.uo[0][oo] = a == 0.0 ? fe[k] : fma(a, d.un[0][oo], b * fe[k]);
    }
    // neighbours sharing a lowered face
    const int nbi[4] = {i - 1, i + 1, i, i}, nbj[4] = {j, j, j - 1, j + 1};
    for (int q = 0; q < 4; ++q) {
      int ii = nbi[q], jj = nbj[q];
      if (g.bc == 1 && (ii < 0 || ii >= g.nx || jj < 0 || jj >= g.ny)) continue;
      ii = wrapi(ii, g.nx);
      jj = wrapi(jj, g.ny);
      double f2[8];
      fe_of(d, g, ii, jj, dt, f2);
      for (int k = 0; k < 8; ++k) {
        const size_t oo = k * cs0 + (size_t)jj * g.nx + ii;
        d.uo[0][oo] = a == 0.0 ? f2[k] : fma(a, d.un[0][oo], b * f2[k]);
      }
      const int id = jj * g.nx + ii;
      if (id > cell && !in_G(f2, g.gm1) && n < AF_MAX_REPAIR) {   // repair it later in the order
        bool listed = false;
        for (int r = p + 1; r < n; ++r) listed |= (list[r] == id);
        if (!listed) {
          int q2 = n++;
          while (q2 > p + 1 && list[q2 - 1] > id) { list[q2] = list[q2 - 1]; --q2; }
          list[q2] = id;
        }
      }
    }
  }
  // atomics: the point list pass may update the same counters concurrently
  if (nshr) {
    atomicAdd(&d.st->cnt[ST_SHRINK], nshr);
    atomicAdd(&d.st->cnt[ST_CELL_SHRINK], nshr);
  }
  if (nbad) {
    atomicAdd(&d.st->cnt[ST_NONADMISSIBLE], nbad);
    atomicOr(&d.st->err, AFE_NONADMISSIBLE);
  }
  d.st->nrepair = 0;
}


// ---------------------------------------------------------------------------
// Kernels: one run (grid over its index points) and a batch of runs (a
// persistent grid walking a (run, tile) work list; tiles are blockDim-sized).
// ---------------------------------------------------------------------------
#define AF_IJ blockIdx.x * blockDim.x + threadIdx.x, blockIdx.y * blockDim.y + threadIdx.y

// On grids with reflective or inflow sides, a thread block whose whole tile
// lies at least kFrame indices inside [0, nx) x [0, ny) touches no ghost (the
// stencils of the point, face and cell passes reach 2 indices), so it runs the
// plain code; only the blocks of the boundary frame resolve ghosts.
constexpr int kFrame = 4;
__device__ __forceinline__ bool interior_block(int nx, int ny) {
  const int i0 = blockIdx.x * blockDim.x, j0 = blockIdx.y * blockDim.y;
  return i0 >= kFrame && j0 >= kFrame && i0 + (int)blockDim.x + kFrame <= nx && j0 + (int)blockDim.y + kFrame <= ny;
}
// ---- limiter slow paths over the work lists (single runs) -------------------
// Points whose high-order update left the floors: Sec. 3.3 LLF state, scaling
// limiter and Remark 4.1 shrink, then the RK combination.
template <bool GB>
__device__ __forceinline__ void b_points_slow(const AfDev &d, const AfGrid &g, double a, double b) {
  const int n = min(*(volatile int *)&d.st->npq, d.pq_cap);
  const double dt = d.sc->dt;
  const size_t PS = (size_t)g.nxa * g.nya;
  int nlim = 0, nshr = 0, nbad = 0;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
    const int packed = d.pq[t], cls = packed >> 28, op = packed & ((1 << 28) - 1);
    const int i = op % g.nxa, j = op / g.nxa;
    double UH[8], out[8], t1, t2;
#pragma unroll
    for (int k = 0; k < 8; ++k) UH[k] = d.pqu[(size_t)k * d.pq_cap + t];
    int lim, shr, bad;
    point_pp<GB>(d, g, cls, i, j, UH, dt, out, lim, shr, bad, t1, t2);
    nlim += lim;
    nshr += shr;
    nbad += bad;
    if (d.rec) {
      const size_t s1 = (size_t)(AFC_P1 + 2 * (cls - 1)) * PS + op;
      d.rec[s1] = t1;
      d.rec[s1 + PS] = t2;
    }
    double *uo = d.uo[cls];
    const size_t cs = (size_t)g.ex[cls] * g.ey[cls], oo = (size_t)j * g.ex[cls] + i;
    if (a == 0.0) {
#pragma unroll
      for (int k = 0; k < 8; ++k) uo[k * cs + oo] = out[k];
    } else {
      const double *un = d.un[cls];
#pragma unroll
      for (int k = 0; k < 8; ++k) uo[k * cs + oo] = fma(a, __ldg(un + k * cs + oo), b * out[k]);
    }
  }
  if (nlim) atomicAdd(&d.st->cnt[ST_POINT_LIMITED], (unsigned long long)nlim);
  if (nshr) atomicAdd(&d.st->cnt[ST_SHRINK], (unsigned long long)nshr);
  if (nbad) {
    atomicAdd(&d.st->cnt[ST_NONADMISSIBLE], (unsigned long long)nbad);
    atomicOr(&d.st->err, AFE_NONADMISSIBLE);
  }
}

// Cells whose box was not certified: Sec. 3.2 step (2) in two dense passes.
// A (one thread per listed cell): the rectangle R_rho; Lambda starts at Lambda^rho;
// the vertices A^k that leave S_p go to the vertex list.  B (one thread per listed
// vertex): the Newton solve for r, then Lambda_I = min(Lambda_I, r A_I) for the I
// with k_I = 1, by an atomic minimum on the bit patterns (Lambda >= 0, for which the
// integer order is the numeric order): exact and order-free, so Lambda equals the
// one-thread box of Sec. 3.2 bit for bit.  The count of cells with Lambda < 1 is
// taken by the final pass.  (For long lists a half-warp per cell, one lane per vertex,
// was measured slower than one thread per cell: every lane repeats the loads and the
// rectangle; short lists take it, for its latency.)
__device__ __forceinline__ void rect_rho(const double *L1, const double (*H)[8], double eps_rho, double *LamRho) {
  double negsum = 0.0;
  for (int J = 0; J < 4; ++J)
    if (H[J][0] < 0.0) negsum = negsum + H[J][0];
  for (int I = 0; I < 4; ++I) {
    LamRho[I] = 1.0;
    if (H[I][0] < 0.0) LamRho[I] = fmin(1.0, (L1[0] - eps_rho) / (1e-12 - negsum));
  }
}
// vertex k of R_rho: A (components Lambda^rho_I for k_I = 1, else 0) and D = sum_I A_I H_I
__device__ __forceinline__ void box_vertex(int kk, const double *LamRho, const double (*H)[8], double *A, double *D) {
  for (int I = 0; I < 4; ++I) A[I] = ((kk >> I) & 1) ? LamRho[I] : 0.0;
  for (int k = 0; k < 8; ++k) {
    double sum = 0.0;
    for (int I = 0; I < 4; ++I) sum = fma(A[I], H[I][k], sum);
    D[k] = sum;
  }
}

// A short list (at most one cell per half-warp of the grid, as on quiet data): a half-warp
// per cell, lane v the vertex A^v with its own Newton solve, the minima by shuffles;
// the whole box is done here (latency: one vertex instead of sixteen in a row).
__device__ __forceinline__ void cells_box_short(const AfDev &d, const AfGrid &g, int n) {
  const double dt = d.sc->dt, cxf = dt * g.rdx, cyf = dt * g.rdy;
  const size_t PS = (size_t)g.nxa * g.nya;
  const int lane = threadIdx.x & 31, v = lane & 15;
  const int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 4;   // one cell per half-warp
  const int tw = (blockIdx.x * blockDim.x + (threadIdx.x & ~31)) >> 4;
  if (tw >= n) return;   // the whole warp is past the list
  const bool live = t < n;
  const int tt = live ? t : tw;
  const int o = d.cq[tt], i = o % g.nxa, j = o / g.nxa;
  double L1[8], H[4][8], LamRho[4], A[4], D[8], V[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) L1[k] = d.lim1[k * PS + o];
  cell_H(d, g, i, j, cxf, cyf, H);
  rect_rho(L1, H, d.cqe[2 * tt], LamRho);
  box_vertex(v, LamRho, H, A, D);
  for (int k = 0; k < 8; ++k) V[k] = L1[k] + D[k];
  NewtonLog nl = {0, 0};
  double r = 1.0;
  if (live && pressure(V, g.gm1) < d.cqe[2 * tt + 1]) r = newton_root(L1, D, d.cqe[2 * tt + 1], g.gm1, nl);
#pragma unroll
  for (int I = 0; I < 4; ++I) {
    double m = ((v >> I) & 1) ? r * A[I] : INFINITY;
#pragma unroll
    for (int off = 1; off < 16; off <<= 1) m = fmin(m, __shfl_xor_sync(0xffffffffu, m, off));
    if (live && v == 0) d.lam[I * PS + o] = fmin(LamRho[I], m);
  }
  if (nl.solves) {
    atomicAdd(&d.st->cnt[ST_NEWTON_SOLVES], (unsigned long long)nl.solves);
    atomicMax(&d.st->cnt[ST_NEWTON_MAXIT], (unsigned long long)nl.maxit);
  }
}

__device__ __forceinline__ void b_cells_box(const AfDev &d, const AfGrid &g) {
  const int n = min(*(volatile int *)&d.st->ncq, d.cq_cap);
  if (n <= (int)((gridDim.x * blockDim.x) >> 4)) {
    cells_box_short(d, g, n);
    return;
  }
  const double dt = d.sc->dt, cxf = dt * g.rdx, cyf = dt * g.rdy;
  const size_t PS = (size_t)g.nxa * g.nya;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
    const int o = d.cq[t], i = o % g.nxa, j = o / g.nxa;
    double L1[8], H[4][8], LamRho[4];
#pragma unroll
    for (int k = 0; k < 8; ++k) L1[k] = d.lim1[k * PS + o];
    cell_H(d, g, i, j, cxf, cyf, H);
    rect_rho(L1, H, d.cqe[2 * t], LamRho);
    const double eps_p = d.cqe[2 * t + 1];
    for (int I = 0; I < 4; ++I) {
      d.cql[4 * (size_t)t + I] = LamRho[I];
      d.lam[I * PS + o] = LamRho[I];
    }
    for (int kk = 0; kk < 16; ++kk) {
      double A[4], D[8], V[8];
      box_vertex(kk, LamRho, H, A, D);
      for (int k = 0; k < 8; ++k) V[k] = L1[k] + D[k];
      if (pressure(V, g.gm1) < eps_p) {
        const int slot = enqueue(d.st, &d.st->nvq, d.vq_cap);
        if (slot >= 0) d.vq[slot] = ((unsigned)t << 4) | (unsigned)kk;
      }
    }
  }
}

__device__ __forceinline__ void b_cells_newton(const AfDev &d, const AfGrid &g) {
  const int n = min(*(volatile int *)&d.st->nvq, d.vq_cap);
  const double dt = d.sc->dt, cxf = dt * g.rdx, cyf = dt * g.rdy;
  const size_t PS = (size_t)g.nxa * g.nya;
  NewtonLog nl = {0, 0};
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    const unsigned packed = d.vq[e];
    const int t = (int)(packed >> 4), kk = (int)(packed & 15u);
    const int o = d.cq[t], i = o % g.nxa, j = o / g.nxa;
    double L1[8], H[4][8], LamRho[4], A[4], D[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) L1[k] = d.lim1[k * PS + o];
    cell_H(d, g, i, j, cxf, cyf, H);
    for (int I = 0; I < 4; ++I) LamRho[I] = d.cql[4 * (size_t)t + I];
    box_vertex(kk, LamRho, H, A, D);
    const double r = newton_root(L1, D, d.cqe[2 * t + 1], g.gm1, nl);
    for (int I = 0; I < 4; ++I)
      if ((kk >> I) & 1)
        atomicMin(reinterpret_cast<unsigned long long *>(d.lam + I * PS + o),
                  (unsigned long long)__double_as_longlong(r * A[I]));
  }
  if (nl.solves) {
    atomicAdd(&d.st->cnt[ST_NEWTON_SOLVES], (unsigned long long)nl.solves);
    atomicMax(&d.st->cnt[ST_NEWTON_MAXIT], (unsigned long long)nl.maxit);
  }
}

#define AF_BATCH_LOOP(call)                                       \
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {       \
    const int4 w = items[it];                                     \
    const AfRun *__restrict__ r = runs + w.x;                     \
    const int i = w.y + threadIdx.x, j = w.z + threadIdx.y;       \
    call;                                                         \
  }

// Launch bounds of the stage kernels (128 threads): a kernel given AF_MINB_x
// resident blocks per SM is capped at 65536 / (128 x blocks) registers; without
// it ptxas picks the count.  The kernels keep the FP64 pipe and the integer
// pipes busy at once; the defaults are the fastest of a sweep on the 2048x2048
// blast (point data at 5 blocks = 96 registers, point pass at 8 = 64, cell pass
// at 5 = 96; faces and final pass at the compiler's count).
#define AF_LB(minb) __launch_bounds__(128, minb)
#ifndef AF_MINB_PD
#define AF_MINB_PD 5
#endif
#define AF_LB_PD AF_LB(AF_MINB_PD)
#ifndef AF_MINB_PT
#define AF_MINB_PT 8
#endif
#define AF_LB_PT AF_LB(AF_MINB_PT)
#ifdef AF_MINB_FC
#define AF_LB_FC AF_LB(AF_MINB_FC)
#else
#define AF_LB_FC __launch_bounds__(128)
#endif
#ifndef AF_MINB_CL
#define AF_MINB_CL 5
#endif
#define AF_LB_CL AF_LB(AF_MINB_CL)
#ifdef AF_MINB_FN
#define AF_LB_FN AF_LB(AF_MINB_FN)
#else
#define AF_LB_FN __launch_bounds__(128)
#endif
__global__ void AF_LB_PD k_pointdata(const __grid_constant__ AfDev d, const __grid_constant__ AfGrid g,
                                                   int reduce_dt) {
  // a stage's first pass: the work lists of its point and cell passes start empty
  if (d.pq && blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0 && threadIdx.y == 0) {
    d.st->npq = 0;
    d.st->ncq = 0;
    d.st->nvq = 0;
  }
  b_pointdata(d, g, AF_IJ, reduce_dt);
}
__global__ void __launch_bounds__(256) kb_pointdata(const AfRun *__restrict__ runs, const int4 *__restrict__ items,
                                                    int nitems, int reduce_dt) {
  AF_BATCH_LOOP(b_pointdata(r->d, r->g, i, j, reduce_dt));
}
__global__ void k_dt(const __grid_constant__ AfDev d, const __grid_constant__ AfGrid g) {
  if (threadIdx.x == 0 && blockIdx.x == 0) b_dt(d, g);
}
__global__ void kb_dt(const AfRun *__restrict__ runs, int nruns) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < nruns) b_dt(runs[t].d, runs[t].g);
}
// At most 128 registers (4 blocks per SM): the limiter slow path spills a
// little, the common path runs at twice the occupancy (measured 8 % faster).
// UP: the velocity-upwind point source (Example 4.2 variant) is compiled in
// only where it is asked for; the central scheme pays nothing for it.
template <bool GB, bool UP>
__global__ void AF_LB_PT k_points(const __grid_constant__ AfDev d, const __grid_constant__ AfGrid g,
                                                double a, double b, int mode) {
  if (GB && interior_block(g.nx, g.ny)) b_points<false, UP>(d, g, AF_IJ, a, b, mode);
  else b_points<GB, UP>(d, g, AF_IJ, a, b, mode);
}
template <bool UP>
__global__ void __launch_bounds__(256, 2) kb_points(const AfRun *__restrict__ runs, const int4 *__restrict__ items,
                                                 int nitems, double a, double b) {
  AF_BATCH_LOOP((b_points<false, UP>(r->d, r->g, i, j, a, b, 0)));
}
template <bool GB>
__global__ void AF_LB_FC k_faces(const __grid_constant__ AfDev d, const __grid_constant__ AfGrid g,
                                               int mode) {
  if (GB && interior_block(g.nx, g.ny)) b_faces<false>(d, g, AF_IJ, mode);
  else b_faces<GB>(d, g, AF_IJ, mode);
}
__global__ void __launch_bounds__(256) kb_faces(const AfRun *__restrict__ runs, const int4 *__restrict__ items,
                                                int nitems) {
  AF_BATCH_LOOP(b_faces<false>(r->d, r->g, i, j, 0));
}
template <bool GB>
__global__ void AF_LB_CL k_cells(const __grid_constant__ AfDev d, const __grid_constant__ AfGrid g,
                                               double a, double b, int mode) {
  if (GB && interior_block(g.nx, g.ny)) b_cells<false>(d, g, AF_IJ, a, b, mode);
  else b_cells<GB>(d, g, AF_IJ, a, b, mode);
}
__global__ void __launch_bounds__(256, 2) kb_cells(const AfRun *__restrict__ runs, const int4 *__restrict__ items,
                                                int nitems, double a, double b) {
  AF_BATCH_LOOP(b_cells<false>(r->d, r->g, i, j, a, b, 0));
}
__global__ void AF_LB_FN k_final(const __grid_constant__ AfDev d, const __grid_constant__ AfGrid g,
                                               double a, double b) {
  b_final(d, g, AF_IJ, a, b);
}
__global__ void __launch_bounds__(256) kb_final(const AfRun *__restrict__ runs, const int4 *__restrict__ items,
                                                int nitems, double a, double b) {
  AF_BATCH_LOOP(if (r->g.pp_on) b_final(r->d, r->g, i, j, a, b));
}
template <bool GB>
__global__ void __launch_bounds__(128) k_points_slow(const __grid_constant__ AfDev d, const __grid_constant__ AfGrid g,
                                                     double a, double b) {
  b_points_slow<GB>(d, g, a, b);
}
__global__ void __launch_bounds__(128) k_cells_box(const __grid_constant__ AfDev d, const __grid_constant__ AfGrid g) {
  b_cells_box(d, g);
}
__global__ void __launch_bounds__(128) k_cells_newton(const __grid_constant__ AfDev d, const __grid_constant__ AfGrid g) {
  b_cells_newton(d, g);
}

__global__ void k_repair(const __grid_constant__ AfDev d, const __grid_constant__ AfGrid g, double a, double b) {
  if (threadIdx.x == 0 && blockIdx.x == 0) b_repair(d, g, a, b);
}
__global__ void kb_repair(const AfRun *__restrict__ runs, int nruns, double a, double b) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < nruns && runs[t].g.pp_on) b_repair(runs[t].d, runs[t].g, a, b);
}

// ---------------------------------------------------------------------------
// math self-check: out = rcp(x) (op 0), ddiv(x, y) (op 1), dsqrt(x) (op 2)
// ---------------------------------------------------------------------------
// point data of the inflow state: out = [U (8)][as a point (AF_NQP)][as an average (AF_NQA)]
__global__ void k_inflow_pd(const __grid_constant__ AfGrid g, const double *U, double *out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double u[8], s1, s2;
  for (int k = 0; k < 8; ++k) out[k] = u[k] = U[k];
  point_data(u, g, out + 8, 1, false, s1, s2);
  point_data(u, g, out + 8 + AF_NQP, 1, true, s1, s2);
}
__global__ void k_math_check(int op, const double *x, const double *y, double *out, long long n) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  if (op == 0) out[t] = rcp(x[t]);
  else if (op == 1) out[t] = ddiv(x[t], y[t]);
  else if (op == 2) out[t] = dsqrt(x[t]);
  else if (op == 3) out[t] = add_i(x[t], y[t]);
  else if (op == 4) out[t] = mul_i(x[t], y[t]);
  else if (op == 5) out[t] = ge_i(x[t], y[t]) ? 1.0 : 0.0;
  else if (op == 6) out[t] = ge_pos(x[t], y[t]) ? 1.0 : 0.0;
  else if (op == 7) out[t] = gt_pos(x[t], y[t]) ? 1.0 : 0.0;
  else if (op == 8) out[t] = ge_zero(x[t]) ? 1.0 : 0.0;
  else if (op == 9) out[t] = qform_cert32(x + 8 * t, y[0]) ? 1.0 : 0.0;   // x: n states of 8
  else {                                                                  // x: n cases of 8 + 4 x 8
    double Gf[4][8];
    for (int q = 0; q < 4; ++q)
      for (int k = 0; k < 8; ++k) Gf[q][k] = x[40 * t + 8 + 8 * q + k];
    out[t] = box_cert32(x + 40 * t, Gf, y[0], y[1], y[2]) ? 1.0 : 0.0;
  }
}

// FP64 FMA throughput probe: 8 independent register chains per thread.
__global__ void k_fp64_probe(double *out, int iters) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  double a0 = 1.0 + t * 1e-9, a1 = a0 + 0.1, a2 = a0 + 0.2, a3 = a0 + 0.3;
  double a4 = a0 + 0.4, a5 = a0 + 0.5, a6 = a0 + 0.6, a7 = a0 + 0.7;
  const double m = 0.999999, c = 1e-7;
  for (int k = 0; k < iters; ++k) {
    a0 = fma(a0, m, c); a1 = fma(a1, m, c); a2 = fma(a2, m, c); a3 = fma(a3, m, c);
    a4 = fma(a4, m, c); a5 = fma(a5, m, c); a6 = fma(a6, m, c); a7 = fma(a7, m, c);
  }
  out[t] = a0 + a1 + a2 + a3 + a4 + a5 + a6 + a7;
}

// ---------------------------------------------------------------------------
// Example 4.4: the discrete divergence measures of the state bound in d.us.
// Per cell: s1 = sum_{l,m} |(div B)^{l,m}| w_l w_m dx dy over the 3x3 nodes of
// eq. (semi_av_src) (centre node: the limited centre value, as in a stage) and
// s2 = |dy/6 ([R] - [L]) + dx/6 ([T] - [B])|, the Simpson edge integral of B.n
// ([.] = corner + 4 face centre + corner).  Each block reduces its cells in a
// fixed order and writes one partial pair; a one-block pass sums the partials
// in a fixed order, so the result does not depend on scheduling.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(128) k_divb(const __grid_constant__ AfDev d, const __grid_constant__ AfGrid g,
                                              double *partials) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
  double s1 = 0.0, s2 = 0.0;
  if (i < g.nx && j < g.ny) {
    const SV Ub = sview(d.us[0], g, 0), X = sview(d.us[1], g, 1), Y = sview(d.us[2], g, 2), C = sview(d.us[3], g, 3);
    const int ip = mface(i + 1, g.nx, g.bc), jp = mface(j + 1, g.ny, g.bc);
    double A[8], uc[8];
    load8(Ub, i, j, A);
    centre_value(d, g, i, j, A, uc);
    double b1[3][3], b2[3][3];   // [l][m]: l along x, m along y
    b1[0][0] = C(i, j, 4); b1[1][0] = Y(i, j, 4); b1[2][0] = C(ip, j, 4);
    b1[0][1] = X(i, j, 4); b1[1][1] = uc[4];      b1[2][1] = X(ip, j, 4);
    b1[0][2] = C(i, jp, 4); b1[1][2] = Y(i, jp, 4); b1[2][2] = C(ip, jp, 4);
    b2[0][0] = C(i, j, 5); b2[1][0] = Y(i, j, 5); b2[2][0] = C(ip, j, 5);
    b2[0][1] = X(i, j, 5); b2[1][1] = uc[5];      b2[2][1] = X(ip, j, 5);
    b2[0][2] = C(i, jp, 5); b2[1][2] = Y(i, jp, 5); b2[2][2] = C(ip, jp, 5);
    const double w[3] = {1.0 / 6.0, 2.0 / 3.0, 1.0 / 6.0};
#pragma unroll
    for (int l = 0; l < 3; ++l)
#pragma unroll
      for (int m = 0; m < 3; ++m) {
        double dx1, dy2;
        if (l == 0) dx1 = fma(4.0, b1[1][m], -3.0 * b1[0][m]) - b1[2][m];
        else if (l == 1) dx1 = b1[2][m] - b1[0][m];
        else dx1 = fma(3.0, b1[2][m], fma(-4.0, b1[1][m], b1[0][m]));
        if (m == 0) dy2 = fma(4.0, b2[l][1], -3.0 * b2[l][0]) - b2[l][2];
        else if (m == 1) dy2 = b2[l][2] - b2[l][0];
        else dy2 = fma(3.0, b2[l][2], fma(-4.0, b2[l][1], b2[l][0]));
        s1 = fma(w[l] * w[m], absd(fma(dx1, g.rdx, dy2 * g.rdy)), s1);
      }
    s1 *= g.dx * g.dy;
    const double right = fma(4.0, b1[2][1], b1[2][0] + b1[2][2]), left = fma(4.0, b1[0][1], b1[0][0] + b1[0][2]);
    const double top = fma(4.0, b2[1][2], b2[0][2] + b2[2][2]), bottom = fma(4.0, b2[1][0], b2[0][0] + b2[2][0]);
    s2 = absd(fma(g.dy, right - left, g.dx * (top - bottom))) * (1.0 / 6.0);
  }
  __shared__ double sh[2][128];
  const int t = threadIdx.y * blockDim.x + threadIdx.x;
  sh[0][t] = s1;
  sh[1][t] = s2;
  __syncthreads();
  for (int h = 64; h > 0; h >>= 1) {
    if (t < h) {
      sh[0][t] += sh[0][t + h];
      sh[1][t] += sh[1][t + h];
    }
    __syncthreads();
  }
  if (t == 0) {
    const size_t b = (size_t)blockIdx.y * gridDim.x + blockIdx.x;
    partials[2 * b] = sh[0][0];
    partials[2 * b + 1] = sh[1][0];
  }
}

// Run diagnostics: per block, the minimum density and pressure of each DoF
// class and the sum of the cell-average densities (AF_NDIAG partials).
__device__ __forceinline__ double nan_min(double a, double b) { return (a != a || a < b) ? a : b; }
__global__ void __launch_bounds__(128) k_diag(const __grid_constant__ AfDev d, const __grid_constant__ AfGrid g,
                                              double *partials) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
  const double inf = __longlong_as_double(0x7ff0000000000000LL);
  double v[AF_NDIAG];
  for (int q = 0; q < 8; ++q) v[q] = inf;
  v[8] = 0.0;
#pragma unroll 1
  for (int c = 0; c < 4; ++c) {
    if (i < g.ex[c] && j < g.ey[c]) {
      double U[8];
      load8(sview(d.us[c], g, c), i, j, U);
      v[c] = U[0];
      v[4 + c] = pressure(U, g.gm1);
      if (c == 0) v[8] = U[0];
    }
  }
  __shared__ double sh[AF_NDIAG][128];
  const int t = threadIdx.y * blockDim.x + threadIdx.x;
  for (int q = 0; q < AF_NDIAG; ++q) sh[q][t] = v[q];
  __syncthreads();
  for (int h = 64; h > 0; h >>= 1) {
    if (t < h) {
      for (int q = 0; q < 8; ++q) sh[q][t] = nan_min(sh[q][t], sh[q][t + h]);
      sh[8][t] += sh[8][t + h];
    }
    __syncthreads();
  }
  if (t == 0) {
    const size_t b = (size_t)blockIdx.y * gridDim.x + blockIdx.x;
    for (int q = 0; q < AF_NDIAG; ++q) partials[AF_NDIAG * b + q] = sh[q][0];
  }
}

__global__ void __launch_bounds__(256) k_diag_sum(const double *partials, int nblocks, double cell_area, double *out) {
  __shared__ double sh[AF_NDIAG][256];
  const int t = threadIdx.x;
  const double inf = __longlong_as_double(0x7ff0000000000000LL);
  double v[AF_NDIAG];
  for (int q = 0; q < 8; ++q) v[q] = inf;
  v[8] = 0.0;
  for (int k = t; k < nblocks; k += 256) {
    for (int q = 0; q < 8; ++q) v[q] = nan_min(v[q], partials[AF_NDIAG * k + q]);
    v[8] += partials[AF_NDIAG * k + 8];
  }
  for (int q = 0; q < AF_NDIAG; ++q) sh[q][t] = v[q];
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if (t < h) {
      for (int q = 0; q < 8; ++q) sh[q][t] = nan_min(sh[q][t], sh[q][t + h]);
      sh[8][t] += sh[8][t + h];
    }
    __syncthreads();
  }
  if (t == 0) {
    for (int q = 0; q < 8; ++q) out[q] = sh[q][0];
    out[8] = sh[8][0] * cell_area;
  }
}

__global__ void __launch_bounds__(256) k_divb_sum(const double *partials, int nblocks, double *out) {
  __shared__ double sh[2][256];
  const int t = threadIdx.x;
  double a = 0.0, b = 0.0;
  for (int k = t; k < nblocks; k += 256) {
    a += partials[2 * k];
    b += partials[2 * k + 1];
  }
  sh[0][t] = a;
  sh[1][t] = b;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if (t < h) {
      sh[0][t] += sh[0][t + h];
      sh[1][t] += sh[1][t + h];
    }
    __syncthreads();
  }
  if (t == 0) {
    out[0] = sh[0][0];
    out[1] = sh[1][0];
  }
}

inline dim3 grid2(int nx, int ny) { return dim3((nx + 31) / 32, (ny + 3) / 4); }

}  // namespace

void af_launch_pointdata(const AfDev &d, const AfGrid &g, int reduce_dt, cudaStream_t s) {
  k_pointdata<<<grid2(g.nxa, g.nya), dim3(32, 4), 0, s>>>(d, g, reduce_dt);
}
void af_launch_dt(const AfDev &d, const AfGrid &g, cudaStream_t s) { k_dt<<<1, 32, 0, s>>>(d, g); }
int af_divb_nblocks(const AfGrid &g) { const dim3 b = grid2(g.nx, g.ny); return (int)(b.x * b.y); }
int af_diag_nblocks(const AfGrid &g) { const dim3 b = grid2(g.nxa, g.nya); return (int)(b.x * b.y); }
void af_launch_diag(const AfDev &d, const AfGrid &g, double *partials, double *out, cudaStream_t s) {
  const dim3 b = grid2(g.nxa, g.nya);
  k_diag<<<b, dim3(32, 4), 0, s>>>(d, g, partials);
  k_diag_sum<<<1, 256, 0, s>>>(partials, (int)(b.x * b.y), g.dx * g.dy, out);
}
void af_launch_divb(const AfDev &d, const AfGrid &g, double *partials, double *out, cudaStream_t s) {
  const dim3 b = grid2(g.nx, g.ny);
  k_divb<<<b, dim3(32, 4), 0, s>>>(d, g, partials);
  k_divb_sum<<<1, 256, 0, s>>>(partials, (int)(b.x * b.y), out);
}
void af_launch_points(const AfDev &d, const AfGrid &g, double a, double b, int mode, cudaStream_t s) {
  const dim3 gr = grid2(g.nxa, g.nya), bl(32, 4);
  if (g.special) {
    if (g.upwind) k_points<true, true><<<gr, bl, 0, s>>>(d, g, a, b, mode);
    else k_points<true, false><<<gr, bl, 0, s>>>(d, g, a, b, mode);
  } else {
    if (g.upwind) k_points<false, true><<<gr, bl, 0, s>>>(d, g, a, b, mode);
    else k_points<false, false><<<gr, bl, 0, s>>>(d, g, a, b, mode);
  }
}
void af_launch_faces(const AfDev &d, const AfGrid &g, int mode, cudaStream_t s) {
  if (g.special) k_faces<true><<<grid2(g.nxa, g.nya), dim3(32, 4), 0, s>>>(d, g, mode);
  else k_faces<false><<<grid2(g.nxa, g.nya), dim3(32, 4), 0, s>>>(d, g, mode);
}
void af_launch_cells(const AfDev &d, const AfGrid &g, double a, double b, int mode, cudaStream_t s) {
  if (g.special) k_cells<true><<<grid2(g.nx, g.ny), dim3(32, 4), 0, s>>>(d, g, a, b, mode);
  else k_cells<false><<<grid2(g.nx, g.ny), dim3(32, 4), 0, s>>>(d, g, a, b, mode);
}
void af_launch_final(const AfDev &d, const AfGrid &g, double a, double b, cudaStream_t s) {
  k_final<<<grid2(g.nx, g.ny), dim3(32, 4), 0, s>>>(d, g, a, b);
}
// a fixed grid of 4 blocks per SM walks the list
void af_launch_points_slow(const AfDev &d, const AfGrid &g, double a, double b, cudaStream_t s) {
  if (!d.pq) return;
  if (g.special) k_points_slow<true><<<152 * 4, 128, 0, s>>>(d, g, a, b);
  else k_points_slow<false><<<152 * 4, 128, 0, s>>>(d, g, a, b);
}
void af_launch_cells_slow(const AfDev &d, const AfGrid &g, cudaStream_t s) {
  if (!d.cq) return;
  k_cells_box<<<152 * 4, 128, 0, s>>>(d, g);
  k_cells_newton<<<152 * 4, 128, 0, s>>>(d, g);
}
void af_launch_repair(const AfDev &d, const AfGrid &g, double a, double b, cudaStream_t s) {
  k_repair<<<1, 32, 0, s>>>(d, g, a, b);
}
float af_run_fp64_probe(cudaStream_t s, double *flops) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int blocks = sms * 8, threads = 256, iters = 8192;
  double *buf = nullptr;
  if (cudaMallocAsync(&buf, sizeof(double) * blocks * threads, s) != cudaSuccess) return -1.f;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  k_fp64_probe<<<blocks, threads, 0, s>>>(buf, 64);   // warm-up
  cudaEventRecord(e0, s);
  k_fp64_probe<<<blocks, threads, 0, s>>>(buf, iters);
  cudaEventRecord(e1, s);
  cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaFreeAsync(buf, s);
  cudaStreamSynchronize(s);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *flops = 2.0 * 8.0 * (double)iters * blocks * threads / (ms * 1e-3);
  return ms;
}

void af_launch_inflow_pd(const AfGrid &g, const double *U, double *out, cudaStream_t s) {
  k_inflow_pd<<<1, 32, 0, s>>>(g, U, out);
}

void af_launch_math_check(int op, const double *x, const double *y, double *out, long long n, cudaStream_t s) {
  if (n <= 0) return;
  k_math_check<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(op, x, y, out, n);
}

void af_launch_batch(int pass, const AfRun *runs, int nruns, const int4 *items, int nitems, dim3 block, int nblocks,
                     double a, double b, int flag, cudaStream_t s) {
  const int reduce_dt = flag;
  switch (pass) {
    case AF_K_POINTDATA: kb_pointdata<<<nblocks, block, 0, s>>>(runs, items, nitems, reduce_dt); break;
    case AF_K_DT: kb_dt<<<(nruns + 127) / 128, 128, 0, s>>>(runs, nruns); break;
    case AF_K_POINTS:
      if (flag) kb_points<true><<<nblocks, block, 0, s>>>(runs, items, nitems, a, b);
      else kb_points<false><<<nblocks, block, 0, s>>>(runs, items, nitems, a, b);
      break;
    case AF_K_FACES: kb_faces<<<nblocks, block, 0, s>>>(runs, items, nitems); break;
    case AF_K_CELLS: kb_cells<<<nblocks, block, 0, s>>>(runs, items, nitems, a, b); break;
    case AF_K_FINAL: kb_final<<<nblocks, block, 0, s>>>(runs, items, nitems, a, b); break;
    case AF_K_REPAIR: kb_repair<<<(nruns + 127) / 128, 128, 0, s>>>(runs, nruns, a, b); break;
    default: break;
  }
}

int af_batch_occupancy(int pass, dim3 block) {
  int n = 0;
  const int threads = block.x * block.y;
  switch (pass) {
    case AF_K_POINTDATA: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kb_pointdata, threads, 0); break;
    case AF_K_POINTS: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kb_points<false>, threads, 0); break;
    case AF_K_FACES: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kb_faces, threads, 0); break;
    case AF_K_CELLS: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kb_cells, threads, 0); break;
    case AF_K_FINAL: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kb_final, threads, 0); break;
    default: n = 1;
  }
  return n > 0 ? n : 1;
}

#include "af_kernels1d.cuh"
