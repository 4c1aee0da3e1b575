// af_kernels1d.cuh -- the 1D AF scheme (Sec. 4: the 1D tests use the 1D AF
// scheme with the LLF FVS and without the Godunov-Powell source), included at
// the end of af_kernels.cu so that it shares the 2D device functions.
//
// The 1D problem runs on the 2D data structures with ny = 1: class 0 holds the
// cell averages (nx), class 1 the interface point values (nxa = nx, or nx + 1
// for outflow; point f is the left face of cell f), pd[4] and uc the cell
// centre values.  With one row the y-neighbours of every index map onto the
// index itself, so the shared pieces reduce to their x parts:
//   - the point update is the x-face line of Sec. 2.3 (point f-1, centre f-1,
//     point f, centre f, point f+1) without the y terms and the source;
//   - the sensor of Sec. 3.4 sees zero y-differences;
//   - the dt pass forms cfl / (max varrho_1 / dx) (the y maximum stays 0).
// Specific to 1D: the centre value of the cell parabola (6 Ubar - U_L - U_R)/4
// (Simpson), the face flux F1 of the face point value (no quadrature across
// the face), the LLF point state between neighbouring points, and the flux
// limiter of Sec. 3.2 with the two faces L, R (the 2D box with the two
// y-directions zero; no source, so U^{Lim,1} = U^LLF).
#pragma once

namespace {

// P1 (1D): point data of the points, the averages and the centre values; dt maximum
__device__ __forceinline__ void b1_pointdata(const AfDev &d, const AfGrid &g, int i, int reduce_dt) {
  const size_t PS = (size_t)g.nxa;
  double m1 = 0.0, s1, s2;
  bool clim = false;
  if (i < g.ex[1]) {
    double U[8];
    load8(sview(d.us[1], g, 1), i, 0, U);
    point_data(U, g, d.pd[1] + i, PS, false, s1, s2);
    m1 = maxnn(m1, s1);
  }
  if (i < g.nx) {
    double A[8], uc[8];
    load8(sview(d.us[0], g, 0), i, 0, A);
    point_data(A, g, d.pd[0] + i, PS, true, s1, s2);
    m1 = maxnn(m1, s1);
    const SV P = sview(d.us[1], g, 1);
    const int ip = mface(i + 1, g.nx, g.bc);
#pragma unroll
    for (int k = 0; k < 8; ++k) uc[k] = (6.0 * A[k] - P(i, 0, k) - P(ip, 0, k)) * 0.25;
    if (!clear_of_floor(uc, g)) {   // Remark 3.2
      double out[8], t1, t2;
      scaling_limiter(uc, A, g.gm1, out, t1, t2);
      clim = t1 < 1.0 || t2 < 1.0;
      for (int k = 0; k < 8; ++k) uc[k] = out[k];
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) d.uc[k * PS + i] = uc[k];
    point_data(uc, g, d.pd[4] + i, PS, false, s1, s2);
  }
  count(d.st, ST_CENTER_LIMITED, clim);
  if (reduce_dt) {
    unsigned long long b1 = (unsigned long long)__double_as_longlong(m1);
    for (int off = 16; off > 0; off >>= 1) {
      const unsigned long long o1 = __shfl_down_sync(0xffffffffu, b1, off);
      b1 = o1 > b1 ? o1 : b1;
    }
    if ((threadIdx.x & 31) == 0) atomicMax(&d.sc->smax[0], b1);
  }
}

// Sec. 3.3 slow path for point f: LLF state from the fluxes between f and its
// neighbouring points, scaling limiter, Remark 4.1 shrink.
__device__ __noinline__ void point_pp1(const AfDev &d, const AfGrid &g, int f, const double *UH, double dt,
                                       double *out, int &limited, int &shrunk, int &bad) {
  const int fm = mface(f - 1, g.nx, g.bc), fp = mface(f + 1, g.nx, g.bc);
  const SV P = sview(d.us[1], g, 1);
  double U[8];
  Full me, nb;
  load8(P, f, 0, U);
  full_data(U, g, me);
  double Fl[8], Fr[8];
  load8(P, fm, 0, U);
  full_data(U, g, nb);
  llf_flux_full(0, nb, me, Fl);
  load8(P, fp, 0, U);
  full_data(U, g, nb);
  llf_flux_full(0, me, nb, Fr);
  const double cxf = dt * g.rdx;
  double UL[8];
  for (int k = 0; k < 8; ++k) UL[k] = me.U[k] - cxf * (Fr[k] - Fl[k]);
  double t1, t2;
  scaling_limiter(UH, UL, g.gm1, out, t1, t2);
  limited = (t1 < 1.0 || t2 < 1.0);
  shrunk = 0;
  bad = 0;
  if (!in_G(out, g.gm1)) {
    shrunk = 1;
    double Us[8];
    for (int k = 0; k < 8; ++k) Us[k] = UH[k];
    Us[0] = fma(t1, UH[0], (1.0 - t1) * UL[0]);
    bool ok = false;
    for (int m = 0; m < 10 && !ok; ++m) {
      const double th = fmax(0.0, t2 - ldexp(1e-8, m));
      for (int k = 0; k < 8; ++k) out[k] = fma(th, Us[k], (1.0 - th) * UL[k]);
      ok = in_G(out, g.gm1);
    }
    if (!ok)
      for (int k = 0; k < 8; ++k) out[k] = UL[k];
    bad = !in_G(out, g.gm1);
  }
}

// P2 (1D): point update, its limiter and the RK combination; the sensor phi
__device__ __forceinline__ void b1_points(const AfDev &d, const AfGrid &g, int f, double a, double b) {
  const size_t PS = (size_t)g.nxa;
  const double dt = d.sc->dt;
  int nlim = 0, nshr = 0, nbad = 0;
  if (f < g.ex[1]) {
    const int fm = mface(f - 1, g.nx, g.bc), fp = mface(f + 1, g.nx, g.bc);
    const int c0 = mcell(f - 1, g.nx, g.bc), c1 = mcell(f, g.nx, g.bc);
    const PP me = pref(d, g, 1, f, 0);
    double acc[8], dB;
#pragma unroll
    for (int k = 0; k < 8; ++k) acc[k] = pu(me, k);
    const PP L[5] = {pref(d, g, 1, fm, 0), pref(d, g, 4, c0, 0), me, pref(d, g, 4, c1, 0), pref(d, g, 1, fp, 0)};
    fvs_line<0>(L, PS, g.nxa, 0.5 * dt * g.rdx, acc, dB, 0);
    if (g.pp_on && !clear_of_floor(acc, g)) {
      double out[8];
      int lim, shr, bad;
      point_pp1(d, g, f, acc, dt, out, lim, shr, bad);
      nlim += lim;
      nshr += shr;
      nbad += bad;
      for (int k = 0; k < 8; ++k) acc[k] = out[k];
    }
    const size_t cs = (size_t)g.ex[1];
    if (a == 0.0) {
#pragma unroll
      for (int k = 0; k < 8; ++k) d.uo[1][k * cs + f] = acc[k];
    } else {
#pragma unroll
      for (int k = 0; k < 8; ++k) d.uo[1][k * cs + f] = fma(a, __ldg(d.un[1] + k * cs + f), b * acc[k]);
    }
  }
  if (f < g.nx && g.kappa != 0.0) {
    double phi[4];
    sensor_phi<false>(d, g, f, 0, phi);
#pragma unroll
    for (int q = 0; q < 4; ++q) d.phi[q * PS + f] = phi[q];
  }
  if (nlim) atomicAdd(&d.st->cnt[ST_POINT_LIMITED], (unsigned long long)nlim);
  if (nshr) atomicAdd(&d.st->cnt[ST_SHRINK], (unsigned long long)nshr);
  if (nbad) {
    atomicAdd(&d.st->cnt[ST_NONADMISSIBLE], (unsigned long long)nbad);
    atomicOr(&d.st->err, AFE_NONADMISSIBLE);
  }
}

// P3 (1D): per face f, F^LLF between the adjacent averages, G = theta^s (F1(U_f) - F^LLF),
// theta^s and alpha^LLF (slots of the 2D face layout)
__device__ __forceinline__ void b1_faces(const AfDev &d, const AfGrid &g, int f) {
  const size_t PS = (size_t)g.nxa;
  int nsens = 0;
  if (f < g.ex[1]) {
    const int ca = mcell(f - 1, g.nx, g.bc), cb = mcell(f, g.nx, g.bc);
    const WV A = wview(d.pd[0], g), PW = wview(d.pd[1], g);
    const SV Ub = sview(d.us[0], g, 0);
    const double Ba[3] = {Ub(ca, 0, 4), Ub(ca, 0, 5), Ub(ca, 0, 6)};
    const double Bb[3] = {Ub(cb, 0, 4), Ub(cb, 0, 5), Ub(cb, 0, 6)};
    const double al = alpha_llf(A(ca, 0, QA_V1), A(cb, 0, QA_V1), A(ca, 0, QA_CF1), A(cb, 0, QA_CF1),
                                A(ca, 0, QA_SRHO), A(cb, 0, QA_SRHO), Ba, Bb);
    // unmapped cell indices: an outflow ghost cell's phi comes from its own (mirrored) neighbours
    const double ts = theta_s<false>(d, g, 0, f - 1, 0, f, 0);
    double *out = d.fx + f;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      double Fh = 0.0, Fl;
      if (k != 4) {
        const int s = QP_F1 + fslot(0, k);
        Fh = PW(f, 0, s);
        Fl = 0.5 * fma(-al, Ub(cb, 0, k) - Ub(ca, 0, k), A(ca, 0, s) + A(cb, 0, s));
      } else {
        Fl = -0.5 * al * (Ub(cb, 0, k) - Ub(ca, 0, k));
      }
      out[(QF_FLLF + k) * PS] = Fl;
      out[(QF_G + k) * PS] = is_one(ts) ? Fh - Fl : ts * (Fh - Fl);
    }
    out[QF_TS * PS] = ts;
    out[QF_AL * PS] = al;
    nsens = ts < 0.99;
  }
  if (g.kappa != 0.0 && nsens) atomicAdd(&d.st->cnt[ST_SENSOR_LT099], 1ull);
}

// P4 (1D): per cell, U^LLF = U^{Lim,1}, the anti-diffusive fluxes H_L, H_R and
// Lambda_L, Lambda_R (or the unlimited update without PP)
// The FP64 bounds D_k = |dt/dx G_L,k| + |dt/dx G_R,k| and box certificate of 1D cell i
// for the states box_cert32 leaves undecided (not inlined; Lim1 by value, G reloaded)
__device__ __noinline__ bool box_cert64_1d(const AfDev &d, const AfGrid &g, int i, int ip, double l0, double l1,
                                           double l2, double l3, double l4, double l5, double l6, double l7,
                                           double cxf) {
  const WV FX = wview(d.fx, g);
  const double L1[8] = {l0, l1, l2, l3, l4, l5, l6, l7};
  double D[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) D[k] = absd(cxf * FX(i, 0, QF_G + k)) + absd(-cxf * FX(ip, 0, QF_G + k));
  return box_certified(L1, D, g);
}

__device__ __forceinline__ void b1_cells(const AfDev &d, const AfGrid &g, int i, double a, double b) {
  const size_t PS = (size_t)g.nxa;
  int nlam = 0, ncfl = 0;
  NewtonLog nl = {0, 0};
  if (i < g.nx) {
    const double dt = d.sc->dt, cxf = dt * g.rdx;
    const int ip = mface(i + 1, g.nx, g.bc);
    const WV FX = wview(d.fx, g);
    const SV Ub = sview(d.us[0], g, 0);
    double Ullf[8], H[4][8], Gf[4][8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const double fl = FX(i, 0, QF_FLLF + k), fr = FX(ip, 0, QF_FLLF + k);
      const double gl = FX(i, 0, QF_G + k), gr = FX(ip, 0, QF_G + k);
      Ullf[k] = fma(-cxf, fr - fl, Ub(i, 0, k));
      H[0][k] = cxf * gl;
      H[1][k] = -cxf * gr;
      H[2][k] = 0.0;
      H[3][k] = 0.0;
      Gf[0][k] = gl;
      Gf[1][k] = gr;
      Gf[2][k] = Gf[3][k] = 0.0;
    }
    const size_t cs0 = (size_t)g.nx;
    if (!g.pp_on) {
      // no PP: the blended high-order update, then the RK combination
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const double fe = Ullf[k] + H[0][k] + H[1][k];
        d.uo[0][k * cs0 + i] = a == 0.0 ? fe : fma(a, __ldg(d.un[0] + k * cs0 + i), b * fe);
      }
    } else {
      if (dt * ((FX(i, 0, QF_AL) + FX(ip, 0, QF_AL)) * g.rdx) > 1.0 + 1e-12) ncfl = 1;   // Lemma 3.1 (count only)
      double Lam[4];
      // fast path: where the box provably needs no limiting, Lambda = 1 exactly
      // (the FP32 certificates of the 2D cell pass, with the lower and upper face values 0;
      // the FP64 forms only for the states they leave undecided)
      bool fast = clear_of_floor(Ullf, g);
      if (fast)
        fast = box_cert32(Ullf, Gf, cxf, 0.0, g.c13) ||
               box_cert64_1d(d, g, i, ip, Ullf[0], Ullf[1], Ullf[2], Ullf[3], Ullf[4], Ullf[5], Ullf[6], Ullf[7], cxf);
      if (fast) {
        Lam[0] = Lam[1] = 1.0;
      } else {
        const double eps_rho = fmin(1e-13, Ullf[0]);
        const double eps_p = fmin(1e-13, pressure(Ullf, g.gm1));
        flux_limiter_box(Ullf, H, eps_rho, eps_p, g.gm1, Lam, nl);
        nlam = lt_one(Lam[0]) || lt_one(Lam[1]);
      }
#pragma unroll
      for (int k = 0; k < 8; ++k) d.lim1[k * PS + i] = Ullf[k];
      d.lam[0 * PS + i] = Lam[0];
      d.lam[1 * PS + i] = Lam[1];
    }
  }
  if (nlam) atomicAdd(&d.st->cnt[ST_LAMBDA_LT1], 1ull);
  if (ncfl) atomicAdd(&d.st->cnt[ST_CFL_VIOLATIONS], 1ull);
  if (nl.solves) {
    atomicAdd(&d.st->cnt[ST_NEWTON_SOLVES], (unsigned long long)nl.solves);
    atomicMax(&d.st->cnt[ST_NEWTON_MAXIT], (unsigned long long)nl.maxit);
  }
}

// face coefficient of face f: min(Lambda_R(f-1), Lambda_L(f)); an outflow
// boundary face takes the Lambda of its one cell
__device__ __forceinline__ double theta1(const AfGrid &g, const WV &L, int f) {
  if (g.bc == 1) {
    if (f == 0) return L(0, 0, 0);
    if (f == g.nx) return L(g.nx - 1, 0, 1);
    return minnn(L(f - 1, 0, 1), L(f, 0, 0));
  }
  return minnn(L(wrapi(f - 1, g.nx), 0, 1), L(wrapi(f, g.nx), 0, 0));
}

__device__ __forceinline__ void value1(const AfDev &d, const AfGrid &g, int i, double tl, double tr, double dt,
                                       double *out) {
  const WV FX = wview(d.fx, g), L1 = wview(d.lim1, g);
  const int ip = mface(i + 1, g.nx, g.bc);
  const double cxf = dt * g.rdx;
#pragma unroll
  for (int k = 0; k < 8; ++k)
    out[k] = fma(cxf, fma(-tr, FX(ip, 0, QF_G + k), tl * FX(i, 0, QF_G + k)), L1(i, 0, k));
}

// P5 (1D): face coefficients, the limited update, the admissibility check, RK
__device__ __forceinline__ void b1_final(const AfDev &d, const AfGrid &g, int i, double a, double b) {
  int nface = 0;
  if (i < g.nx) {
    const double dt = d.sc->dt;
    const WV L = wview(d.lam, g);
    const double tl = theta1(g, L, i), tr = theta1(g, L, i + 1);
    d.thx[i] = tl;
    nface += lt_one(tl);
    if (g.bc == 1 && i == g.nx - 1) {
      d.thx[i + 1] = tr;
      nface += lt_one(tr);
    }
    double fe[8];
    value1(d, g, i, tl, tr, dt, fe);
    bool ok = fe[0] > 0.0 && qform(fe, 0.0) > 0.0;
#pragma unroll
    for (int k = 0; k < 8; ++k) ok = ok && finite_bits(fe[k]);
    if (!ok) {
      const int slot = atomicAdd(&d.st->nrepair, 1);
      if (slot < AF_MAX_REPAIR) d.st->repair[slot] = i;
      else atomicOr(&d.st->err, AFE_REPAIR_OVERFLOW);
    }
    const size_t cs0 = (size_t)g.nx;
#pragma unroll
    for (int k = 0; k < 8; ++k) d.uo[0][k * cs0 + i] = a == 0.0 ? fe[k] : fma(a, __ldg(d.un[0] + k * cs0 + i), b * fe[k]);
  }
  if (nface) atomicAdd(&d.st->cnt[ST_FACE_THETA_LT1], (unsigned long long)nface);
}

// Remark 4.1 for the flagged cells, one thread, in cell order (as in 2D, two faces)
__device__ void b1_repair(const AfDev &d, const AfGrid &g, double a, double b) {
  int n = d.st->nrepair;
  if (n <= 0) return;
  if (n > AF_MAX_REPAIR) n = AF_MAX_REPAIR;
  int *list = d.st->repair;
  for (int p = 1; p < n; ++p) {
    int v = list[p], q = p - 1;
    while (q >= 0 && list[q] > v) { list[q + 1] = list[q]; --q; }
    list[q + 1] = v;
  }
  const double dt = d.sc->dt;
  const size_t cs0 = (size_t)g.nx;
  unsigned long long nshr = 0, nbad = 0;
  auto face_idx = [&](int f) { return g.bc == 0 ? wrapi(f, g.nx) : f; };
  auto store = [&](int c, const double *fe) {
    for (int k = 0; k < 8; ++k)
      d.uo[0][k * cs0 + c] = a == 0.0 ? fe[k] : fma(a, d.un[0][k * cs0 + c], b * fe[k]);
  };
  for (int p = 0; p < n; ++p) {
    const int i = list[p];
    double fe[8];
    value1(d, g, i, d.thx[face_idx(i)], d.thx[face_idx(i + 1)], dt, fe);
    if (in_G(fe, g.gm1)) continue;
    nshr++;
    const double t0[2] = {d.thx[face_idx(i)], d.thx[face_idx(i + 1)]};
    for (int m = 0; m <= 10; ++m) {
      double t[2];
      for (int I = 0; I < 2; ++I) t[I] = (m < 10) ? fmax(0.0, t0[I] - ldexp(1e-8, m)) : 0.0;
      value1(d, g, i, t[0], t[1], dt, fe);
      if (in_G(fe, g.gm1) || m == 10) {
        d.thx[face_idx(i)] = t[0];
        d.thx[face_idx(i + 1)] = t[1];
        store(i, fe);
        if (!in_G(fe, g.gm1)) nbad++;
        break;
      }
    }
    for (int q = -1; q <= 1; q += 2) {
      int c = i + q;
      if (g.bc == 1 && (c < 0 || c >= g.nx)) continue;
      c = wrapi(c, g.nx);
      value1(d, g, c, d.thx[face_idx(c)], d.thx[face_idx(c + 1)], dt, fe);
      store(c, fe);
    }
  }
  d.st->nrepair = 0;
  if (nshr) {
    d.st->cnt[ST_SHRINK] += nshr;
    d.st->cnt[ST_CELL_SHRINK] += nshr;
  }
  if (nbad) {
    d.st->cnt[ST_NONADMISSIBLE] += nbad;
    d.st->err |= AFE_NONADMISSIBLE;
  }
}

__global__ void __launch_bounds__(128) k1_pointdata(const __grid_constant__ AfDev d, const __grid_constant__ AfGrid g,
                                                    int reduce_dt) {
  b1_pointdata(d, g, blockIdx.x * blockDim.x + threadIdx.x, reduce_dt);
}
__global__ void __launch_bounds__(128) k1_points(const __grid_constant__ AfDev d, const __grid_constant__ AfGrid g,
                                                 double a, double b) {
  b1_points(d, g, blockIdx.x * blockDim.x + threadIdx.x, a, b);
}
__global__ void __launch_bounds__(128) k1_faces(const __grid_constant__ AfDev d, const __grid_constant__ AfGrid g) {
  b1_faces(d, g, blockIdx.x * blockDim.x + threadIdx.x);
}
__global__ void __launch_bounds__(128) k1_cells(const __grid_constant__ AfDev d, const __grid_constant__ AfGrid g,
                                                double a, double b) {
  b1_cells(d, g, blockIdx.x * blockDim.x + threadIdx.x, a, b);
}
__global__ void __launch_bounds__(128) k1_final(const __grid_constant__ AfDev d, const __grid_constant__ AfGrid g,
                                                double a, double b) {
  b1_final(d, g, blockIdx.x * blockDim.x + threadIdx.x, a, b);
}
__global__ void k1_repair(const __grid_constant__ AfDev d, const __grid_constant__ AfGrid g, double a, double b) {
  if (blockIdx.x == 0 && threadIdx.x == 0) b1_repair(d, g, a, b);
}

}  // namespace

// One 1D stage: P1 (with the dt pass when reduce_dt), P2..P5 and the repair
// pass; t (may be NULL) brackets each launch with an event pair.
void af_launch_stage1d(const AfDev &d, const AfGrid &g, double a, double b, int reduce_dt, cudaStream_t s,
                       AfEventTimer *t) {
  const unsigned nb = (unsigned)((g.nxa + 127) / 128);
  auto timed = [&](int k, auto launch) {
    const bool on = t && t->begin(k, s);
    launch();
    if (t) t->end(on, s);
  };
  timed(AF_K_POINTDATA, [&] { k1_pointdata<<<nb, 128, 0, s>>>(d, g, reduce_dt); });
  if (reduce_dt) timed(AF_K_DT, [&] { k_dt<<<1, 32, 0, s>>>(d, g); });
  timed(AF_K_POINTS, [&] { k1_points<<<nb, 128, 0, s>>>(d, g, a, b); });
  timed(AF_K_FACES, [&] { k1_faces<<<nb, 128, 0, s>>>(d, g); });
  timed(AF_K_CELLS, [&] { k1_cells<<<nb, 128, 0, s>>>(d, g, a, b); });
  if (g.pp_on) {
    timed(AF_K_FINAL, [&] { k1_final<<<nb, 128, 0, s>>>(d, g, a, b); });
    timed(AF_K_REPAIR, [&] { k1_repair<<<1, 32, 0, s>>>(d, g, a, b); });
  }
}
void af_launch_dt1d(const AfDev &d, const AfGrid &g, cudaStream_t s) {
  const unsigned nb = (unsigned)((g.nxa + 127) / 128);
  k1_pointdata<<<nb, 128, 0, s>>>(d, g, 1);
  k_dt<<<1, 32, 0, s>>>(d, g);
}
