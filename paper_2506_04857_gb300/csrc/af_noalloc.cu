// af_noalloc.cu -- af_rhs_noalloc: the semi-discrete right-hand side of
// af_rhs for callers that must not allocate device memory.
//
// Why: some host code cannot call cudaMalloc on its hot path -- for instance a
// framework that owns all device memory through its own pool and forbids
// allocations after start-up, or a real-time loop where a device allocation
// (which can block, synchronise the device, or fail under memory pressure) is
// not acceptable.  Such a caller passes the state and the output buffers and
// gets the right-hand side computed in a fixed scratch area that lives in
// this library's static device memory.
//
// The scratch is one file-scope __device__ array of fixed size, sized for
// index grids of up to AF_NOALLOC_MAX_POINTS = (nx [+1 for outflow]) x
// (ny [+1 for outflow]) points (4225, e.g. 64 x 64 outflow or 65 x 65
// periodic grids), 4.9 MB.  Every GPU on which the library's module is loaded
// holds it until the process exits.  Every call shares the array and leaves
// its last contents there; calls that overlap on the GPU (on different
// streams, or from different host threads) race on it.
#include <mutex>

#include "../../include/af.h"
#include "af_internal.h"

namespace {

constexpr int kMaxPoints = AF_NOALLOC_MAX_POINTS;
// doubles per work point used by the rhs kernels: point data of the four DoF
// classes and the centres (AF_NQA + 4 AF_NQP), centre values (8), face data (2 AF_NQF)
constexpr size_t kPerPoint = AF_NQA + 4 * AF_NQP + 8 + 2 * AF_NQF;
constexpr size_t kWorkDoubles = kPerPoint * kMaxPoints;
// scalars and status follow the work arrays, each at a 256-byte boundary
constexpr size_t kScalarsOff = (kWorkDoubles * sizeof(double) + 255) / 256 * 256;
constexpr size_t kStatusOff = kScalarsOff + (sizeof(AfScalars) + 255) / 256 * 256;
constexpr size_t kBytes = kStatusOff + (sizeof(AfStatus) + 255) / 256 * 256;

static __device__ __align__(256) unsigned char g_scratch[kBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char *g_addr[kMaxDevices];   // device address of g_scratch on each device (set-up once per device)

// Set-up on the current device: the symbol's name in host code is only a host
// stand-in, so the device address is looked up once per device with that
// device current.
int scratch_address(unsigned char **out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return AF_ECUDA;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) return AF_ECUDA;
    g_addr[dev] = (unsigned char *)p;
  }
  *out = g_addr[dev];
  return AF_OK;
}

}  // namespace

extern "C" int af_rhs_noalloc(int nx, int ny, double gamma, int bc, double x0, double x1, double y0, double y1,
                              const double *const U[4], double *const dUdt[4], void *stream) {
  if (nx < 4 || ny < 4 || !(gamma > 1.0) || (bc != AF_BC_PERIODIC && bc != AF_BC_OUTFLOW) || !(x1 > x0) ||
      !(y1 > y0) || !U || !dUdt)
    return AF_EINVAL;
  for (int c = 0; c < 4; ++c)
    if (!U[c] || !dUdt[c]) return AF_EINVAL;
  const int nxa = bc == AF_BC_OUTFLOW ? nx + 1 : nx, nya = bc == AF_BC_OUTFLOW ? ny + 1 : ny;
  if ((long long)nxa * nya > kMaxPoints) return AF_EBOUNDS;   // grid larger than the static scratch
  // dUdt must not overlap U: the kernels read U while they write dUdt.
  const size_t cls_bytes[4] = {8 * sizeof(double) * nx * ny, 8 * sizeof(double) * nxa * ny,
                               8 * sizeof(double) * nx * nya, 8 * sizeof(double) * nxa * nya};
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 4; ++b) {
      const char *o0 = (const char *)dUdt[a], *o1 = o0 + cls_bytes[a];
      const char *i0 = (const char *)U[b], *i1 = i0 + cls_bytes[b];
      if (o0 < i1 && i0 < o1) return AF_EINVAL;
    }
  unsigned char *base = nullptr;
  int rc = scratch_address(&base);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;

  AfGrid g{};
  g.nx = nx;
  g.ny = ny;
  g.bc = bc;
  g.nxa = nxa;
  g.nya = nya;
  g.ex[0] = nx;  g.ey[0] = ny;
  g.ex[1] = nxa; g.ey[1] = ny;
  g.ex[2] = nx;  g.ey[2] = nya;
  g.ex[3] = nxa; g.ey[3] = nya;
  g.dx = (x1 - x0) / nx;
  g.dy = (y1 - y0) / ny;
  g.rdx = 1.0 / g.dx;
  g.rdy = 1.0 / g.dy;
  g.gamma = gamma;
  g.gm1 = gamma - 1.0;
  g.kappa = 0.0;
  g.cfl = 0.2;
  g.c13 = 1e-13 / (gamma - 1.0);
  g.pp_on = 0;
  g.src_cell_on = 1;
  g.src_point_on = 1;
  g.upwind = 0;
  for (int k = 0; k < 4; ++k) g.side[k] = 0;
  g.special = 0;
  g.x0 = 0.0;
  g.in_lo = g.in_hi = 0.0;

  const size_t PS = (size_t)nxa * nya;
  double *w = (double *)base;
  AfDev d{};
  for (int c = 0; c < 4; ++c) {
    d.un[c] = U[c];
    d.us[c] = U[c];
    d.uo[c] = dUdt[c];
  }
  d.pd[0] = w; w += AF_NQA * PS;
  for (int k = 1; k <= 4; ++k) { d.pd[k] = w; w += AF_NQP * PS; }
  d.uc = w; w += 8 * PS;
  d.fx = w; w += AF_NQF * PS;
  d.fy = w; w += AF_NQF * PS;
  d.phi = d.lam = d.lim1 = d.thx = d.thy = nullptr;   // not touched by the rhs kernels
  d.sc = (AfScalars *)(base + kScalarsOff);
  d.st = (AfStatus *)(base + kStatusOff);
  // the event counters accumulate with atomics: start them at zero
  if (cudaMemsetAsync(d.st, 0, sizeof(AfStatus), s) != cudaSuccess) return AF_ECUDA;

  af_launch_pointdata(d, g, 0, s);
  af_launch_points(d, g, 0.0, 1.0, 1, s);
  af_launch_faces(d, g, 1, s);
  af_launch_cells(d, g, 0.0, 1.0, 1, s);
  return cudaGetLastError() == cudaSuccess ? AF_OK : AF_ECUDA;
}
