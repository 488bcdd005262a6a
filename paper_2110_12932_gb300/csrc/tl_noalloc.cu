// tl_box_step_noalloc: one backward-Euler step of the heat equation on a plate
// mesh, run by the same persistent solve kernel as the two-level path, with
// all of its scratch memory taken from a fixed, file-scope device array.
//
// Who needs this: callers that may not allocate device memory once they are
// running -- a host application whose own allocator owns the whole GPU, a
// real-time loop that forbids allocation after set-up, a plugin handed only
// input and output buffers.  They pass inputs and outputs; everything else
// the solve needs lives in `g_box_scratch` below, which every GPU that loads
// this library holds (about 19.2 MB) until the process exits.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

#include "tl.h"
#define TL_SOLVE_KERNEL_ONLY
#include "tl_solve.cuh"

using namespace tl;

namespace {

constexpr size_t kMaxNodes = TL_NOALLOC_MAX_NODES;
constexpr int kMaxGrid = 1024;       // cooperative grid cap (4 blocks per SM on up to 256 SMs)
static_assert(kMaxGrid <= MAX_GRID_BLOCKS, "reductions over at most MAX_GRID_BLOCKS slots");
constexpr size_t kAlign = 256;
constexpr int kMaxDevices = 64;

constexpr size_t align_up(size_t b) { return (b + kAlign - 1) / kAlign * kAlign; }

// Worst case over all meshes with at most kMaxNodes nodes: 24 nodal FP64 arrays
// (u, r x2, p x2, s x2, q x2, dinv and 2 x 7 exchange arrays), 10 per-element
// values (s_e, k_e and 8 eigenvalues; at most as many elements as nodes), the
// new element states (one byte per element), the top-face load (at most half
// the nodes) and its 1D factor tables (nnx + nny <= kMaxNodes / 4 + 2 per
// factor), the reduction slots, barrier / status words and the counters.
constexpr size_t kScratchBytes =
    24 * align_up(kMaxNodes * sizeof(double)) + 2 * align_up(kMaxNodes * sizeof(double)) +
    align_up(8 * kMaxNodes * sizeof(double)) + align_up(kMaxNodes) +
    align_up(kMaxNodes / 2 * sizeof(double)) + align_up((size_t)MAXRECT * (kMaxNodes / 4 + 2) * sizeof(double)) + align_up((size_t)RS_N * kMaxGrid * sizeof(double)) + align_up((size_t)RS_N * kMaxGrid * sizeof(float)) +
    align_up(BAR_WORDS * sizeof(unsigned int)) + align_up(sizeof(DevStats)) + 4 * kAlign;

}  // namespace

// The scratch array.  In host code `g_box_scratch` is only a host-side stand-in
// for the symbol, never a device address: its device address is looked up with
// cudaGetSymbolAddress once per device (see device_scratch) and passed on.
static __device__ __align__(256) unsigned char g_box_scratch[kScratchBytes];

namespace {

std::mutex g_mutex;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device; looked up on the
// first call for that device (with the device current) and cached.
tl_status device_scratch(unsigned char** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return TL_ECUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) return TL_ECUDA;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_box_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      return TL_ECUDA;
    }
    g_scratch_addr[dev] = p;
  }
  *out = (unsigned char*)g_scratch_addr[dev];
  return TL_OK;
}

struct Carver {
  unsigned char* p;
  size_t used = 0;
  template <typename T>
  T* take(size_t n) {
    T* r = (T*)(p + used);
    used += align_up(n * sizeof(T));
    return r;
  }
};

void box_constants(const Grid3& g, SolveArgs& a) {
  const double h[3] = {g.hx, g.hy, g.hz};
  double mu[3][2], ka[3][2];
  for (int d = 0; d < 3; ++d) {
    mu[d][0] = h[d] / 2.0;
    mu[d][1] = h[d] / 6.0;
    ka[d][0] = 0.0;
    ka[d][1] = 2.0 / h[d];
  }
  for (int m = 0; m < 8; ++m) {
    int mx = m & 1, my = (m >> 1) & 1, mz = (m >> 2) & 1;
    a.Mc[m] = 0.125 * mu[0][mx] * mu[1][my] * mu[2][mz];
    a.Kc[m] = 0.125 * (ka[0][mx] * mu[1][my] * mu[2][mz] + mu[0][mx] * ka[1][my] * mu[2][mz] +
                       mu[0][mx] * mu[1][my] * ka[2][mz]);
  }
  to_pair_form(a.Mc);
  to_pair_form(a.Kc);
  a.Md = (h[0] / 3.0) * (h[1] / 3.0) * (h[2] / 3.0);
  a.Kd = (1.0 / h[0]) * (h[1] / 3.0) * (h[2] / 3.0) + (h[0] / 3.0) * (1.0 / h[1]) * (h[2] / 3.0) +
         (h[0] / 3.0) * (h[1] / 3.0) * (1.0 / h[2]);
  a.vol8 = h[0] * h[1] * h[2] / 8.0;
  for (int i = 0; i < 8; ++i)
    for (int j = 0; j < 8; ++j) {
      double m1[3], k1[3];
      for (int d = 0; d < 3; ++d) {
        int id = (i >> d) & 1, jd = (j >> d) & 1;
        m1[d] = h[d] / 6.0 * (id == jd ? 2.0 : 1.0);
        k1[d] = (id == jd ? 1.0 : -1.0) / h[d];
      }
      a.Mhat[i * 8 + j] = m1[0] * m1[1] * m1[2];
      a.Khat[i * 8 + j] = k1[0] * m1[1] * m1[2] + m1[0] * k1[1] * m1[2] + m1[0] * m1[1] * k1[2];
    }
}

Tiling box_tiling(const Grid3& g, int target) {
  Tiling t{};
  t.ex = std::min(TXE, g.nx);
  t.ey = std::min(TYE, g.ny);
  t.ntx = (g.nx + t.ex - 1) / t.ex;
  t.nty = (g.ny + t.ey - 1) / t.ey;
  long long nxy = (long long)t.ntx * t.nty;
  long long ez = (g.nz * nxy + target - 1) / target;
  t.ez = (int)std::max<long long>(1, std::min<long long>(ez, g.nz));
  t.ntz = (g.nz + t.ez - 1) / t.ez;
  return t;
}

bool bad_desc(const tl_box_step_desc* d) {
  if (!d) return true;
  if (d->nx < 1 || d->ny < 1 || d->nz < 1) return true;
  if (!(d->Lx > 0 && d->Ly > 0 && d->Lz > 0 && d->dt > 0)) return true;
  if (!(d->rho > 0) || !(d->c0 > 0) || !(d->k0 > 0) || !(d->powder_factor > 0)) return true;
  if (d->laser_on && (!(d->radius > 0) || !(d->P >= 0) || !(d->eta >= 0))) return true;
  if (!(d->tol > 0) || d->max_iter < 1) return true;
  return false;
}

}  // namespace

extern "C" tl_status tl_box_step_noalloc(const tl_box_step_desc* d, const double* T_in, double* T_out,
                                         uint8_t* state, void* stream) {
  if (bad_desc(d) || !T_in || !T_out || !state) return TL_EINVAL;
  const long long nnx = (long long)d->nx + 1, nny = (long long)d->ny + 1, nnz = (long long)d->nz + 1;
  if (nnx * nny * nnz > (long long)kMaxNodes) return TL_EINVAL;  // beyond the fixed scratch
  unsigned char* base = nullptr;
  tl_status s = device_scratch(&base);
  if (s != TL_OK) return s;

  int dev = 0, nsm = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute((const void*)solve_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, STAGE_BYTES);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void*)solve_kernel<0>, NT, STAGE_BYTES);
  if (e != cudaSuccess || per_sm < 1) {
    cudaGetLastError();
    return TL_ECUDA;
  }

  SolveArgs a{};
  a.g = Grid3{d->nx, d->ny, d->nz, (int)nnx, (int)nny, (int)nnz, d->Lx / d->nx, d->Ly / d->ny, d->Lz / d->nz};
  a.t = box_tiling(a.g, nsm);
  const int ntiles = a.t.ntx * a.t.nty * a.t.ntz;
  const int grid = std::min(std::min(per_sm * nsm, kMaxGrid), ntiles);
  const size_t nn = (size_t)(nnx * nny * nnz), ne = (size_t)d->nx * d->ny * d->nz;

  Carver c{base};
  a.u = c.take<double>(nn);
  a.r = c.take<double>(nn);
  a.r2 = c.take<double>(nn);
  a.p0 = c.take<double>(nn);
  a.p1 = c.take<double>(nn);
  a.s0 = c.take<double>(nn);
  a.s1 = c.take<double>(nn);
  a.q = c.take<double>(nn);
  a.q2 = c.take<double>(nn);
  a.dinv = c.take<double>(nn);
  a.X = c.take<double>((size_t)xplane((int)nn) * NXB);
  a.X2 = c.take<double>((size_t)xplane((int)nn) * NXB);
  a.s_e = c.take<double>(ne);
  a.k_e = c.take<double>(ne);
  a.lam = c.take<double>(8 * ne);
  a.st_new = c.take<uint8_t>(ne);
  a.F = c.take<double>((size_t)(nnx * nny));
  a.G = c.take<double>((size_t)MAXRECT * (nnx + nny));
  a.red = c.take<double>((size_t)RS_N * kMaxGrid);
  a.red32 = c.take<float>((size_t)RS_N * kMaxGrid);
  unsigned int* words = c.take<unsigned int>(BAR_WORDS);  // barrier arrivals / generation, status
  a.stats = c.take<DevStats>(1);
  if (c.used > kScratchBytes) return TL_EINVAL;
  a.red_stride = kMaxGrid;
  a.bar = Barrier{reinterpret_cast<unsigned long long*>(words), (int*)(words + BAR_STATUS), BAR_DEFAULT_LIMIT_NS};

  a.T_in = T_in;
  a.T_out = T_out;
  a.state = state;
  a.st_sx = d->nx;
  a.st_sy = d->ny;
  a.st_ox = 0;
  a.st_oy = 0;
  a.dir.faces = 16;  // Dirichlet bottom; the other faces adiabatic
  a.dir.box[0] = 1; a.dir.box[1] = 0; a.dir.box[2] = 1; a.dir.box[3] = 0; a.dir.box[4] = 1; a.dir.box[5] = 0;
  a.dv.kind = 1;
  a.dv.T_bottom = d->T_bottom;
  a.dv.inj = nullptr;  // no injected nodes: never read
  if (d->laser_on && d->P != 0.0) {
    a.ld.kind = 1;
    a.ld.amp = 3.0 * d->eta * d->P / (M_PI * d->radius * d->radius);
    a.ld.alpha = std::sqrt(3.0) / d->radius;
    a.ld.xc = d->xc;
    a.ld.yc = d->yc;
  }
  a.mat = Material{d->rho, d->c0, d->c1, d->k0, d->k1, d->Tref, d->powder_factor, d->T_melt};
  a.dt = d->dt;
  a.tol = d->tol;
  a.max_iter = d->max_iter;
  a.energy = 0;
  a.update_state = 1;
  a.level = 1;
  box_constants(a.g, a);

  // The array keeps the previous call's contents: the barrier words, the
  // status word and the counters must start at zero.  Nothing else is read
  // before the solve writes it.
  cudaStream_t st = (cudaStream_t)stream;
  e = cudaMemsetAsync(words, 0, BAR_WORDS * sizeof(unsigned int), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(a.stats, 0, sizeof(DevStats), st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return TL_ECUDA;
  }
  void* args[] = {(void*)&a};
  e = cudaLaunchCooperativeKernel((const void*)solve_kernel<0>, dim3(grid), dim3(NT), args, STAGE_BYTES, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  int status = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&status, words + BAR_STATUS, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return TL_ECUDA;
  }
  return (tl_status)status;
}
