// C ABI of the two-level LPBF heat solve (declarations and contracts in
// include/tl.h).  Host side: validation, device memory, the macro-step state
// machine of Algorithm 1 (Section 4), laser path arithmetic, launches.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <tuple>
#include <vector>

#include "tl.h"
#include "tl_solve.cuh"

using namespace tl;

namespace {

enum Phase { NEED_PREDICT = 0, IN_SUBSTEPS = 1, NEED_CORRECT = 2 };

struct Level {
  Grid3 g{};
  Tiling t{};
  Tiling tb{};   // tiling used in batched launches (a slice of the grid)
  Tiling tw{};   // refined path on large meshes: wide tiles of the FP32 inner CG
  Tiling tp{};   // node tiles of the tensor preconditioner's pass
  int wide = 0;
  int tuned = 0; // 1: the tilings were chosen by timing (the autotuner)
  int grid = 0;  // cooperative grid size
  double* T = nullptr;    // current temperature
  double* T2 = nullptr;   // coarse: predictor T~+; fine: move double buffer
  double* u = nullptr;
  double* r = nullptr;
  double* r2 = nullptr;
  double* F = nullptr;
  double* G = nullptr;
  double* p0 = nullptr;
  double* p1 = nullptr;
  double* s0 = nullptr;
  double* s1 = nullptr;
  double* q = nullptr;
  double* X = nullptr;
  double* q2 = nullptr;
  double* X2 = nullptr;
  double* dinv = nullptr;
  double* s_e = nullptr;
  double* k_e = nullptr;
  double* lam = nullptr;
  float* d32 = nullptr;   // refined precision only
  float* r32 = nullptr;
  float* r32b = nullptr;
  float* q32 = nullptr;
  float* X32 = nullptr;
  float* q32b = nullptr;
  float* X32b = nullptr;
  float* p0f = nullptr;
  float* p1f = nullptr;
  float* s0f = nullptr;
  float* s1f = nullptr;
  float* dinv32 = nullptr;
  float* sk32 = nullptr;
  double* inj = nullptr;  // coarse only
  double* T3 = nullptr;   // iterated coupling (coarse): the corrected fields of two consecutive sweeps
  double* T3b = nullptr;
  uint8_t* state_snap = nullptr;  // iterated coupling: states before the superseded solve (fine: patch window)
  double* Tp = nullptr;           // Picard iterations: the coefficient temperature between solves
  unsigned long long* trace = nullptr;  // phase timestamps of the level's last solve
  uint8_t* state = nullptr;
  uint8_t* st_new = nullptr;  // new element states of a solve until its commit
  double* hf = nullptr;       // top-surface losses: transfer coefficient per top face
  float* hf32 = nullptr;
  int st_sx = 0, st_sy = 0, st_sz = 0;
  double Mc[8], Kc[8], Md = 0, Kd = 0, vol8 = 0, Mhat[64], Khat[64];
};

}  // namespace

struct tl_problem {
  tl_config cfg{};
  std::vector<tl_track> tracks;
  std::vector<double> t_start, t_end, dur;
  Level C, Fi;
  int oi = 0, oj = 0, ok = 0;
  int n = 0;        // macro step index
  int sub = 0;      // micro steps done in the current macro step
  int phase = NEED_PREDICT;
  long long patch_moves = 0;
  long long launches = 0;
  cudaStream_t stream = nullptr;
  unsigned int* bar = nullptr;  // grid barrier words (BAR_WORDS), status included
  int* status = nullptr;
  double* red = nullptr;
  float* red32 = nullptr;
  int red_stride = 0;   // reduction slots per row: the cooperative grid cap
  int max_slice = 0;    // the most blocks a solve of this problem uses
  unsigned int* tune_bar = nullptr;  // barrier / status words of the tuner's timing runs
  DevStats* stats = nullptr;
  unsigned long long* d_diff = nullptr;  // iterated coupling: max |change|, max |T+| (IEEE bits)
  long long coupling_resolves = 0;
  std::vector<void*> allocs;
  int nsm = 0, max_coop = 0;
};

namespace {

// The solve kernel for a precision mode (0 plain FP64, 1 refined, 2 either).
const void* solve_kernel_for(int pmode) {
  return pmode == 0 ? (const void*)solve_kernel<0> : (const void*)solve_kernel<1>;
}
const void* batch_kernel_for(int pmode) {
  return pmode == 0 ? (const void*)solve_batch_kernel<0>
                    : (pmode == 1 ? (const void*)solve_batch_kernel<1> : (const void*)solve_batch_kernel<2>);
}
int pmode_of(const tl_config& c) { return c.precision == TL_FP32_REFINED ? 1 : 0; }

tl_status dev_alloc(tl_problem* p, void** out, size_t bytes) {
  *out = nullptr;
  if (bytes == 0) bytes = 16;
  void* ptr = nullptr;
  if (p->cfg.alloc) {
    ptr = p->cfg.alloc(bytes, (void*)p->stream, p->cfg.alloc_ctx);
    if (!ptr) return TL_ENOMEM;
    if (reinterpret_cast<uintptr_t>(ptr) % 16 != 0) {  // the kernels use 16-byte vector accesses
      if (p->cfg.free) p->cfg.free(ptr, (void*)p->stream, p->cfg.alloc_ctx);
      return TL_EINVAL;
    }
  } else {
    cudaError_t e = cudaMalloc(&ptr, bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return e == cudaErrorMemoryAllocation ? TL_ENOMEM : TL_ECUDA;
    }
  }
  p->allocs.push_back(ptr);
  *out = ptr;
  return TL_OK;
}

template <typename T>
tl_status alloc_n(tl_problem* p, T** out, size_t n) {
  void* v = nullptr;
  tl_status s = dev_alloc(p, &v, n * sizeof(T));
  *out = (T*)v;
  return s;
}

// Element constants of a box element hx*hy*hz (see tl_device.cuh): the Hadamard
// eigenvalue factors Mc, Kc (1/8 folded in), the diagonal factors and the
// explicit element matrices used for the Dirichlet reactions.
void element_constants(Level& L) {
  const double h[3] = {L.g.hx, L.g.hy, L.g.hz};
  double mu[3][2], ka[3][2];
  for (int d = 0; d < 3; ++d) {
    mu[d][0] = h[d] / 2.0;
    mu[d][1] = h[d] / 6.0;
    ka[d][0] = 0.0;
    ka[d][1] = 2.0 / h[d];
  }
  for (int m = 0; m < 8; ++m) {
    int mx = m & 1, my = (m >> 1) & 1, mz = (m >> 2) & 1;
    L.Mc[m] = 0.125 * mu[0][mx] * mu[1][my] * mu[2][mz];
    L.Kc[m] = 0.125 * (ka[0][mx] * mu[1][my] * mu[2][mz] + mu[0][mx] * ka[1][my] * mu[2][mz] +
                       mu[0][mx] * mu[1][my] * ka[2][mz]);
  }
  L.Md = (h[0] / 3.0) * (h[1] / 3.0) * (h[2] / 3.0);
  L.Kd = (1.0 / h[0]) * (h[1] / 3.0) * (h[2] / 3.0) + (h[0] / 3.0) * (1.0 / h[1]) * (h[2] / 3.0) +
         (h[0] / 3.0) * (h[1] / 3.0) * (1.0 / h[2]);
  L.vol8 = h[0] * h[1] * h[2] / 8.0;
  for (int a = 0; a < 8; ++a)
    for (int b = 0; b < 8; ++b) {
      double m1[3], k1[3];
      for (int d = 0; d < 3; ++d) {
        int ad = (a >> d) & 1, bd = (b >> d) & 1;
        m1[d] = h[d] / 6.0 * (ad == bd ? 2.0 : 1.0);
        k1[d] = (ad == bd ? 1.0 : -1.0) / h[d];
      }
      L.Mhat[a * 8 + b] = m1[0] * m1[1] * m1[2];
      L.Khat[a * 8 + b] = k1[0] * m1[1] * m1[2] + m1[0] * k1[1] * m1[2] + m1[0] * m1[1] * k1[2];
    }
}

// Tile shape for the apply.  The FP64 apply is bound by the SM's FP64 pipe, so
// the time of a step is set by the SM that holds the most element work: the
// model charges an SM (blocks it hosts) x (tiles per block) tiles of
// ex*ey*ez elements at the per-element FP64 instruction count of the tile
// shape (window columns and partial node layers cost extra), plus a fixed
// cost per layer and tile for the block barriers, divided by the pipe
// utilisation that one or two resident 8-warp blocks reach.
void choose_tiling(Level& L, int nsm, int per_sm, std::vector<Tiling>* ranked = nullptr) {
  const Grid3& g = L.g;
  double best = 1e300;
  Tiling bt{};
  std::vector<std::pair<double, Tiling>> all;
  const int exs[] = {16, 8};
  const int eys[] = {8, 4, 2, 1};
  for (int ex0 : exs)
    for (int ey0 : eys)
      for (int ez = 1; ez <= g.nz; ++ez) {
        const int ex = std::min(ex0, g.nx), ey = std::min(ey0, g.ny);
        const long long T = (long long)((g.nx + ex - 1) / ex) * ((g.ny + ey - 1) / ey) * ((g.nz + ez - 1) / ez);
        const double rxy = (double)(ex + 1) * (ey + 1) / ((double)ex * ey);
        const double rz = (double)(ez + 1) / ez;
        const double ops = 2 * rxy + 2 * rxy * rz + 4.0 * (ex + 1) / ex + 20 + 8.0 * (ex + 1) / ex + 5 * rxy + rxy * rz;
        const double per_tile = (double)ex * ey * ez * ops + 1500.0 * (ez + 1);
        const long long G = std::min<long long>(T, (long long)nsm * per_sm);
        const long long b = (G + nsm - 1) / nsm, tb = (T + G - 1) / G;
        const double eff = b >= 4 ? 0.85 : (b >= 2 ? 0.7 : 0.4);
        const double cost = (double)(b * tb) * per_tile / eff;
        const Tiling t{ex, ey, ez, (g.nx + ex - 1) / ex, (g.ny + ey - 1) / ey, (g.nz + ez - 1) / ez};
        if (ranked) all.push_back({cost, t});
        if (cost < best * (1 - 1e-9)) {
          best = cost;
          bt = t;
        }
      }
  L.t = bt;
  if (ranked) {  // distinct shapes, cheapest first
    std::stable_sort(all.begin(), all.end(), [](const auto& x, const auto& y) { return x.first < y.first; });
    ranked->clear();
    for (const auto& c : all) {
      bool dup = false;
      for (const Tiling& r : *ranked) dup |= r.ex == c.second.ex && r.ey == c.second.ey && r.ntz == c.second.ntz;
      if (!dup) ranked->push_back(c.second);
    }
  }
}

// Wide tiles (AX x AY x ez elements) of the FP32 inner CG on large meshes.
// The tile depth is set empirically: a sweep of the wide apply over
// ez = 2 ... nz on 256 x 256 x 128, 128 x 128 x 64 and 192 x 96 x 48 element
// meshes (608 blocks) was fastest at ez = 16-24, 8 and 4-8, i.e. about nz / 8,
// within 4 % of the best everywhere.
Tiling wide_tiling(const Grid3& g, int /*nblk*/) {
  const int ntx = (g.nx + AX - 1) / AX, nty = (g.ny + AY - 1) / AY;
  const int ez = std::max(1, (g.nz + 4) / 8);
  return Tiling{AX, AY, ez, ntx, nty, (g.nz + ez - 1) / ez};
}

// Node-owned tiles of the tensor preconditioner's pass: rows split into equal
// widths of at most 64 columns (two per thread), as many rows as fill the
// block, and the
// z-depth ez that minimises the layer steps of the busiest block: a tile of ez
// owned layers marches through ez + 2 layers and costs about PC_TILE_STEPS
// more for its prologue and drain, and a block runs ceil(tiles / blocks)
// tiles.  (On the 20 mm patch the earlier rule, about four tiles per block,
// gave 3-layer tiles and 28 step-equivalents per block; this one gives
// 13-layer tiles and 17.)
constexpr int PC_TILE_STEPS = 2;

Tiling pc_tiling(const Grid3& g, int nblk) {
  const int ntx = (g.nnx + 63) / 64;
  const int tx = (g.nnx + ntx - 1) / ntx;                 // at most 64 columns, two per thread
  // rows: as many as the block's threads cover, the stored window (rows of
  // tx + 2 nodes at an even pitch, ty + 2 rows) at most PC_WN_MAX
  const int ty = std::max(1, std::min({g.nny, NT / ((tx + 1) / 2), PC_WN_MAX / ((tx + 3) & ~1) - 2}));
  const int nty = (g.nny + ty - 1) / ty;
  const long long cols = (long long)ntx * nty;
  const long long B = std::max(1, nblk);
  int best_ez = g.nnz;
  long long best = -1;
  for (int ez = std::min(2, g.nnz); ez <= g.nnz; ++ez) {
    const long long ntz = (g.nnz + ez - 1) / ez;
    if (ez > 2 && (g.nnz + ez - 2) / (ez - 1) == ntz) continue;  // same chunk count as a thinner ez
    const long long cost = (cols * ntz + B - 1) / B * (ez + 2 + PC_TILE_STEPS);
    if (best < 0 || cost < best) {
      best = cost;
      best_ez = ez;
    }
  }
  return Tiling{tx, ty, best_ez, ntx, nty, (g.nnz + best_ez - 1) / best_ez};
}

// With inner_tiles = 0 the refined path runs its inner CG on wide tiles when
// the mesh gives the blocks that solve it at least this many elements each.
// Measured: the fused element-tile CG is faster with 256 elements per block
// (10 mm patch on the whole GPU; a batch job alone), the wide two-phase CG
// with 1.7e3 (20 mm patch), 1.4e4 (256 x 256 x 128) and ~2e4 (crowded batch
// rounds, 64 jobs).
constexpr long long WIDE_MIN_ELEMS_PER_BLOCK = 1024;

bool use_wide(const tl_config& c, const Grid3& g, int blocks) {
  if (c.precision != TL_FP32_REFINED) return false;
  if (c.inner_tiles != 0) return c.inner_tiles == 2;
  return (long long)g.nx * g.ny * g.nz >= WIDE_MIN_ELEMS_PER_BLOCK * std::max(1, blocks);
}

// Stefan-Boltzmann constant (CODATA 2018) [W/(m^2 K^4)].
constexpr double SIGMA_SB = 5.670374419e-8;

bool surface_on(const tl_config& c) { return c.h_conv > 0 || c.emissivity > 0; }

tl_status alloc_level(tl_problem* p, Level& L, bool coarse) {
  const size_t nn = (size_t)L.g.nnx * L.g.nny * L.g.nnz;
  const size_t ne = (size_t)L.g.nx * L.g.ny * L.g.nz;
  tl_status s;
  if ((s = alloc_n(p, &L.T, nn)) != TL_OK) return s;
  if ((s = alloc_n(p, &L.T2, nn)) != TL_OK) return s;
  if ((s = alloc_n(p, &L.u, nn)) != TL_OK) return s;
  if ((s = alloc_n(p, &L.r, nn)) != TL_OK) return s;
  if ((s = alloc_n(p, &L.F, (size_t)L.g.nnx * L.g.nny)) != TL_OK) return s;
  if ((s = alloc_n(p, &L.G, (size_t)MAXRECT * (L.g.nnx + L.g.nny))) != TL_OK) return s;
  if ((s = alloc_n(p, &L.q, nn)) != TL_OK) return s;
  if ((s = alloc_n(p, &L.X, (size_t)xplane((int)nn) * NXB)) != TL_OK) return s;
  if (p->cfg.precision == TL_FP64) {
    if ((s = alloc_n(p, &L.r2, nn)) != TL_OK) return s;
    if ((s = alloc_n(p, &L.p0, nn)) != TL_OK) return s;
    if ((s = alloc_n(p, &L.p1, nn)) != TL_OK) return s;
    if ((s = alloc_n(p, &L.s0, nn)) != TL_OK) return s;
    if ((s = alloc_n(p, &L.s1, nn)) != TL_OK) return s;
    if ((s = alloc_n(p, &L.q2, nn)) != TL_OK) return s;
    if ((s = alloc_n(p, &L.X2, (size_t)xplane((int)nn) * NXB)) != TL_OK) return s;
  }
  if ((s = alloc_n(p, &L.dinv, nn)) != TL_OK) return s;
  if ((s = alloc_n(p, &L.s_e, ne)) != TL_OK) return s;
  if ((s = alloc_n(p, &L.k_e, ne)) != TL_OK) return s;
  if ((s = alloc_n(p, &L.lam, 8 * ne)) != TL_OK) return s;
  if (p->cfg.precision == TL_FP32_REFINED) {
    if ((s = alloc_n(p, &L.d32, nn)) != TL_OK) return s;
    if ((s = alloc_n(p, &L.r32, nn)) != TL_OK) return s;
    if ((s = alloc_n(p, &L.r32b, nn)) != TL_OK) return s;
    if ((s = alloc_n(p, &L.q32, nn)) != TL_OK) return s;
    if ((s = alloc_n(p, &L.X32, (size_t)xplane((int)nn) * NXB)) != TL_OK) return s;
    if ((s = alloc_n(p, &L.q32b, nn)) != TL_OK) return s;
    if ((s = alloc_n(p, &L.X32b, (size_t)xplane((int)nn) * NXB)) != TL_OK) return s;
    if ((s = alloc_n(p, &L.p0f, nn)) != TL_OK) return s;
    if ((s = alloc_n(p, &L.p1f, nn)) != TL_OK) return s;
    if ((s = alloc_n(p, &L.s0f, nn)) != TL_OK) return s;
    if ((s = alloc_n(p, &L.s1f, nn)) != TL_OK) return s;
    if ((s = alloc_n(p, &L.dinv32, nn)) != TL_OK) return s;
    if ((s = alloc_n(p, &L.sk32, 2 * ne)) != TL_OK) return s;
  }
  if (coarse && (s = alloc_n(p, &L.inj, nn)) != TL_OK) return s;
  if (p->cfg.coupling_sweeps > 1) {
    if (coarse) {
      if ((s = alloc_n(p, &L.T3, nn)) != TL_OK) return s;
      if ((s = alloc_n(p, &L.T3b, nn)) != TL_OK) return s;
    }
    if ((s = alloc_n(p, &L.state_snap, ne)) != TL_OK) return s;
  }
  if (p->cfg.picard_iters > 1 && (s = alloc_n(p, &L.Tp, nn)) != TL_OK) return s;
  if ((s = alloc_n(p, &L.trace, 2 * TRACE_CAP)) != TL_OK) return s;
  if ((s = alloc_n(p, &L.state, (size_t)L.st_sx * L.st_sy * L.st_sz)) != TL_OK) return s;
  if ((s = alloc_n(p, &L.st_new, ne)) != TL_OK) return s;
  if (surface_on(p->cfg)) {
    const size_t nf = (size_t)L.g.nx * L.g.ny;
    if ((s = alloc_n(p, &L.hf, nf)) != TL_OK) return s;
    if (p->cfg.precision == TL_FP32_REFINED && (s = alloc_n(p, &L.hf32, nf)) != TL_OK) return s;
  }
  return TL_OK;
}

tl_status cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return TL_OK;
  cudaGetLastError();
  return e == cudaErrorMemoryAllocation ? TL_ENOMEM : TL_ECUDA;
}

// ---- laser path (Section 5.2-5.3): tracks back to back from t = 0 --------
bool laser_at(const tl_problem* p, double t, double* x, double* y) {
  for (size_t j = 0; j < p->tracks.size(); ++j) {
    if (t <= p->t_end[j]) {
      const tl_track& k = p->tracks[j];
      double f = (t - p->t_start[j]) / p->dur[j];
      *x = k.x0 + f * (k.x1 - k.x0);
      *y = k.y0 + f * (k.y1 - k.y0);
      return true;
    }
  }
  return false;
}

// Patch origin (coarse node indices) centring the patch on (x, y), clamped to the plate.
void origin_at(const tl_problem* p, double x, double y, int* oi, int* oj) {
  const tl_config& c = p->cfg;
  const double hcx = c.Lx / c.NXc, hcy = c.Ly / c.NYc;
  int ii = (int)std::floor((x - 0.5 * c.pNXc * hcx) / hcx + 0.5);
  int jj = (int)std::floor((y - 0.5 * c.pNYc * hcy) / hcy + 0.5);
  *oi = std::min(std::max(ii, 0), c.NXc - c.pNXc);
  *oj = std::min(std::max(jj, 0), c.NYc - c.pNYc);
}

// Origin for macro step n: laser position at t_n + Dt/2; unchanged if the laser is off.
void origin_for(const tl_problem* p, int n, int* oi, int* oj) {
  const double Dt = p->cfg.dt_coarse;
  double x, y;
  if (!laser_at(p, n * Dt + 0.5 * Dt, &x, &y)) return;
  origin_at(p, x, y, oi, oj);
}

LoadSpec gaussian_load(const tl_problem* p, const Level& L, double t, double ox, double oy) {
  LoadSpec ld{};
  double x, y;
  if (!laser_at(p, t, &x, &y) || p->cfg.P == 0.0) {
    ld.kind = 0;
    return ld;
  }
  const double R = p->cfg.radius;
  ld.kind = 1;
  ld.amp = 3.0 * p->cfg.eta * p->cfg.P / (M_PI * R * R);
  ld.alpha = std::sqrt(3.0) / R;
  ld.xc = x;
  ld.yc = y;
  ld.ox = ox;
  ld.oy = oy;
  (void)L;
  return ld;
}

// Coarse source over [t_n, t_n + Dt]: surface analogue of Q+ = P eta/(r d v Dt)
// (Section 5.2) on the R-wide rectangle swept along each axis-aligned track.
LoadSpec box_load(const tl_problem* p, int n) {
  LoadSpec ld{};
  const tl_config& c = p->cfg;
  const double Dt = c.dt_coarse, R = c.radius;
  const double ta = n * Dt, tb = (n + 1) * Dt;
  ld.kind = 2;
  ld.ox = 0.0;
  ld.oy = 0.0;
  for (size_t j = 0; j < p->tracks.size() && ld.nrect < MAXRECT; ++j) {
    double a = std::max(ta, p->t_start[j]);
    double b = std::min(tb, p->t_end[j]);
    if (!(b > a)) continue;
    const tl_track& k = p->tracks[j];
    double fa = (a - p->t_start[j]) / p->dur[j], fb = (b - p->t_start[j]) / p->dur[j];
    double xa = k.x0 + fa * (k.x1 - k.x0), ya = k.y0 + fa * (k.y1 - k.y0);
    double xb = k.x0 + fb * (k.x1 - k.x0), yb = k.y0 + fb * (k.y1 - k.y0);
    double q = c.eta * c.P / (R * k.speed * Dt);
    double* rc = ld.rect[ld.nrect];
    if (k.y0 == k.y1) {
      rc[0] = std::min(xa, xb); rc[1] = std::max(xa, xb);
      rc[2] = k.y0 - 0.5 * R;   rc[3] = k.y0 + 0.5 * R;
    } else {
      rc[0] = k.x0 - 0.5 * R;   rc[1] = k.x0 + 0.5 * R;
      rc[2] = std::min(ya, yb); rc[3] = std::max(ya, yb);
    }
    rc[4] = q;
    ld.nrect++;
  }
  if (ld.nrect == 0 || c.P == 0.0) ld.kind = 0;
  return ld;
}

// Time limit of the device barriers' waits: barrier_timeout seconds, 1 s by default.
unsigned long long barrier_limit_ns(const tl_config& c) {
  if (!(c.barrier_timeout > 0)) return BAR_DEFAULT_LIMIT_NS;
  const double ns = c.barrier_timeout * 1e9;
  return ns < 1.0 ? 1ull : (ns > 6e10 ? 60000000000ull : (unsigned long long)ns);
}

void fill_common(const tl_problem* p, const Level& L, SolveArgs& a) {
  a.g = L.g;
  a.t = L.t;
  a.wide = L.wide;
  a.tw = L.tw;
  a.tp = L.tp;
  a.u = L.u;
  a.r = L.r;
  a.r2 = L.r2;
  a.p0 = L.p0;
  a.p1 = L.p1;
  a.s0 = L.s0;
  a.s1 = L.s1;
  a.q = L.q;
  a.X = L.X;
  a.q2 = L.q2;
  a.X2 = L.X2;
  a.dinv = L.dinv;
  a.s_e = L.s_e;
  a.k_e = L.k_e;
  a.lam = L.lam;
  a.d32 = L.d32;
  a.r32 = L.r32;
  a.r32b = L.r32b;
  a.q32 = L.q32;
  a.X32 = L.X32;
  a.q32b = L.q32b;
  a.X32b = L.X32b;
  a.p0f = L.p0f;
  a.p1f = L.p1f;
  a.s0f = L.s0f;
  a.s1f = L.s1f;
  a.dinv32 = L.dinv32;
  a.sk32 = L.sk32;
  a.precision = p->cfg.precision == TL_FP32_REFINED ? PREC_FP32_REFINED : PREC_FP64;
  a.tol_inner = p->cfg.tol_inner;
  a.max_outer = 20;
  // preconditioner: 1 Jacobi; 0 (default) or 2 the tensor-product one, which
  // was faster in both precisions on every measured patch (139k to 8.5M
  // nodes): its extra pass costs less than the iterations it saves
  a.precond = p->cfg.precond == 1 ? 0 : 1;
  a.F = L.F;
  a.G = L.G;
  a.state = L.state;
  a.st_new = L.st_new;
  const tl_config& c = p->cfg;
  // top-surface losses (Section 3.1): convection on both levels, radiation on
  // the local (fine) level only
  a.surf = surface_on(c) ? 1 : 0;
  a.h_conv = c.h_conv;
  a.rad = &L == &p->Fi ? SIGMA_SB * c.emissivity : 0.0;
  a.T_amb = c.T_amb;
  a.hf = L.hf;
  a.hf32 = L.hf32;
  a.Mfx[0] = L.g.hx / 3.0;
  a.Mfx[1] = L.g.hx / 6.0;
  a.Mfy[0] = L.g.hy / 3.0;
  a.Mfy[1] = L.g.hy / 6.0;
  a.mat = Material{c.rho, c.c0, c.c1, c.k0, c.k1, c.Tref, c.powder_factor, c.T_melt,
                   c.latent, c.pc_sharpness, 0.5 * (c.T_solidus + c.T_liquidus)};
  a.tol = c.tol;
  a.max_iter = c.max_iter;
  std::memcpy(a.Mc, L.Mc, sizeof a.Mc);
  std::memcpy(a.Kc, L.Kc, sizeof a.Kc);
  to_pair_form(a.Mc);
  to_pair_form(a.Kc);
  a.Md = L.Md;
  a.Kd = L.Kd;
  a.vol8 = L.vol8;
  std::memcpy(a.Mhat, L.Mhat, sizeof a.Mhat);
  std::memcpy(a.Khat, L.Khat, sizeof a.Khat);
  a.bar = Barrier{reinterpret_cast<unsigned long long*>(p->bar), p->status, barrier_limit_ns(c)};
  a.red = p->red;
  a.red32 = p->red32;
  a.red_stride = p->red_stride;
  a.stats = p->stats;
  a.trace = L.trace;
}

tl_status launch_solve(tl_problem* p, const Level& L, SolveArgs& a) {
  void* args[] = {(void*)&a};
  cudaError_t e = cudaLaunchCooperativeKernel(solve_kernel_for(pmode_of(p->cfg)), dim3(L.grid), dim3(NT), args,
                                              STAGE_BYTES, p->stream);
  p->launches++;
  return cuda_status(e);
}

// One backward-Euler step as picard_iters solves: every solve starts from
// T_in; solve j takes its coefficients at the temperature T*_j (T*_0 = T_in,
// then L.Tp), and every solve but the last writes only
// T*_{j+1} = T*_j + (T_j - T*_j) / 2 into L.Tp, without touching T_out, the
// states or the energy account.
tl_status launch_picard(tl_problem* p, const Level& L, SolveArgs& a) {
  const int K = std::max(1, p->cfg.picard_iters);
  if (K == 1) return launch_solve(p, L, a);
  const int upd = a.update_state, en = a.energy;
  for (int j = 0; j < K; ++j) {
    const bool last = j + 1 == K;
    a.T_coef = j == 0 ? nullptr : L.Tp;
    a.T_relax = last ? nullptr : L.Tp;
    a.update_state = last ? upd : 0;
    a.energy = last ? en : 0;
    const tl_status s = launch_solve(p, L, a);
    if (s != TL_OK) return s;
  }
  return TL_OK;
}

int fine_dir_faces(const tl_problem* p) {
  const tl_config& c = p->cfg;
  int f = 16;  // patch bottom: interface or plate bottom, Dirichlet either way
  if (p->oi > 0) f |= 1;
  if (p->oi + c.pNXc < c.NXc) f |= 2;
  if (p->oj > 0) f |= 4;
  if (p->oj + c.pNYc < c.NYc) f |= 8;
  return f;
}

void injection_box(const tl_problem* p, int box[6]) {
  const tl_config& c = p->cfg;
  int f = fine_dir_faces(p);
  box[0] = p->oi + ((f & 1) ? 1 : 0);
  box[1] = p->oi + c.pNXc - ((f & 2) ? 1 : 0);
  box[2] = p->oj + ((f & 4) ? 1 : 0);
  box[3] = p->oj + c.pNYc - ((f & 8) ? 1 : 0);
  box[4] = p->ok + 1;
  box[5] = c.NZc;
}

// Arguments of the coarse backward-Euler step (predictor, or corrector with the
// injected nodes as Dirichlet data: from the restriction buffer, or read from
// the fine field when the restriction is fused into the solve).
void build_coarse_args(tl_problem* p, bool correct, bool fused_inject, SolveArgs& a) {
  const tl_config& c = p->cfg;
  Level& L = p->C;
  fill_common(p, L, a);
  a.T_in = L.T;
  a.T_out = correct ? L.T : L.T2;
  a.st_sx = L.g.nx;
  a.st_sy = L.g.ny;
  a.st_ox = 0;
  a.st_oy = 0;
  a.dir.faces = 16;
  if (correct) {
    injection_box(p, a.dir.box);
  } else {
    a.dir.box[0] = 1; a.dir.box[1] = 0; a.dir.box[2] = 1; a.dir.box[3] = 0; a.dir.box[4] = 1; a.dir.box[5] = 0;
  }
  a.dv.kind = (correct && fused_inject) ? 2 : 1;
  a.dv.T_bottom = c.T_bottom;
  a.dv.inj = L.inj;
  a.dv.Tf = p->Fi.T;
  a.dv.fg = p->Fi.g;
  a.dv.cg = L.g;
  a.dv.oi = p->oi;
  a.dv.oj = p->oj;
  a.dv.ok = p->ok;
  a.dv.r = c.r;
  if (c.coarse_source == 1)
    a.ld = gaussian_load(p, L, (p->n + 1) * c.dt_coarse, 0.0, 0.0);
  else
    a.ld = box_load(p, p->n);
  a.dt = c.dt_coarse;
  a.energy = correct ? c.energy : 0;
  a.update_state = correct ? 1 : 0;
  a.level = 0;
  if (correct && c.interface_coupling == 1) {
    // flux-jump coupling: the plate's own boundary conditions and the
    // interface load the restriction step formed (in the injection buffer)
    a.dir.box[0] = 1; a.dir.box[1] = 0; a.dir.box[2] = 1; a.dir.box[3] = 0; a.dir.box[4] = 1; a.dir.box[5] = 0;
    a.dv.kind = 1;
    a.Fx = L.inj;
  }
}

tl_status coarse_solve(tl_problem* p, bool correct) {
  SolveArgs a{};
  build_coarse_args(p, correct, false, a);
  return launch_picard(p, p->C, a);
}

// Arguments of fine micro step i of the current macro step.
void build_fine_args(tl_problem* p, int i, SolveArgs& a) {
  const tl_config& c = p->cfg;
  Level& L = p->Fi;
  fill_common(p, L, a);
  a.T_in = L.T;
  a.T_out = L.T;
  a.st_sx = L.st_sx;
  a.st_sy = L.st_sy;
  a.st_ox = p->oi * c.r;
  a.st_oy = p->oj * c.r;
  a.dir.faces = fine_dir_faces(p);
  a.dir.box[0] = 1; a.dir.box[1] = 0; a.dir.box[2] = 1; a.dir.box[3] = 0; a.dir.box[4] = 1; a.dir.box[5] = 0;
  a.dv.kind = 0;
  a.dv.T_bottom = c.T_bottom;
  a.dv.w = c.bc_weight_literal ? (double)i / c.m : (double)(i + 1) / c.m;
  a.dv.Tc0 = p->C.T;
  a.dv.Tc1 = p->C.T2;
  a.dv.cg = p->C.g;
  a.dv.oi = p->oi;
  a.dv.oj = p->oj;
  a.dv.ok = p->ok;
  a.dv.r = c.r;
  const double dt = c.dt_coarse / c.m;
  const double t = ((double)p->n * c.m + i + 1) * dt;
  a.ld = gaussian_load(p, L, t, p->oi * (c.Lx / c.NXc), p->oj * (c.Ly / c.NYc));
  a.dt = dt;
  a.energy = c.energy;
  a.update_state = 1;
  a.level = 1;
}

tl_status fine_solve(tl_problem* p, int i) {
  SolveArgs a{};
  build_fine_args(p, i, a);
  return launch_picard(p, p->Fi, a);
}

tl_status validate(const tl_config* c) {
  if (!c) return TL_EINVAL;
  if (!(c->Lx > 0 && c->Ly > 0 && c->Lz > 0)) return TL_EINVAL;
  if (c->NXc < 1 || c->NYc < 1 || c->NZc < 1) return TL_EINVAL;
  if (c->pNXc < 1 || c->pNYc < 1 || c->pNZc < 1) return TL_EINVAL;
  if (c->pNXc > c->NXc || c->pNYc > c->NYc || c->pNZc > c->NZc) return TL_EINVAL;
  if (c->r < 1 || c->m < 1 || c->r > 64 || c->m > 1024) return TL_EINVAL;
  if (!(c->dt_coarse > 0)) return TL_EINVAL;
  if (!(c->rho > 0) || !(c->c0 > 0) || !(c->k0 > 0) || !(c->powder_factor > 0)) return TL_EINVAL;
  if (!(c->radius > 0) || !(c->P >= 0) || !(c->eta >= 0)) return TL_EINVAL;
  if (c->ntracks < 0 || (c->ntracks > 0 && !c->path)) return TL_EINVAL;
  if (!(c->tol > 0) || c->max_iter < 1) return TL_EINVAL;
  if (c->precision != TL_FP64 && c->precision != TL_FP32_REFINED) return TL_EINVAL;
  if (c->precision == TL_FP32_REFINED && !(c->tol_inner > 0 && c->tol_inner < 1)) return TL_EINVAL;
  if (c->inner_tiles < 0 || c->inner_tiles > 2) return TL_EINVAL;
  if (c->coupling_sweeps > 1 && !(c->coupling_tol > 0)) return TL_EINVAL;
  if (c->picard_iters < 0 || c->picard_iters > 50) return TL_EINVAL;
  if (c->picard_iters > 1 && c->coupling_sweeps > 1) return TL_EINVAL;
  if (!(c->latent >= 0)) return TL_EINVAL;
  if (c->latent > 0 && (!(c->pc_sharpness > 0) || !(c->T_liquidus >= c->T_solidus))) return TL_EINVAL;
  if (c->precond < 0 || c->precond > 2) return TL_EINVAL;
  if ((c->alloc == nullptr) != (c->free == nullptr)) return TL_EINVAL;
  if (!(c->barrier_timeout >= 0) || c->barrier_timeout > 60.0) return TL_EINVAL;
  if (c->autotune < 0 || c->autotune > 1) return TL_EINVAL;
  if (c->interface_coupling < 0 || c->interface_coupling > 1) return TL_EINVAL;
  if (c->interface_coupling == 1 && c->coupling_sweeps > 1) return TL_EINVAL;
  if (!(c->h_conv >= 0) || !(c->emissivity >= 0) || c->emissivity > 1.0) return TL_EINVAL;
  if ((c->h_conv > 0 || c->emissivity > 0) && !(c->T_amb > 0)) return TL_EINVAL;
  // the surface term rides on the apply of the stored CG direction, which the
  // Jacobi forms (fused update) do not keep
  if ((c->h_conv > 0 || c->emissivity > 0) && c->precond == 1) return TL_EINVAL;
  for (int j = 0; j < c->ntracks; ++j) {
    const tl_track& k = c->path[j];
    if (!(k.speed > 0)) return TL_EINVAL;
    if (k.x0 == k.x1 && k.y0 == k.y1) return TL_EINVAL;
    if (c->coarse_source == 0 && k.x0 != k.x1 && k.y0 != k.y1) return TL_EINVAL;
  }
  if (c->coarse_source != 0 && c->coarse_source != 1) return TL_EINVAL;
  const long long fx = (long long)c->pNXc * c->r, fy = (long long)c->pNYc * c->r, fz = (long long)c->pNZc * c->r;
  // 32-bit node indices with 8 eigenvalues per element and 7 exchange arrays
  if ((fx + 1) * (fy + 1) * (fz + 1) > (1LL << 28)) return TL_EINVAL;
  if ((long long)(c->NXc + 1) * (c->NYc + 1) * (c->NZc + 1) > (1LL << 28)) return TL_EINVAL;
  return TL_OK;
}

void release(tl_problem* p) {
  for (void* ptr : p->allocs) {
    if (p->cfg.free)
      p->cfg.free(ptr, (void*)p->stream, p->cfg.alloc_ctx);
    else
      cudaFree(ptr);
  }
  p->allocs.clear();
}

tl_status launch_fill(tl_problem* p, double* x, size_t n, double v) {
  fill_kernel<<<std::max(1, std::min(1024, (int)((n + 255) / 256))), 256, 0, p->stream>>>(x, (long long)n, v);
  return cuda_status(cudaGetLastError());
}

tl_status move_patch(tl_problem* p) {
  int ni = p->oi, nj = p->oj;
  origin_for(p, p->n, &ni, &nj);
  if (ni == p->oi && nj == p->oj) return TL_OK;
  Level& F = p->Fi;
  const long long nn = (long long)F.g.nnx * F.g.nny * F.g.nnz;
  int blocks = (int)std::min<long long>(4096, (nn + 255) / 256);
  move_patch_kernel<<<blocks, 256, 0, p->stream>>>(F.g, p->C.g, F.T, F.T2, p->C.T, p->oi, p->oj, ni, nj, p->ok,
                                                   p->cfg.r);
  p->launches++;
  tl_status s = cuda_status(cudaGetLastError());
  if (s != TL_OK) return s;
  std::swap(F.T, F.T2);
  p->oi = ni;
  p->oj = nj;
  p->patch_moves++;
  return TL_OK;
}

// Advance p's Algorithm-1 sequence by one solve for a batched launch and fill
// its arguments: one macro step = predictor (patch motion fused into it) + m
// micro steps + corrector (restriction fused into its boundary data).
// *weight gets the solve's element count.
void next_batched_solve(tl_problem* p, SolveArgs& a, long long* weight) {
  const tl_config& c = p->cfg;
  a = SolveArgs{};
  if (p->phase == NEED_PREDICT) {
    int ni = p->oi, nj = p->oj;
    origin_for(p, p->n, &ni, &nj);
    build_coarse_args(p, false, false, a);
    a.t = p->C.tb;
    if (ni != p->oi || nj != p->oj) {
      Level& F = p->Fi;
      a.mv = MoveSpec{1, F.T, F.T2, p->C.T, F.g, p->C.g, p->oi, p->oj, ni, nj, p->ok, c.r};
      std::swap(F.T, F.T2);
      p->oi = ni;
      p->oj = nj;
      p->patch_moves++;
    }
    p->phase = IN_SUBSTEPS;
    p->sub = 0;
    *weight = (long long)p->C.g.nx * p->C.g.ny * p->C.g.nz;
    return;
  }
  if (p->phase == IN_SUBSTEPS && p->sub < c.m) {
    build_fine_args(p, p->sub, a);
    a.t = p->Fi.tb;
    p->sub++;
    *weight = (long long)p->Fi.g.nx * p->Fi.g.ny * p->Fi.g.nz;
    return;
  }
  build_coarse_args(p, true, true, a);
  a.t = p->C.tb;
  p->phase = NEED_PREDICT;
  p->n++;
  *weight = (long long)p->C.g.nx * p->C.g.ny * p->C.g.nz;
}


// Flux-jump coupling: the interface load of the fine field at the end of the
// macro step into the coarse level's `inj` buffer (cleared first).
tl_status launch_interface_load(tl_problem* p) {
  const tl_config& c = p->cfg;
  Level& C = p->C;
  const size_t nc = (size_t)C.g.nnx * C.g.nny * C.g.nnz;
  cudaError_t e = cudaMemsetAsync(C.inj, 0, nc * sizeof(double), p->stream);
  if (e != cudaSuccess) return cuda_status(e);
  IfaceSpec sp{};
  sp.fg = p->Fi.g;
  sp.cg = C.g;
  sp.oi = p->oi;
  sp.oj = p->oj;
  sp.ok = p->ok;
  sp.r = c.r;
  sp.pnx = c.pNXc;
  sp.pny = c.pNYc;
  sp.pnz = c.pNZc;
  const int f = fine_dir_faces(p);
  sp.faces = (f & 15) | (p->ok > 0 ? 16 : 0);
  sp.Tf = p->Fi.T;
  sp.Tc = C.T;
  sp.st_f = p->Fi.state;
  sp.st_sx = p->Fi.st_sx;
  sp.st_sy = p->Fi.st_sy;
  sp.st_c = C.state;
  sp.mat = Material{c.rho, c.c0, c.c1, c.k0, c.k1, c.Tref, c.powder_factor, c.T_melt,
                    c.latent, c.pc_sharpness, 0.5 * (c.T_solidus + c.T_liquidus)};
  sp.G = C.inj;
  const long long nb = (long long)(c.pNXc + 1) * (c.pNYc + 1) * (c.NZc - p->ok + 1);
  interface_load_kernel<<<(int)std::min<long long>(1024, (nb + 127) / 128), 128, 0, p->stream>>>(sp);
  p->launches++;
  return cuda_status(cudaGetLastError());
}

// Injection of the fine field at the coarse nodes that coincide with free
// fine nodes (into the coarse level's `inj`).
tl_status launch_restrict(tl_problem* p) {
  int box[6];
  injection_box(p, box);
  if (box[0] <= box[1] && box[2] <= box[3] && box[4] <= box[5]) {
    long long nb = (long long)(box[1] - box[0] + 1) * (box[3] - box[2] + 1) * (box[5] - box[4] + 1);
    int blocks = (int)std::min<long long>(1024, (nb + 255) / 256);
    restrict_kernel<<<blocks, 256, 0, p->stream>>>(p->Fi.g, p->C.g, p->Fi.T, p->C.inj, box[0], box[1], box[2],
                                                   box[3], box[4], box[5], p->oi, p->oj, p->ok, p->cfg.r);
    p->launches++;
    return cuda_status(cudaGetLastError());
  }
  return TL_OK;
}

// The fine element states of the patch window <-> the compact snapshot
// (a fine solve changes no other entry of the plate-wide map).
tl_status copy_state_window(tl_problem* p, bool save) {
  Level& F = p->Fi;
  const size_t ox = (size_t)p->oi * p->cfg.r, oy = (size_t)p->oj * p->cfg.r;
  for (int k = 0; k < F.g.nz; ++k) {
    uint8_t* win = F.state + (size_t)F.st_sx * F.st_sy * k + oy * F.st_sx + ox;
    uint8_t* cmp = F.state_snap + (size_t)F.g.nx * F.g.ny * k;
    cudaError_t e = save ? cudaMemcpy2DAsync(cmp, (size_t)F.g.nx, win, (size_t)F.st_sx, (size_t)F.g.nx,
                                             (size_t)F.g.ny, cudaMemcpyDeviceToDevice, p->stream)
                         : cudaMemcpy2DAsync(win, (size_t)F.st_sx, cmp, (size_t)F.g.nx, (size_t)F.g.nx,
                                             (size_t)F.g.ny, cudaMemcpyDeviceToDevice, p->stream);
    if (e != cudaSuccess) return cuda_status(e);
  }
  return TL_OK;
}

// Iterated coupling: the start of the last micro step (fine field into the
// move buffer T2, which is free between patch moves; states of the window).
tl_status save_last_start(tl_problem* p) {
  Level& F = p->Fi;
  const size_t nf = (size_t)F.g.nnx * F.g.nny * F.g.nnz;
  cudaError_t e = cudaMemcpyAsync(F.T2, F.T, nf * sizeof(double), cudaMemcpyDeviceToDevice, p->stream);
  if (e != cudaSuccess) return cuda_status(e);
  return copy_state_window(p, true);
}

// The correction step with the iterated coupling: correction into T3; then,
// while sweeps remain and the corrected field still moves by more than
// coupling_tol of its size, the last micro step again from its start with the
// corrected field as its end data, injection, and the correction again from
// T+^n with the coarse states of t_n.  Superseded solves leave the energy
// account.  The final corrected field becomes T+^{n+1}.  After a failed
// solve (sticky device status) the coarse field is left at T+^n.
tl_status coupled_correct(tl_problem* p) {
  const tl_config& c = p->cfg;
  Level& C = p->C;
  Level& F = p->Fi;
  const size_t nc = (size_t)C.g.nnx * C.g.nny * C.g.nnz, ec = (size_t)C.g.nx * C.g.ny * C.g.nz;
  const size_t nf = (size_t)F.g.nnx * F.g.nny * F.g.nnz;
  cudaError_t e = cudaMemcpyAsync(C.state_snap, C.state, ec, cudaMemcpyDeviceToDevice, p->stream);
  if (e != cudaSuccess) return cuda_status(e);
  double* cur = C.T3;
  double* prev = C.T3b;
  SolveArgs a{};
  build_coarse_args(p, true, false, a);
  a.T_out = cur;
  tl_status s = launch_solve(p, C, a);
  if (s != TL_OK) return s;
  int st = 0;
  for (int k = 1; k < c.coupling_sweeps; ++k) {
    if ((s = copy_state_window(p, false)) != TL_OK) return s;
    e = cudaMemcpyAsync(F.T, F.T2, nf * sizeof(double), cudaMemcpyDeviceToDevice, p->stream);
    if (e != cudaSuccess) return cuda_status(e);
    if (c.energy) {
      energy_rollback_kernel<<<1, 32, 0, p->stream>>>(p->stats, 1);
      p->launches++;
    }
    SolveArgs af{};
    build_fine_args(p, c.m - 1, af);
    af.dv.Tc1 = cur;
    if ((s = launch_solve(p, F, af)) != TL_OK) return s;
    if ((s = launch_restrict(p)) != TL_OK) return s;
    e = cudaMemcpyAsync(C.state, C.state_snap, ec, cudaMemcpyDeviceToDevice, p->stream);
    if (e != cudaSuccess) return cuda_status(e);
    if (c.energy) {
      energy_rollback_kernel<<<1, 32, 0, p->stream>>>(p->stats, 0);
      p->launches++;
    }
    SolveArgs ac{};
    build_coarse_args(p, true, false, ac);
    ac.T_out = prev;
    if ((s = launch_solve(p, C, ac)) != TL_OK) return s;
    std::swap(cur, prev);
    p->coupling_resolves++;
    e = cudaMemsetAsync(p->d_diff, 0, 2 * sizeof(unsigned long long), p->stream);
    if (e != cudaSuccess) return cuda_status(e);
    const int blocks = (int)std::min<size_t>(1024, (nc + 255) / 256);
    max_diff_kernel<<<blocks, 256, 0, p->stream>>>(cur, prev, (long long)nc, p->d_diff);
    p->launches++;
    unsigned long long h[2] = {0, 0};
    e = cudaMemcpyAsync(h, p->d_diff, sizeof h, cudaMemcpyDeviceToHost, p->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&st, p->status, sizeof st, cudaMemcpyDeviceToHost, p->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
    if (e != cudaSuccess) return cuda_status(e);
    if (st != 0) return TL_OK;  // reported by tl_sync; T+^n kept
    double d, m;
    std::memcpy(&d, &h[0], sizeof d);
    std::memcpy(&m, &h[1], sizeof m);
    if (d <= c.coupling_tol * m) break;
  }
  e = cudaMemcpyAsync(C.T, cur, nc * sizeof(double), cudaMemcpyDeviceToDevice, p->stream);
  return cuda_status(e);
}

// ---- the tiling autotuner -------------------------------------------------
// Tilings only decide how the blocks of a solve walk the mesh; which one is
// fastest depends on the mesh, the grid and the GPU in ways the cost models
// above only approximate.  For a level of at least AUTOTUNE_MIN_NODES nodes the
// tuner times dry solves (the level's first solve as it will run, committing
// nothing but a scratch output, on separate barrier and status words) of a few
// candidates per tiling, one tiling at a time: the preconditioner pass's
// z-depth (the model's, half, one and a half and twice it), then on the
// refined path the inner tile family (wide or element tiles, unless
// inner_tiles forces one), then the wide tiles' depth (nz / 16 ... nz / 4) or
// the element tile shape (the cost model's three cheapest shapes), keeping
// the fastest of each (the best of two timed runs after one warm-up).  Picks are cached per mesh shape,
// precision, preconditioner and grid cap for the life of the process.
constexpr long long AUTOTUNE_MIN_NODES = 65536;

struct TuneKey {
  int nx, ny, nz, prec, precond, wide, grid_cap, fine;
  bool operator<(const TuneKey& o) const {
    return std::tie(nx, ny, nz, prec, precond, wide, grid_cap, fine) <
           std::tie(o.nx, o.ny, o.nz, o.prec, o.precond, o.wide, o.grid_cap, o.fine);
  }
};
struct TunePick {
  Tiling t, tw, tp;
  int grid, wide;
};
std::mutex g_tune_mutex;
std::map<TuneKey, TunePick> g_tune_cache;

// Dry-run arguments of the level's first solve: a fine micro step (output
// into the move buffer) or a coarse predictor (its output is the predictor
// buffer, rewritten by the first real predictor).
void dry_args(tl_problem* p, Level& L, bool fine, SolveArgs& a) {
  if (fine) {
    build_fine_args(p, 0, a);
    a.T_out = L.T2;
  } else {
    build_coarse_args(p, false, false, a);
  }
  a.update_state = 0;
  a.energy = 0;
  a.dry = 1;
  a.trace = nullptr;
  a.bar = Barrier{reinterpret_cast<unsigned long long*>(p->tune_bar), (int*)(p->tune_bar + BAR_STATUS),
                  barrier_limit_ns(p->cfg)};
}

// Best of `reps` timed dry solves after one warm-up, in ms; < 0 on a failed
// run (then the tuner keeps the models' picks).
float time_dry(tl_problem* p, Level& L, bool fine, cudaEvent_t e0, cudaEvent_t e1, int reps = 2) {
  float best = -1.0f;
  for (int k = 0; k <= reps; ++k) {
    SolveArgs a{};
    dry_args(p, L, fine, a);
    if (cudaMemsetAsync(p->tune_bar, 0, BAR_WORDS * sizeof(unsigned int), p->stream) != cudaSuccess) return -1.0f;
    cudaEventRecord(e0, p->stream);
    void* args[] = {(void*)&a};
    cudaError_t e = cudaLaunchCooperativeKernel(solve_kernel_for(pmode_of(p->cfg)), dim3(L.grid), dim3(NT), args,
                                                STAGE_BYTES, p->stream);
    cudaEventRecord(e1, p->stream);
    int st = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&st, p->tune_bar + BAR_STATUS, sizeof st, cudaMemcpyDeviceToHost, p->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return -1.0f;
    }
    if (st != 0) return -1.0f;
    if (k > 0 && (best < 0 || ms < best)) best = ms;
  }
  return best;
}

tl_status autotune_level(tl_problem* p, Level& L, bool fine) {
  const long long nn = (long long)L.g.nnx * L.g.nny * L.g.nnz;
  if (nn < AUTOTUNE_MIN_NODES) return TL_OK;
  const tl_config& c = p->cfg;
  const TuneKey key{L.g.nx, L.g.ny, L.g.nz, (int)c.precision, c.precond == 1 ? 1 : 0, L.wide, p->max_coop,
                    fine ? 1 : 0};
  {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      L.t = it->second.t;
      L.tw = it->second.tw;
      L.tp = it->second.tp;
      L.grid = it->second.grid;
      L.wide = it->second.wide;
      L.tuned = 1;
      return TL_OK;
    }
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    cudaGetLastError();
    if (e0) cudaEventDestroy(e0);
    return TL_ECUDA;
  }
  bool ok = true;
  float best = time_dry(p, L, fine, e0, e1);
  ok = best >= 0;
  // 1. the preconditioner pass's z-depth (tensor preconditioner only)
  if (ok && c.precond != 1) {
    const Tiling t0 = L.tp;
    // half, one and a half and twice the model's depth
    const int cands[3] = {t0.ez / 2, (3 * t0.ez + 1) / 2, 2 * t0.ez};
    Tiling win = t0;
    for (int ez0 : cands) {
      const int ez = std::min(L.g.nnz, std::max(2, ez0));
      if (ez == win.ez || ez == t0.ez) continue;
      L.tp = Tiling{t0.ex, t0.ey, ez, t0.ntx, t0.nty, (L.g.nnz + ez - 1) / ez};
      const float ms = time_dry(p, L, fine, e0, e1);
      if (ms >= 0 && ms < best) {
        best = ms;
        win = L.tp;
      }
    }
    L.tp = win;
  }
  // 2. the refined path's inner tile family: wide tiles where the size rule
  // chose element tiles, and the other way round (not when inner_tiles forces one)
  if (ok && c.precision == TL_FP32_REFINED && c.inner_tiles == 0) {
    const int w0 = L.wide;
    const Tiling tw0 = L.tw;
    L.wide = !w0;
    if (L.wide) L.tw = wide_tiling(L.g, L.grid);
    const float ms = time_dry(p, L, fine, e0, e1);
    if (ms >= 0 && ms < best) {
      best = ms;
    } else {
      L.wide = w0;
      L.tw = tw0;
    }
  }
  // 3. the wide tiles' depth, or the element tile shape
  if (ok && L.wide) {
    const Tiling t0 = L.tw;
    Tiling win = t0;
    for (int div : {16, 12, 6, 4}) {
      const int ez = std::max(1, (L.g.nz + div / 2) / div);
      if (ez == win.ez || ez == t0.ez) continue;
      L.tw = Tiling{AX, AY, ez, t0.ntx, t0.nty, (L.g.nz + ez - 1) / ez};
      const float ms = time_dry(p, L, fine, e0, e1);
      if (ms >= 0 && ms < best) {
        best = ms;
        win = L.tw;
      }
    }
    L.tw = win;
  } else if (ok) {
    std::vector<Tiling> ranked;
    Level tmp = L;
    int per_sm = std::max(1, p->max_coop / std::max(1, p->nsm));
    choose_tiling(tmp, p->nsm, per_sm, &ranked);
    const Tiling t0 = L.t;
    const int g0 = L.grid;
    Tiling win = t0;
    int wgrid = g0;
    for (size_t k = 0; k < ranked.size() && k < 3; ++k) {
      const Tiling& t = ranked[k];
      if (t.ex == t0.ex && t.ey == t0.ey && t.ez == t0.ez) continue;
      L.t = t;
      L.grid = std::min(p->max_coop, t.ntx * t.nty * t.ntz);
      const float ms = time_dry(p, L, fine, e0, e1);
      if (ms >= 0 && ms < best) {
        best = ms;
        win = t;
        wgrid = L.grid;
      }
    }
    L.t = win;
    L.grid = wgrid;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (!ok) return TL_OK;  // a failed timing run: the models' picks stay
  L.tuned = 1;
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  g_tune_cache[key] = TunePick{L.t, L.tw, L.tp, L.grid, L.wide};
  return TL_OK;
}

}  // namespace

struct tl_batch {
  struct Job {
    tl_problem* p;
    long long target;          // macro steps to reach
    cudaStream_t saved_stream;
    bool active;
  };
  cudaStream_t stream = nullptr;
  int R = 0;                   // cooperative launches per round
  int cap = 0;                 // jobs per launch at most (one block each at least)
  int max_coop = 0, nsm = 0;    // co-resident blocks of the slowest-to-fit kernel variant
  int max_coop_v[3] = {0, 0, 0}; // ... of each precision mode's batch kernel
  std::vector<Job> jobs;
  std::vector<int> finished;   // ids that reached their target, not yet polled
  BatchTable* d_tab = nullptr; // R tables
  SolveArgs* d_args = nullptr; // R x cap job arguments
  BatchTable* h_tab = nullptr; // pinned staging of the same
  SolveArgs* h_args = nullptr;
  int* d_st = nullptr;         // per launch slot: the job's status word at the end of the round
  int* h_st = nullptr;         // pinned copy
  std::vector<int> round_ids;  // job id of each launch slot of the last round
  long long launches = 0, rounds = 0;
};

extern "C" {

const char* tl_status_string(tl_status s) {
  switch (s) {
    case TL_OK: return "ok";
    case TL_EINVAL: return "invalid argument";
    case TL_ENOMEM: return "device allocation failed";
    case TL_ENOCONV: return "CG did not converge within max_iter";
    case TL_ESTATE: return "call out of order";
    case TL_ECUDA: return "CUDA runtime error";
    case TL_ETIMEOUT: return "device barrier timed out";
  }
  return "unknown status";
}

tl_status tl_create_problem(const tl_config* cfg, tl_problem** out) {
  if (!out) return TL_EINVAL;
  *out = nullptr;
  tl_status s = validate(cfg);
  if (s != TL_OK) return s;
  tl_problem* p = new (std::nothrow) tl_problem();
  if (!p) return TL_ENOMEM;
  p->cfg = *cfg;
  p->tracks.assign(cfg->path, cfg->path + cfg->ntracks);
  p->cfg.path = nullptr;
  double t = 0.0;
  for (const tl_track& k : p->tracks) {
    double d = std::hypot(k.x1 - k.x0, k.y1 - k.y0) / k.speed;
    p->t_start.push_back(t);
    p->dur.push_back(d);
    t = t + d;
    p->t_end.push_back(t);
  }
  p->stream = (cudaStream_t)cfg->stream;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&p->nsm, cudaDevAttrMultiProcessorCount, dev);
  int per_sm = 0;
  const void* kern = solve_kernel_for(pmode_of(*cfg));
  if (e == cudaSuccess) e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, STAGE_BYTES);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, STAGE_BYTES);
  if (e != cudaSuccess || per_sm < 1) {
    delete p;
    cudaGetLastError();
    return TL_ECUDA;
  }
  p->max_coop = std::min(per_sm * p->nsm, MAX_GRID_BLOCKS);
  const tl_config& c = p->cfg;
  const int r = c.r;
  // coarse level
  Level& C = p->C;
  C.g = Grid3{c.NXc, c.NYc, c.NZc, c.NXc + 1, c.NYc + 1, c.NZc + 1, c.Lx / c.NXc, c.Ly / c.NYc, c.Lz / c.NZc};
  C.st_sx = c.NXc; C.st_sy = c.NYc; C.st_sz = c.NZc;
  // fine patch; its states live in a plate-wide map over the patch depth
  Level& F = p->Fi;
  F.g = Grid3{c.pNXc * r, c.pNYc * r, c.pNZc * r, c.pNXc * r + 1, c.pNYc * r + 1, c.pNZc * r + 1,
              C.g.hx / r, C.g.hy / r, C.g.hz / r};
  F.st_sx = c.NXc * r; F.st_sy = c.NYc * r; F.st_sz = c.pNZc * r;
  element_constants(C);
  element_constants(F);
  choose_tiling(C, p->nsm, per_sm);
  choose_tiling(F, p->nsm, per_sm);
  C.grid = std::min(p->max_coop, C.t.ntx * C.t.nty * C.t.ntz);
  F.grid = std::min(p->max_coop, F.t.ntx * F.t.nty * F.t.ntz);
  p->red_stride = p->max_coop;
  p->max_slice = std::max(C.grid, F.grid);
  for (Level* L : {&C, &F}) {
    L->wide = use_wide(c, L->g, L->grid);
    if (L->wide) L->tw = wide_tiling(L->g, L->grid);
    L->tp = pc_tiling(L->g, L->grid);
  }
  if ((s = alloc_level(p, C, true)) != TL_OK || (s = alloc_level(p, F, false)) != TL_OK ||
      (s = alloc_n(p, &p->bar, BAR_WORDS)) != TL_OK ||
      (s = alloc_n(p, &p->red, (size_t)RS_N * p->red_stride)) != TL_OK ||
      (s = alloc_n(p, &p->red32, (size_t)RS_N * p->red_stride)) != TL_OK ||
      (s = alloc_n(p, &p->stats, 1)) != TL_OK || (s = alloc_n(p, &p->d_diff, 2)) != TL_OK ||
      (s = alloc_n(p, &p->tune_bar, BAR_WORDS)) != TL_OK) {
    release(p);
    delete p;
    return s;
  }
  p->status = (int*)(p->bar + BAR_STATUS);
  p->ok = c.NZc - c.pNZc;
  p->oi = 0;
  p->oj = 0;
  {
    // laser position at Dt/2, or the plate centre when the laser is off then
    double x = 0.5 * c.Lx, y = 0.5 * c.Ly;
    laser_at(p, 0.5 * c.dt_coarse, &x, &y);
    origin_at(p, x, y, &p->oi, &p->oj);
  }
  const size_t ncn = (size_t)C.g.nnx * C.g.nny * C.g.nnz, nfn = (size_t)F.g.nnx * F.g.nny * F.g.nnz;
  const int nb = 256;
  if ((s = launch_fill(p, C.T, ncn, c.T0)) != TL_OK || (s = launch_fill(p, C.T2, ncn, c.T0)) != TL_OK ||
      (s = launch_fill(p, F.T, nfn, c.T0)) != TL_OK || (s = launch_fill(p, C.inj, ncn, c.T0)) != TL_OK) {
    release(p);
    delete p;
    return s;
  }
  // buffers read before being written in a solve start at zero
  for (Level* L : {&C, &F}) {
    size_t nn = (size_t)L->g.nnx * L->g.nny * L->g.nnz;
    cudaMemsetAsync(L->X, 0, (size_t)xplane((int)nn) * NXB * sizeof(double), p->stream);
  }
  cudaMemsetAsync(p->bar, 0, BAR_WORDS * sizeof(unsigned int), p->stream);
  cudaMemsetAsync(C.trace, 0, 2 * TRACE_CAP * sizeof(unsigned long long), p->stream);
  cudaMemsetAsync(F.trace, 0, 2 * TRACE_CAP * sizeof(unsigned long long), p->stream);
  cudaMemsetAsync(p->stats, 0, sizeof(DevStats), p->stream);
  init_state_kernel<<<256, nb, 0, p->stream>>>(C.state, C.st_sx, C.st_sy, C.st_sz, 0.0, C.g.hz, c.Lz,
                                               c.powder_depth);
  init_state_kernel<<<1024, nb, 0, p->stream>>>(F.state, F.st_sx, F.st_sy, F.st_sz, p->ok * C.g.hz, F.g.hz, c.Lz,
                                                c.powder_depth);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
  if (e != cudaSuccess) {
    s = cuda_status(e);
    release(p);
    delete p;
    return s;
  }
  if (c.autotune) {
    for (Level* L : {&F, &C}) {
      if ((s = autotune_level(p, *L, L == &F)) != TL_OK) {
        release(p);
        delete p;
        return s;
      }
    }
    p->max_slice = std::max(C.grid, F.grid);
  }
  *out = p;
  return TL_OK;
}

tl_status tl_coarse_step(tl_problem* p, tl_phase phase) {
  if (!p) return TL_EINVAL;
  if (phase == TL_PREDICT) {
    if (p->phase != NEED_PREDICT) return TL_ESTATE;
    tl_status s = move_patch(p);
    if (s != TL_OK) return s;
    s = coarse_solve(p, false);
    if (s != TL_OK) return s;
    p->phase = IN_SUBSTEPS;
    p->sub = 0;
    return TL_OK;
  }
  if (phase == TL_CORRECT) {
    if (p->phase != NEED_CORRECT) return TL_ESTATE;
    tl_status s = p->cfg.coupling_sweeps > 1 ? coupled_correct(p) : coarse_solve(p, true);
    if (s != TL_OK) return s;
    p->phase = NEED_PREDICT;
    p->n++;
    return TL_OK;
  }
  return TL_EINVAL;
}

tl_status tl_fine_substeps(tl_problem* p, int nsub) {
  if (!p || nsub < 0) return TL_EINVAL;
  if (p->phase != IN_SUBSTEPS || p->sub + nsub > p->cfg.m) return TL_ESTATE;
  for (int k = 0; k < nsub; ++k) {
    if (p->cfg.coupling_sweeps > 1 && p->sub == p->cfg.m - 1) {
      tl_status s = save_last_start(p);
      if (s != TL_OK) return s;
    }
    tl_status s = fine_solve(p, p->sub);
    if (s != TL_OK) return s;
    p->sub++;
  }
  return TL_OK;
}

tl_status tl_restrict(tl_problem* p) {
  if (!p) return TL_EINVAL;
  if (p->phase != IN_SUBSTEPS || p->sub != p->cfg.m) return TL_ESTATE;
  tl_status s = p->cfg.interface_coupling == 1 ? launch_interface_load(p) : launch_restrict(p);
  if (s != TL_OK) return s;
  p->phase = NEED_CORRECT;
  return TL_OK;
}

tl_status tl_sync(tl_problem* p) {
  if (!p) return TL_EINVAL;
  cudaError_t e = cudaStreamSynchronize(p->stream);
  if (e != cudaSuccess) return cuda_status(e);
  int st = 0;
  e = cudaMemcpy(&st, p->status, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_status(e);
  return (tl_status)st;
}

tl_status tl_macro_steps(tl_problem* p, int nmacro) {
  if (!p || nmacro < 0) return TL_EINVAL;
  for (int k = 0; k < nmacro; ++k) {
    tl_status s;
    if ((s = tl_coarse_step(p, TL_PREDICT)) != TL_OK) return s;
    if ((s = tl_fine_substeps(p, p->cfg.m)) != TL_OK) return s;
    if ((s = tl_restrict(p)) != TL_OK) return s;
    if ((s = tl_coarse_step(p, TL_CORRECT)) != TL_OK) return s;
  }
  return tl_sync(p);
}

size_t tl_node_count(const tl_problem* p, tl_level level) {
  if (!p) return 0;
  const Level& L = level == TL_COARSE ? p->C : p->Fi;
  if (level != TL_COARSE && level != TL_FINE) return 0;
  return (size_t)L.g.nnx * L.g.nny * L.g.nnz;
}

tl_status tl_get_temperature(const tl_problem* p, tl_level level, double* host_out, size_t n, int origin_out[3]) {
  if (!p || !host_out || (level != TL_COARSE && level != TL_FINE)) return TL_EINVAL;
  if (n != tl_node_count(p, level)) return TL_EINVAL;
  const Level& L = level == TL_COARSE ? p->C : p->Fi;
  cudaError_t e = cudaStreamSynchronize(p->stream);
  if (e == cudaSuccess) e = cudaMemcpy(host_out, L.T, n * sizeof(double), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_status(e);
  if (origin_out) {
    origin_out[0] = p->oi;
    origin_out[1] = p->oj;
    origin_out[2] = p->ok;
  }
  return TL_OK;
}

tl_status tl_get_state(const tl_problem* p, tl_level level, uint8_t* host_out, size_t n) {
  if (!p || !host_out) return TL_EINVAL;
  cudaError_t e = cudaStreamSynchronize(p->stream);
  if (e != cudaSuccess) return cuda_status(e);
  if (level == TL_COARSE) {
    const Level& C = p->C;
    if (n != (size_t)C.g.nx * C.g.ny * C.g.nz) return TL_EINVAL;
    e = cudaMemcpy(host_out, C.state, n, cudaMemcpyDeviceToHost);
    return cuda_status(e);
  }
  if (level != TL_FINE) return TL_EINVAL;
  const Level& F = p->Fi;
  if (n != (size_t)F.g.nx * F.g.ny * F.g.nz) return TL_EINVAL;
  // gather the patch window of the plate-wide map, one row at a time
  const size_t ox = (size_t)p->oi * p->cfg.r, oy = (size_t)p->oj * p->cfg.r;
  for (int k = 0; k < F.g.nz; ++k) {
    const size_t plane = (size_t)F.st_sx * F.st_sy * k;
    e = cudaMemcpy2D(host_out + (size_t)F.g.nx * F.g.ny * k, (size_t)F.g.nx, F.state + plane + oy * F.st_sx + ox,
                     (size_t)F.st_sx, (size_t)F.g.nx, (size_t)F.g.ny, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_status(e);
  }
  return TL_OK;
}

// Checkpoint layout: header, coarse T, fine T (doubles), the device counters,
// coarse states, plate-wide fine state map (bytes).
struct CkptHeader {
  uint64_t magic;
  uint32_t version, stats_bytes;
  int32_t dims[12];   // NXc NYc NZc, fine nx ny nz, map sx sy sz, r, m, precision
  int32_t n, oi, oj, ok;
  int64_t patch_moves, coupling_resolves;
  uint64_t cfg_hash;  // config_hash: every value that fixes the results, the scan path, the build
};
constexpr uint64_t CKPT_MAGIC = 0x746c636b70743031ull;  // "tlckpt01"
constexpr uint32_t CKPT_VERSION = 2;

// 64-bit FNV-1a over the values of the configuration that fix a run's results
// (geometry, material, process, solver and coupling settings, the tracks) and
// an identifier of this library build; the stream, the allocator and the
// barrier time limit are left out.
static uint64_t config_hash(const tl_problem* p) {
  uint64_t h = 1469598103934665603ull;
  auto add = [&](const void* v, size_t n) {
    const unsigned char* b = static_cast<const unsigned char*>(v);
    for (size_t i = 0; i < n; ++i) {
      h ^= b[i];
      h *= 1099511628211ull;
    }
  };
  const tl_config& c = p->cfg;
  const double d[] = {c.Lx, c.Ly, c.Lz, c.dt_coarse, c.T0, c.T_bottom, c.rho, c.c0, c.c1, c.k0, c.k1, c.Tref,
                      c.powder_depth, c.powder_factor, c.T_melt, c.P, c.eta, c.radius, c.tol, c.tol_inner,
                      c.coupling_tol, c.latent, c.T_solidus, c.T_liquidus, c.pc_sharpness, c.h_conv,
                      c.emissivity, c.T_amb};
  const int32_t i[] = {c.NXc, c.NYc, c.NZc, c.pNXc, c.pNYc, c.pNZc, c.r, c.m, c.coarse_source,
                       c.bc_weight_literal, c.energy, (int32_t)c.precision, c.max_iter, c.inner_tiles,
                       c.coupling_sweeps, c.precond, c.picard_iters, c.autotune, c.interface_coupling,
                       (int32_t)p->tracks.size()};
  add(d, sizeof d);
  add(i, sizeof i);
  for (const tl_track& k : p->tracks) {
    const double t[5] = {k.x0, k.y0, k.x1, k.y1, k.speed};
    add(t, sizeof t);
  }
  static const char build[] = __DATE__ " " __TIME__;
  const uint64_t sizes[2] = {sizeof(SolveArgs), sizeof(DevStats)};
  add(build, sizeof build - 1);
  add(sizes, sizeof sizes);
  return h;
}

static void ckpt_dims(const tl_problem* p, int32_t (&d)[12]) {
  const Level &C = p->C, &F = p->Fi;
  const int32_t v[12] = {C.g.nx, C.g.ny, C.g.nz, F.g.nx, F.g.ny, F.g.nz, F.st_sx, F.st_sy, F.st_sz,
                         p->cfg.r, p->cfg.m, (int32_t)p->cfg.precision};
  for (int i = 0; i < 12; ++i) d[i] = v[i];
}

static size_t ckpt_bytes(const tl_problem* p) {
  const Level &C = p->C, &F = p->Fi;
  const size_t nc = (size_t)C.g.nnx * C.g.nny * C.g.nnz, nf = (size_t)F.g.nnx * F.g.nny * F.g.nnz;
  const size_t ec = (size_t)C.g.nx * C.g.ny * C.g.nz, sm = (size_t)F.st_sx * F.st_sy * F.st_sz;
  return sizeof(CkptHeader) + (nc + nf) * sizeof(double) + sizeof(DevStats) + ec + sm;
}

static tl_status ckpt_ready(const tl_problem* p) {
  if (p->phase != NEED_PREDICT) return TL_ESTATE;
  cudaError_t e = cudaStreamSynchronize(p->stream);
  if (e != cudaSuccess) return cuda_status(e);
  int st = 0;
  e = cudaMemcpy(&st, p->status, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_status(e);
  return st == 0 ? TL_OK : TL_ESTATE;
}

tl_status tl_checkpoint_size(const tl_problem* p, size_t* bytes) {
  if (!p || !bytes) return TL_EINVAL;
  *bytes = ckpt_bytes(p);
  return TL_OK;
}

tl_status tl_checkpoint_save(const tl_problem* p, void* host_out, size_t bytes) {
  if (!p || !host_out || bytes != ckpt_bytes(p)) return TL_EINVAL;
  tl_status s = ckpt_ready(p);
  if (s != TL_OK) return s;
  const Level &C = p->C, &F = p->Fi;
  const size_t nc = (size_t)C.g.nnx * C.g.nny * C.g.nnz, nf = (size_t)F.g.nnx * F.g.nny * F.g.nnz;
  const size_t ec = (size_t)C.g.nx * C.g.ny * C.g.nz, sm = (size_t)F.st_sx * F.st_sy * F.st_sz;
  unsigned char* b = static_cast<unsigned char*>(host_out);
  CkptHeader h{};
  h.magic = CKPT_MAGIC;
  h.version = CKPT_VERSION;
  h.cfg_hash = config_hash(p);
  h.stats_bytes = (uint32_t)sizeof(DevStats);
  ckpt_dims(p, h.dims);
  h.n = p->n;
  h.oi = p->oi;
  h.oj = p->oj;
  h.ok = p->ok;
  h.patch_moves = p->patch_moves;
  h.coupling_resolves = p->coupling_resolves;
  std::memcpy(b, &h, sizeof h);
  b += sizeof h;
  cudaError_t e = cudaMemcpy(b, C.T, nc * sizeof(double), cudaMemcpyDeviceToHost);
  b += nc * sizeof(double);
  if (e == cudaSuccess) e = cudaMemcpy(b, F.T, nf * sizeof(double), cudaMemcpyDeviceToHost);
  b += nf * sizeof(double);
  if (e == cudaSuccess) e = cudaMemcpy(b, p->stats, sizeof(DevStats), cudaMemcpyDeviceToHost);
  b += sizeof(DevStats);
  if (e == cudaSuccess) e = cudaMemcpy(b, C.state, ec, cudaMemcpyDeviceToHost);
  b += ec;
  if (e == cudaSuccess) e = cudaMemcpy(b, F.state, sm, cudaMemcpyDeviceToHost);
  return cuda_status(e);
}

tl_status tl_checkpoint_load(tl_problem* p, const void* host_in, size_t bytes) {
  if (!p || !host_in || bytes != ckpt_bytes(p)) return TL_EINVAL;
  CkptHeader h;
  std::memcpy(&h, host_in, sizeof h);
  int32_t d[12];
  ckpt_dims(p, d);
  if (h.magic != CKPT_MAGIC || h.version != CKPT_VERSION || h.stats_bytes != sizeof(DevStats) ||
      std::memcmp(d, h.dims, sizeof d) != 0 || h.cfg_hash != config_hash(p))
    return TL_EINVAL;
  if (h.n < 0 || h.oi < 0 || h.oj < 0 || h.oi + p->cfg.pNXc > p->cfg.NXc || h.oj + p->cfg.pNYc > p->cfg.NYc ||
      h.ok != p->ok)
    return TL_EINVAL;
  tl_status s = ckpt_ready(p);
  if (s != TL_OK) return s;
  const Level &C = p->C, &F = p->Fi;
  const size_t nc = (size_t)C.g.nnx * C.g.nny * C.g.nnz, nf = (size_t)F.g.nnx * F.g.nny * F.g.nnz;
  const size_t ec = (size_t)C.g.nx * C.g.ny * C.g.nz, sm = (size_t)F.st_sx * F.st_sy * F.st_sz;
  const unsigned char* b = static_cast<const unsigned char*>(host_in) + sizeof h;
  cudaError_t e = cudaMemcpy(C.T, b, nc * sizeof(double), cudaMemcpyHostToDevice);
  b += nc * sizeof(double);
  if (e == cudaSuccess) e = cudaMemcpy(F.T, b, nf * sizeof(double), cudaMemcpyHostToDevice);
  b += nf * sizeof(double);
  if (e == cudaSuccess) e = cudaMemcpy(p->stats, b, sizeof(DevStats), cudaMemcpyHostToDevice);
  b += sizeof(DevStats);
  if (e == cudaSuccess) e = cudaMemcpy(C.state, b, ec, cudaMemcpyHostToDevice);
  b += ec;
  if (e == cudaSuccess) e = cudaMemcpy(F.state, b, sm, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_status(e);
  p->n = h.n;
  p->oi = h.oi;
  p->oj = h.oj;
  p->patch_moves = h.patch_moves;
  p->coupling_resolves = h.coupling_resolves;
  p->sub = 0;
  p->phase = NEED_PREDICT;
  return TL_OK;
}

tl_status tl_get_stats(const tl_problem* p, tl_stats* out) {
  if (!p || !out) return TL_EINVAL;
  DevStats d{};
  cudaError_t e = cudaStreamSynchronize(p->stream);
  if (e == cudaSuccess) e = cudaMemcpy(&d, p->stats, sizeof d, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_status(e);
  std::memset(out, 0, sizeof *out);
  out->macro_steps = p->n;
  out->substeps = (int64_t)p->n * p->cfg.m + (p->phase == IN_SUBSTEPS || p->phase == NEED_CORRECT ? p->sub : 0);
  out->cg_iters_coarse = d.iters[0];
  out->cg_iters_fine = d.iters[1];
  out->outer_iters_coarse = d.outer[0];
  out->outer_iters_fine = d.outer[1];
  out->solves_coarse = d.solves[0];
  out->solves_fine = d.solves[1];
  out->max_iters_coarse = d.max_iters[0];
  out->max_iters_fine = d.max_iters[1];
  out->origin[0] = p->oi;
  out->origin[1] = p->oj;
  out->origin[2] = p->ok;
  out->patch_moves = p->patch_moves;
  out->launches = p->launches;
  out->energy_coarse_stored = d.e_stored[0];
  out->energy_coarse_laser = d.e_laser[0];
  out->energy_coarse_flux = d.e_flux[0];
  out->energy_fine_stored = d.e_stored[1];
  out->energy_fine_laser = d.e_laser[1];
  out->energy_fine_flux = d.e_flux[1];
  out->energy_fine_loss = d.e_loss[1];
  out->energy_coarse_loss = d.e_loss[0];
  out->time = p->n * p->cfg.dt_coarse;
  out->coupling_resolves = p->coupling_resolves;
  return TL_OK;
}

tl_status tl_get_tiling(const tl_problem* p, tl_level level, int32_t out[11]) {
  if (!p || !out || (level != TL_COARSE && level != TL_FINE)) return TL_EINVAL;
  const Level& L = level == TL_COARSE ? p->C : p->Fi;
  const int32_t v[11] = {L.t.ex, L.t.ey, L.t.ez, L.wide ? L.tw.ex : 0, L.wide ? L.tw.ey : 0, L.wide ? L.tw.ez : 0,
                         L.tp.ex, L.tp.ey, L.tp.ez, L.grid, L.tuned};
  std::memcpy(out, v, sizeof v);
  return TL_OK;
}

tl_status tl_trace_last_solve(const tl_problem* p, tl_level level, uint64_t* host_out, size_t cap, size_t* n_out) {
  if (!p || !host_out || !n_out || (level != TL_COARSE && level != TL_FINE)) return TL_EINVAL;
  const Level& L = level == TL_COARSE ? p->C : p->Fi;
  std::vector<unsigned long long> buf(2 * TRACE_CAP);
  cudaError_t e = cudaStreamSynchronize(p->stream);
  if (e == cudaSuccess)
    e = cudaMemcpy(buf.data(), L.trace, buf.size() * sizeof(unsigned long long), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_status(e);
  const size_t n = std::min<size_t>((size_t)buf[0], TRACE_CAP - 1);
  const size_t m = std::min(n, cap);
  for (size_t i = 0; i < m; ++i) {
    host_out[2 * i] = buf[2 * (i + 1)];
    host_out[2 * i + 1] = buf[2 * (i + 1) + 1];
  }
  *n_out = n;
  return TL_OK;
}

// ---- batched jobs --------------------------------------------------------

tl_status tl_batch_create(void* stream, int launches_per_round, int max_jobs, tl_batch** out) {
  if (!out) return TL_EINVAL;
  *out = nullptr;
  if (launches_per_round < 1 || launches_per_round > 64 || max_jobs < 1 || max_jobs > BATCH_MAX) return TL_EINVAL;
  tl_batch* b = new (std::nothrow) tl_batch();
  if (!b) return TL_ENOMEM;
  b->stream = (cudaStream_t)stream;
  b->R = launches_per_round;
  int dev = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->nsm, cudaDevAttrMultiProcessorCount, dev);
  b->max_coop = 1 << 30;
  for (int m = 0; m < 3 && e == cudaSuccess; ++m) {
    e = cudaFuncSetAttribute(batch_kernel_for(m), cudaFuncAttributeMaxDynamicSharedMemorySize, STAGE_BYTES);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_kernel_for(m), NT, STAGE_BYTES);
    if (e == cudaSuccess && per_sm < 1) e = cudaErrorInvalidConfiguration;
    b->max_coop_v[m] = std::min(per_sm * b->nsm, MAX_GRID_BLOCKS);
    b->max_coop = std::min(b->max_coop, b->max_coop_v[m]);
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    delete b;
    return TL_ECUDA;
  }
  b->cap = std::min(max_jobs, b->max_coop);
  const size_t targs = (size_t)b->R * b->cap * sizeof(SolveArgs), ttab = sizeof(BatchTable);
  e = cudaMalloc(&b->d_tab, ttab);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_args, targs);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_st, BATCH_MAX * sizeof(int));
  if (e == cudaSuccess) e = cudaHostAlloc(&b->h_tab, ttab, cudaHostAllocDefault);
  if (e == cudaSuccess) e = cudaHostAlloc(&b->h_args, targs, cudaHostAllocDefault);
  if (e == cudaSuccess) e = cudaHostAlloc(&b->h_st, BATCH_MAX * sizeof(int), cudaHostAllocDefault);
  if (e != cudaSuccess) {
    cudaGetLastError();
    cudaFree(b->d_tab);
    cudaFree(b->d_args);
    cudaFree(b->d_st);
    cudaFreeHost(b->h_tab);
    cudaFreeHost(b->h_args);
    cudaFreeHost(b->h_st);
    delete b;
    return e == cudaErrorMemoryAllocation ? TL_ENOMEM : TL_ECUDA;
  }
  *out = b;
  return TL_OK;
}

tl_status tl_batch_add(tl_batch* b, tl_problem* p, int macro_steps, int* id_out) {
  if (!b || !p || macro_steps < 0 || !id_out) return TL_EINVAL;
  if (p->cfg.coupling_sweeps > 1) return TL_EINVAL;  // batched sequences use the one-pass correction
  if (p->cfg.picard_iters > 1) return TL_EINVAL;     // ... and one solve per step
  if (p->cfg.interface_coupling != 0) return TL_EINVAL;  // ... and the restriction coupling
  if (p->phase != NEED_PREDICT) return TL_ESTATE;  // join only between macro steps
  int active = 0;
  for (const auto& j : b->jobs) active += j.active ? 1 : 0;
  if (active >= b->cap) return TL_ENOMEM;            // every launch slot is taken
  for (const auto& j : b->jobs)
    if (j.active && j.p == p) return TL_EINVAL;
  cudaError_t e = cudaStreamSynchronize(p->stream);  // the problem's own pending work first
  if (e != cudaSuccess) return cuda_status(e);
  // the whole-grid tiling: a job that runs (almost) alone in its launch can
  // then spread over most of the grid; crowded launches loop over tiles
  p->C.tb = p->C.t;
  p->Fi.tb = p->Fi.t;
  tl_batch::Job job{p, (long long)p->n + macro_steps, p->stream, true};
  p->stream = b->stream;
  int id = -1;
  for (size_t k = 0; k < b->jobs.size(); ++k)
    if (!b->jobs[k].active && b->jobs[k].p == nullptr) { id = (int)k; break; }
  if (id < 0) {
    id = (int)b->jobs.size();
    b->jobs.push_back(job);
  } else {
    b->jobs[id] = job;
  }
  *id_out = id;
  return TL_OK;
}

namespace {

// After the stream is synchronised: jobs whose solve failed in the last round
// leave the batch (their problem keeps its status word, which tl_sync reports).
void retire_failed(tl_batch* b) {
  for (size_t q = 0; q < b->round_ids.size(); ++q) {
    auto& j = b->jobs[b->round_ids[q]];
    if (j.active && b->h_st[q] != 0) {
      j.active = false;
      b->finished.push_back(b->round_ids[q]);
    }
  }
  b->round_ids.clear();
}

// Split the blocks of one launch over its jobs in proportion to their element
// counts (at least one block each, at most the job's reduction width).
void allocate_blocks(const std::vector<long long>& w, const std::vector<int>& capb, int B, std::vector<int>& nb) {
  const size_t J = w.size();
  nb.assign(J, 1);
  long long tw = 0;
  for (long long x : w) tw += x;
  int used = (int)J;
  for (size_t j = 0; j < J; ++j) {
    int want = (int)std::floor((double)B * w[j] / std::max(1LL, tw));
    want = std::min(std::max(want, 1), capb[j]);
    used += want - nb[j];
    nb[j] = want;
  }
  while (used > B) {  // trim the largest shares
    size_t k = 0;
    for (size_t j = 1; j < J; ++j)
      if (nb[j] > nb[k]) k = j;
    if (nb[k] <= 1) break;
    nb[k]--;
    used--;
  }
  while (used < B) {  // hand out the rest where work per block is largest
    int k = -1;
    double best = 0;
    for (size_t j = 0; j < J; ++j) {
      if (nb[j] >= capb[j]) continue;
      double r = (double)w[j] / nb[j];
      if (r > best) { best = r; k = (int)j; }
    }
    if (k < 0) break;
    nb[k]++;
    used++;
  }
}

}  // namespace

tl_status tl_batch_round(tl_batch* b, int* active_out) {
  if (!b) return TL_EINVAL;
  cudaError_t e = cudaStreamSynchronize(b->stream);  // staging buffers free again
  if (e != cudaSuccess) return cuda_status(e);
  retire_failed(b);
  BatchTable& tab = *b->h_tab;
  std::vector<long long> w;
  std::vector<int> capb;
  int nj = 0;
  int seen = 0;  // bit 0: a plain FP64 job, bit 1: a refined job in this round
  for (size_t id = 0; id < b->jobs.size(); ++id) {
    auto& j = b->jobs[id];
    if (!j.active) continue;
    if (j.p->n >= j.target && j.p->phase == NEED_PREDICT) {
      j.active = false;
      b->finished.push_back((int)id);
      continue;
    }
    // the job's next R solves (fewer if it reaches its target first)
    SolveArgs* args = b->h_args + (size_t)nj * b->R;
    long long work = 0;
    int ns = 0, cap_tiles = 1 << 30;
    while (ns < b->R && !(j.p->n >= j.target && j.p->phase == NEED_PREDICT)) {
      long long wt = 0;
      next_batched_solve(j.p, args[ns], &wt);
      const Tiling& t = args[ns].t;
      cap_tiles = std::min(cap_tiles, t.ntx * t.nty * t.ntz);
      work += wt;
      j.p->launches++;
      ++ns;
    }
    tab.nsolves[nj] = ns;
    b->round_ids.push_back((int)id);
    seen |= 1 << pmode_of(j.p->cfg);
    capb.push_back(j.p->max_slice);
    w.push_back(work);
    ++nj;
  }
  if (active_out) *active_out = nj;
  std::vector<int> nb;
  const int mode = seen == 1 ? 0 : (seen == 2 ? 1 : 2);
  allocate_blocks(w, capb, b->max_coop_v[mode], nb);
  // tile each solve for the slice it got: few large tiles in a crowded round,
  // many in a sparse one (tiling only sets how the slice walks the mesh)
  {
    int q = 0;
    for (size_t id = 0; id < b->jobs.size() && q < nj; ++id) {
      auto& j = b->jobs[id];
      if (!j.active) continue;
      Level tmpc = j.p->C, tmpf = j.p->Fi;
      choose_tiling(tmpc, nb[q], 1);
      choose_tiling(tmpf, nb[q], 1);
      SolveArgs* args = b->h_args + (size_t)q * b->R;
      // inner CG tiling for the slice: wide tiles when the slice is crowded
      const bool wc = use_wide(j.p->cfg, tmpc.g, nb[q]), wf = use_wide(j.p->cfg, tmpf.g, nb[q]);
      const Tiling twc = wc ? wide_tiling(tmpc.g, nb[q]) : Tiling{};
      const Tiling twf = wf ? wide_tiling(tmpf.g, nb[q]) : Tiling{};
      for (int sv = 0; sv < tab.nsolves[q]; ++sv) {
        const bool fine = args[sv].level == 1;
        args[sv].t = fine ? tmpf.t : tmpc.t;
        args[sv].wide = fine ? wf : wc;
        args[sv].tw = fine ? twf : twc;
        args[sv].tp = pc_tiling(fine ? tmpf.g : tmpc.g, nb[q]);
      }
      ++q;
    }
  }
  tab.njobs = nj;
  tab.per_job = b->R;
  tab.first[0] = 0;
  for (int q = 0; q < nj; ++q) tab.first[q + 1] = tab.first[q] + nb[q];
  if (nj == 0) return TL_OK;
  e = cudaMemcpyAsync(b->d_tab, b->h_tab, sizeof(BatchTable), cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->d_args, b->h_args, (size_t)nj * b->R * sizeof(SolveArgs), cudaMemcpyHostToDevice,
                        b->stream);
  if (e != cudaSuccess) return cuda_status(e);
  const BatchTable* tp = b->d_tab;
  const SolveArgs* ap = b->d_args;
  int* sp = b->d_st;
  void* kargs[] = {(void*)&tp, (void*)&ap, (void*)&sp};
  e = cudaLaunchCooperativeKernel(batch_kernel_for(mode), dim3(tab.first[nj]), dim3(NT), kargs, STAGE_BYTES,
                                  b->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->h_st, b->d_st, (size_t)nj * sizeof(int), cudaMemcpyDeviceToHost, b->stream);
  if (e != cudaSuccess) {
    b->round_ids.clear();
    return cuda_status(e);
  }
  b->launches++;
  b->rounds++;
  return TL_OK;
}

tl_status tl_batch_poll(tl_batch* b, int* ids, int cap, int* n_out) {
  if (!b || !n_out || (cap > 0 && !ids)) return TL_EINVAL;
  cudaError_t e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return cuda_status(e);
  retire_failed(b);
  // jobs that just reached their target are retired here too
  for (size_t id = 0; id < b->jobs.size(); ++id) {
    auto& j = b->jobs[id];
    if (j.active && j.p->n >= j.target && j.p->phase == NEED_PREDICT) {
      j.active = false;
      b->finished.push_back((int)id);
    }
  }
  int n = 0;
  while (!b->finished.empty() && n < cap) {
    const int id = b->finished.front();
    b->finished.erase(b->finished.begin());
    auto& j = b->jobs[id];
    j.p->stream = j.saved_stream;  // the problem leaves the batch
    j.p = nullptr;
    ids[n++] = id;
  }
  *n_out = n;
  return TL_OK;
}

tl_status tl_batch_info(const tl_batch* b, int* active, long long* launches) {
  if (!b) return TL_EINVAL;
  int a = 0;
  for (const auto& j : b->jobs) a += j.active ? 1 : 0;
  if (active) *active = a;
  if (launches) *launches = b->launches;
  return TL_OK;
}

void tl_batch_destroy(tl_batch* b) {
  if (!b) return;
  cudaStreamSynchronize(b->stream);
  for (auto& j : b->jobs)
    if (j.p) j.p->stream = j.saved_stream;
  cudaFree(b->d_tab);
  cudaFree(b->d_args);
  cudaFree(b->d_st);
  cudaFreeHost(b->h_tab);
  cudaFreeHost(b->h_args);
  cudaFreeHost(b->h_st);
  delete b;
}

void tl_destroy_problem(tl_problem* p) {
  if (!p) return;
  cudaStreamSynchronize(p->stream);
  release(p);
  delete p;
}

}  // extern "C"
