// Persistent cooperative backward-Euler solve on one uniform hexahedral mesh
// (fine patch or coarse plate), sm_103a.
//
// One launch performs a whole backward-Euler step of the heat equation
// (Section 2.1, Eq. thermalEqn) for the local problem Eq. (localProblemTime)
// or the global problem (Section 3), in phases separated by time-limited grid
// barriers:
//   0  element coefficients s_e = rho c(Tbar_e)/dt, k_e (lagged, state at T^k),
//      Dirichlet increments u_D = g - T_D, free guess 0, laser load F;
//   1  Jacobi diagonal, right-hand side of the increment system
//      A u = F - K T^k - A u_D  (partial sums per tile);
//   2  PCG on the free nodes: q = A p (fused p = z + beta p and <p,q>),
//      x/r update with fused <r,z>, <r,r>; stop at ||r|| <= tol ||r_0||;
//   3  T^{k+1} = T^k + u, element states, energy account.
//
// Matrix-free apply (the hot kernel): elements are owned by tiles of at most
// TXE x TYE x (any) elements; a tile marches up its element layers, computing
// each element's separable Hadamard transform exactly once, and writes the
// partial nodal sums of its window.  Window nodes owned by a neighbouring tile
// (the tile's high faces) go to one of seven exchange buffers indexed by which
// high faces they lie on; the owner adds them in a fixed order after the next
// barrier, so results are deterministic.
#pragma once

#include "tl_device.cuh"

namespace tl {

constexpr int TXE = 32;               // max tile width in elements (x)
constexpr int TYE = 8;                // max tile depth in elements (y)
constexpr int WX = TXE + 1, WY = TYE + 1;
constexpr int NT = 256;               // threads per block
constexpr int WPT = (WX * WY + NT - 1) / NT;  // window columns per thread
constexpr int MAXRECT = 8;
constexpr int NXB = 7;                // exchange buffers

struct DirSpec {
  int faces;    // bit0 x=0, bit1 x=nx, bit2 y=0, bit3 y=ny, bit4 z=0
  int box[6];   // extra Dirichlet nodes i0,i1,j0,j1,k0,k1 (inclusive); empty if i0 > i1
};

__device__ inline bool is_dir(const Grid3& g, const DirSpec& d, int i, int j, int k) {
  if ((d.faces & 1) && i == 0) return true;
  if ((d.faces & 2) && i == g.nx) return true;
  if ((d.faces & 4) && j == 0) return true;
  if ((d.faces & 8) && j == g.ny) return true;
  if ((d.faces & 16) && k == 0) return true;
  return i >= d.box[0] && i <= d.box[1] && j >= d.box[2] && j <= d.box[3] &&
         k >= d.box[4] && k <= d.box[5];
}

// Dirichlet values.  kind 0 (fine patch): nodes on the plate bottom take
// T_bottom, the others the blend (1-w) I(Tc0) + w I(Tc1) of the trilinear
// interpolants of two coarse fields.  kind 1 (coarse): k = 0 takes T_bottom,
// the box nodes take the injected fine values `inj`.
struct DirValues {
  int kind;
  double T_bottom, w;
  const double* Tc0;
  const double* Tc1;
  const double* inj;
  Grid3 cg;
  int oi, oj, ok, r;
};

__device__ inline double trilinear_at(const double* Tc, const Grid3& cg, int gi, int gj, int gk, int r) {
  int I = min(gi / r, cg.nx - 1), J = min(gj / r, cg.ny - 1), K = min(gk / r, cg.nz - 1);
  double tx = (double)(gi - I * r) / r, ty = (double)(gj - J * r) / r, tz = (double)(gk - K * r) / r;
  double v = 0.0;
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    int ax = a & 1, ay = (a >> 1) & 1, az = (a >> 2) & 1;
    double w = (ax ? tx : 1.0 - tx) * (ay ? ty : 1.0 - ty) * (az ? tz : 1.0 - tz);
    v += w * __ldcg(Tc + node_id(cg, I + ax, J + ay, K + az));
  }
  return v;
}

__device__ inline double dir_value(const DirValues& dv, int i, int j, int k, long long n) {
  if (dv.kind == 0) {
    int gi = i + dv.oi * dv.r, gj = j + dv.oj * dv.r, gk = k + dv.ok * dv.r;
    if (gk == 0) return dv.T_bottom;
    double a = trilinear_at(dv.Tc0, dv.cg, gi, gj, gk, dv.r);
    double b = trilinear_at(dv.Tc1, dv.cg, gi, gj, gk, dv.r);
    return (1.0 - dv.w) * a + dv.w * b;
  }
  if (k == 0) return dv.T_bottom;
  return __ldcg(dv.inj + n);
}

// Top-surface load: kind 1 the Gaussian amp exp(-alpha^2 |x - c|^2)
// (alpha = sqrt(3)/R, amp = 3 eta P/(pi R^2)); kind 2 a sum of constant
// fluxes on axis-aligned rectangles; both integrated exactly against the
// bilinear hats of the top face.  Node (i, j) sits at (ox + i hx, oy + j hy).
struct LoadSpec {
  int kind;
  double amp, alpha, xc, yc;
  double ox, oy;
  int nrect;
  double rect[MAXRECT][5];  // x0, x1, y0, y1, q
};

// int hat_i(x) exp(-alpha^2 (x-c)^2) dx over the mesh's extent (hat of node i
// of n+1 nodes, spacing h, origin o), in closed form with erf / exp.
__device__ inline double hat_gauss(int i, int n, double h, double o, double c, double alpha) {
  const double sp = 0.88622692545275801365;  // sqrt(pi)/2
  double G = 0.0;
  if (i > 0) {  // element [x_{i-1}, x_i]; node i carries (x - a)/h
    double a = o + h * (i - 1), b = o + h * i;
    double E0 = sp / alpha * (erf(alpha * (b - c)) - erf(alpha * (a - c)));
    double E1 = (exp(-(alpha * (a - c)) * (alpha * (a - c))) - exp(-(alpha * (b - c)) * (alpha * (b - c)))) /
                (2.0 * alpha * alpha);
    G += (E1 + (c - a) * E0) / h;
  }
  if (i < n) {  // element [x_i, x_{i+1}]; node i carries (b - x)/h
    double a = o + h * i, b = o + h * (i + 1);
    double E0 = sp / alpha * (erf(alpha * (b - c)) - erf(alpha * (a - c)));
    double E1 = (exp(-(alpha * (a - c)) * (alpha * (a - c))) - exp(-(alpha * (b - c)) * (alpha * (b - c)))) /
                (2.0 * alpha * alpha);
    G += ((b - c) * E0 - E1) / h;
  }
  return G;
}

// int_{x0}^{x1} hat_i(x) dx (interval clipped to the mesh).
__device__ inline double hat_box(int i, int n, double h, double o, double x0, double x1) {
  x0 = fmax(x0, o);
  x1 = fmin(x1, o + h * n);
  if (x1 <= x0) return 0.0;
  double H = 0.0;
  if (i > 0) {
    double a = o + h * (i - 1), b = o + h * i;
    double lo = fmax(x0, a), hi = fmin(x1, b);
    if (hi > lo) H += ((hi - a) * (hi - a) - (lo - a) * (lo - a)) / (2.0 * h);
  }
  if (i < n) {
    double a = o + h * i, b = o + h * (i + 1);
    double lo = fmax(x0, a), hi = fmin(x1, b);
    if (hi > lo) H += ((b - lo) * (b - lo) - (b - hi) * (b - hi)) / (2.0 * h);
  }
  return H;
}

__device__ inline double top_load(const LoadSpec& L, const Grid3& g, int i, int j) {
  if (L.kind == 1) {
    return L.amp * hat_gauss(i, g.nx, g.hx, L.ox, L.xc, L.alpha) *
           hat_gauss(j, g.ny, g.hy, L.oy, L.yc, L.alpha);
  }
  if (L.kind == 2) {
    double F = 0.0;
    for (int a = 0; a < L.nrect; ++a) {
      double hx = hat_box(i, g.nx, g.hx, L.ox, L.rect[a][0], L.rect[a][1]);
      double hy = hat_box(j, g.ny, g.hy, L.oy, L.rect[a][2], L.rect[a][3]);
      F += L.rect[a][4] * hx * hy;
    }
    return F;
  }
  return 0.0;
}

// Counters written by block 0 at the end of each solve (index: 0 coarse, 1 fine).
struct DevStats {
  double e_stored[2], e_laser[2], e_flux[2];
  long long iters[2], solves[2];
  int max_iters[2], last_iters[2];
};

struct Tiling {
  int ex, ey, ez;     // tile size in elements
  int ntx, nty, ntz;  // tile counts
};

template <typename R>
struct SolveArgs {
  Grid3 g;
  Tiling t;
  const double* T_in;
  double* T_out;
  double* u;   // increment
  double* r;   // residual
  R* p0;
  R* p1;
  R* q;
  R* X;        // NXB exchange buffers of nnode each
  R* dinv;
  R* s_e;
  R* k_e;
  double* F;   // top-face load, (nx+1)(ny+1)
  uint8_t* state;
  int st_sx, st_sy, st_ox, st_oy;  // element (ie,je,ke) -> state[(ke st_sy + je + st_oy) st_sx + ie + st_ox]
  DirSpec dir;
  DirValues dv;
  LoadSpec ld;
  Material mat;
  double dt, tol;
  int max_iter;
  int energy, update_state, level;
  double Mc[8], Kc[8], Md, Kd, vol8;
  double Mhat[64], Khat[64];
  Barrier bar;
  double* red;     // reduction slots [16][red_stride]
  int red_stride;
  DevStats* stats;
};

template <typename R>
struct ApplySmem {
  R X[2][WY][WX];                          // input values of two node layers
  union {
    R Z[2][WY][WX];                        // z sum / difference per node column
    struct { R L[2][TYE][WX]; R H[2][TYE][WX]; } yb;  // y-backward to low / high node row
  } a;
  R Y[4][TYE][WX];                         // (y,z)-modes per element row x node column
  R XL[4][TYE][TXE];                       // x-backward to the element's left node column
  R XR[4][TYE][TXE];                       // ... and to its right node column
};

// Apply one tile: for every window node n of tile `tile`, call
// emit(slot, li, lj, n, i, j, k, y, xin) with y the tile's partial of (A x)_n
// and xin = x_n as loaded; `load(n)` returns x_n (called once per window node).
// lam(e, lam8) fills the eight Hadamard eigenvalues of element e.
template <typename R, class Load, class Lam, class Emit>
__device__ inline void apply_tile(const Grid3& g, const Tiling& t, int tile, ApplySmem<R>& sm,
                                  Load load, Lam lam, Emit emit) {
  const int tid = threadIdx.x;
  const int tix = tile % t.ntx, tiy = (tile / t.ntx) % t.nty, tiz = tile / (t.ntx * t.nty);
  const int ie0 = tix * t.ex, je0 = tiy * t.ey, ke0 = tiz * t.ez;
  const int ex = min(t.ex, g.nx - ie0), ey = min(t.ey, g.ny - je0), ke1 = min(ke0 + t.ez, g.nz);
  const int wx = ex + 1, wy = ey + 1, nwin = wx * wy;
  int cur = 0;
  for (int idx = tid; idx < nwin; idx += NT) {
    int li = idx % wx, lj = idx / wx;
    sm.X[cur][lj][li] = load(node_id(g, ie0 + li, je0 + lj, ke0));
  }
  R carry[WPT];
#pragma unroll
  for (int w = 0; w < WPT; ++w) carry[w] = R(0);
  __syncthreads();
  for (int ke = ke0; ke < ke1; ++ke) {
    const int nxt = cur ^ 1;
    // stage 1: next layer, z-direction Hadamard per window column
    for (int idx = tid; idx < nwin; idx += NT) {
      int li = idx % wx, lj = idx / wx;
      R hi = load(node_id(g, ie0 + li, je0 + lj, ke + 1));
      R lo = sm.X[cur][lj][li];
      sm.X[nxt][lj][li] = hi;
      sm.a.Z[0][lj][li] = lo + hi;
      sm.a.Z[1][lj][li] = lo - hi;
    }
    __syncthreads();
    // stage 2: y-direction per element row and node column
    for (int idx = tid; idx < ey * wx; idx += NT) {
      int li = idx % wx, ly = idx / wx;
#pragma unroll
      for (int z = 0; z < 2; ++z) {
        R a = sm.a.Z[z][ly][li], b = sm.a.Z[z][ly + 1][li];
        sm.Y[2 * z][ly][li] = a + b;
        sm.Y[2 * z + 1][ly][li] = a - b;
      }
    }
    __syncthreads();
    // stage 3: per element, x-direction, eigenvalue scaling, x-backward
    for (int idx = tid; idx < ey * ex; idx += NT) {
      int lx = idx % ex, ly = idx / ex;
      R l8[8];
      lam(elem_id(g, ie0 + lx, je0 + ly, ke), l8);
#pragma unroll
      for (int m4 = 0; m4 < 4; ++m4) {
        R a = sm.Y[m4][ly][lx], b = sm.Y[m4][ly][lx + 1];
        R ys = l8[2 * m4] * (a + b);
        R yd = l8[2 * m4 + 1] * (a - b);
        sm.XL[m4][ly][lx] = ys + yd;
        sm.XR[m4][ly][lx] = ys - yd;
      }
    }
    __syncthreads();
    // stage 4: gather x-backward per node column, y-backward
    for (int idx = tid; idx < ey * wx; idx += NT) {
      int li = idx % wx, ly = idx / wx;
      R B[4];
#pragma unroll
      for (int m4 = 0; m4 < 4; ++m4) {
        R v = li < ex ? sm.XL[m4][ly][li] : R(0);
        if (li > 0) v += sm.XR[m4][ly][li - 1];
        B[m4] = v;
      }
#pragma unroll
      for (int z = 0; z < 2; ++z) {
        sm.a.yb.L[z][ly][li] = B[2 * z] + B[2 * z + 1];
        sm.a.yb.H[z][ly][li] = B[2 * z] - B[2 * z + 1];
      }
    }
    __syncthreads();
    // stage 5: gather y-backward per node column, z-backward, emit layer ke
#pragma unroll
    for (int w = 0; w < WPT; ++w) {
      int idx = tid + w * NT;
      if (idx < nwin) {
        int li = idx % wx, lj = idx / wx;
        R C0 = lj < ey ? sm.a.yb.L[0][lj][li] : R(0);
        R C1 = lj < ey ? sm.a.yb.L[1][lj][li] : R(0);
        if (lj > 0) {
          C0 += sm.a.yb.H[0][lj - 1][li];
          C1 += sm.a.yb.H[1][lj - 1][li];
        }
        const int i = ie0 + li, j = je0 + lj;
        emit(li, lj, ex, ey, node_id(g, i, j, ke), i, j, ke, carry[w] + (C0 + C1), sm.X[cur][lj][li]);
        carry[w] = C0 - C1;
      }
    }
    __syncthreads();
    cur = nxt;
  }
  // top node layer of the tile: only the contributions of element layer ke1-1
#pragma unroll
  for (int w = 0; w < WPT; ++w) {
    int idx = tid + w * NT;
    if (idx < nwin) {
      int li = idx % wx, lj = idx / wx;
      const int i = ie0 + li, j = je0 + lj;
      emit(li, lj, ex, ey, node_id(g, i, j, ke1), i, j, ke1, carry[w], sm.X[cur][lj][li]);
    }
  }
  __syncthreads();
}

// Which exchange buffer a window node's partial goes to: 0 = owned by this
// tile (write to the primary array), else 1 + (high-x) + 2 (high-y) + 4 (high-z) - 1.
__device__ inline int window_slot(const Grid3& g, const Tiling& t, int tile, int i, int j, int k) {
  const int tix = tile % t.ntx, tiy = (tile / t.ntx) % t.nty, tiz = tile / (t.ntx * t.nty);
  const int ie1 = min((tix + 1) * t.ex, g.nx), je1 = min((tiy + 1) * t.ey, g.ny),
            ke1 = min((tiz + 1) * t.ez, g.nz);
  return (i == ie1 && ie1 < g.nx ? 1 : 0) | (j == je1 && je1 < g.ny ? 2 : 0) | (k == ke1 && ke1 < g.nz ? 4 : 0);
}

// Full nodal value: own partial plus the neighbours' exchange partials, fixed order.
template <typename R>
__device__ inline R gather_partials(const Grid3& g, const Tiling& t, const R* prim, const R* X,
                                    long long nn, long long n, int i, int j, int k) {
  R v = __ldcg(prim + n);
  const bool lx = i > 0 && i < g.nx && (i % t.ex) == 0;
  const bool ly = j > 0 && j < g.ny && (j % t.ey) == 0;
  const bool lz = k > 0 && k < g.nz && (k % t.ez) == 0;
  if (lx) v += __ldcg(X + 0 * nn + n);
  if (ly) v += __ldcg(X + 1 * nn + n);
  if (lx && ly) v += __ldcg(X + 2 * nn + n);
  if (lz) v += __ldcg(X + 3 * nn + n);
  if (lx && lz) v += __ldcg(X + 4 * nn + n);
  if (ly && lz) v += __ldcg(X + 5 * nn + n);
  if (lx && ly && lz) v += __ldcg(X + 6 * nn + n);
  return v;
}

template <typename R>
__device__ inline void store_partial(R* prim, R* X, long long nn, long long n, int slot, R v, bool add) {
  R* dst = slot == 0 ? prim + n : X + (long long)(slot - 1) * nn + n;
  if (add) v += *dst;
  *dst = v;
}

enum RedSlot { RS_RZ0 = 0, RS_BB = 1, RS_PQ = 2, RS_RZ = 3, RS_RR = 4, RS_ES = 5, RS_EL = 6, RS_EF = 7, RS_N = 8 };

template <typename R>
__global__ void __launch_bounds__(NT, 2) solve_kernel(const SolveArgs<R> a) {
  __shared__ ApplySmem<R> sm;
  __shared__ double s_Mhat[64], s_Khat[64];
  if (ld_volatile_i32(a.bar.status) != 0) return;  // an earlier solve failed: leave state untouched
  const Grid3 g = a.g;
  const Tiling t = a.t;
  const long long nn = (long long)g.nnx * g.nny * g.nnz;
  const long long ne = (long long)g.nx * g.ny * g.nz;
  const long long gtid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long gstride = (long long)gridDim.x * blockDim.x;
  const int ntiles = t.ntx * t.nty * t.ntz;
  if (threadIdx.x < 64) {
    s_Mhat[threadIdx.x] = a.Mhat[threadIdx.x];
    s_Khat[threadIdx.x] = a.Khat[threadIdx.x];
  }

  // ---- phase 0: coefficients, Dirichlet increments, load ------------------
  for (long long e = gtid; e < ne; e += gstride) {
    int ie = (int)(e % g.nx), je = (int)((e / g.nx) % g.ny), ke = (int)(e / ((long long)g.nx * g.ny));
    double s = __ldcg(a.T_in + node_id(g, ie, je, ke));
    s += __ldcg(a.T_in + node_id(g, ie + 1, je, ke));
    s += __ldcg(a.T_in + node_id(g, ie, je + 1, ke));
    s += __ldcg(a.T_in + node_id(g, ie + 1, je + 1, ke));
    s += __ldcg(a.T_in + node_id(g, ie, je, ke + 1));
    s += __ldcg(a.T_in + node_id(g, ie + 1, je, ke + 1));
    s += __ldcg(a.T_in + node_id(g, ie, je + 1, ke + 1));
    s += __ldcg(a.T_in + node_id(g, ie + 1, je + 1, ke + 1));
    const double Tb = s * 0.125;
    const uint8_t st = a.state[((long long)ke * a.st_sy + je + a.st_oy) * a.st_sx + ie + a.st_ox];
    const double rc = a.mat.rho * (a.mat.c0 + a.mat.c1 * (Tb - a.mat.Tref));
    double k = a.mat.k0 + a.mat.k1 * (Tb - a.mat.Tref);
    if (st == POWDER) k = a.mat.powder_factor * k;
    a.s_e[e] = (R)(rc / a.dt);
    a.k_e[e] = (R)k;
  }
  for (long long n = gtid; n < nn; n += gstride) {
    int i = (int)(n % g.nnx), j = (int)((n / g.nnx) % g.nny), k = (int)(n / ((long long)g.nnx * g.nny));
    double u = 0.0;
    if (is_dir(g, a.dir, i, j, k)) u = dir_value(a.dv, i, j, k, n) - __ldcg(a.T_in + n);
    a.u[n] = u;
  }
  for (long long n = gtid; n < (long long)g.nnx * g.nny; n += gstride) {
    int i = (int)(n % g.nnx), j = (int)(n / g.nnx);
    a.F[n] = top_load(a.ld, g, i, j);
  }
  if (!grid_sync(a.bar)) return;

  // ---- phase 1: Jacobi diagonal and right-hand side partials --------------
  for (long long n = gtid; n < nn; n += gstride) {
    int i = (int)(n % g.nnx), j = (int)((n / g.nnx) % g.nny), k = (int)(n / ((long long)g.nnx * g.nny));
    R di = R(0);
    if (!is_dir(g, a.dir, i, j, k)) {
      double d = 0.0;
      for (int dz = -1; dz <= 0; ++dz)
        for (int dy = -1; dy <= 0; ++dy)
          for (int dx = -1; dx <= 0; ++dx) {
            int ie = i + dx, je = j + dy, ke = k + dz;
            if (ie < 0 || je < 0 || ke < 0 || ie >= g.nx || je >= g.ny || ke >= g.nz) continue;
            long long e = elem_id(g, ie, je, ke);
            d += (double)__ldcg(a.s_e + e) * a.Md + (double)__ldcg(a.k_e + e) * a.Kd;
          }
      di = (R)(1.0 / d);
    }
    a.dinv[n] = di;
  }
  {
    // r_partial = A u_D-guess (s and k) + K T  via two passes
    auto lam_full = [&](long long e, R (&l8)[8]) {
      R s = __ldcg(a.s_e + e), k = __ldcg(a.k_e + e);
      l8[0] = s * (R)a.Mc[0];
#pragma unroll
      for (int m = 1; m < 8; ++m) l8[m] = s * (R)a.Mc[m] + k * (R)a.Kc[m];
    };
    auto lam_k = [&](long long e, R (&l8)[8]) {
      R k = __ldcg(a.k_e + e);
      l8[0] = R(0);
#pragma unroll
      for (int m = 1; m < 8; ++m) l8[m] = k * (R)a.Kc[m];
    };
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
      auto load_u = [&](long long n) -> R { return (R)__ldcg(a.u + n); };
      auto load_T = [&](long long n) -> R { return (R)__ldcg(a.T_in + n); };
      auto emit1 = [&](int li, int lj, int ex, int ey, long long n, int i, int j, int k, R y, R xin) {
        store_partial(a.q, a.X, nn, n, window_slot(g, t, tile, i, j, k), y, false);
      };
      auto emit2 = [&](int li, int lj, int ex, int ey, long long n, int i, int j, int k, R y, R xin) {
        store_partial(a.q, a.X, nn, n, window_slot(g, t, tile, i, j, k), y, true);
      };
      apply_tile<R>(g, t, tile, sm, load_u, lam_full, emit1);
      apply_tile<R>(g, t, tile, sm, load_T, lam_k, emit2);
    }
  }
  if (!grid_sync(a.bar)) return;
  {
    double v[2] = {0.0, 0.0};
    for (long long n = gtid; n < nn; n += gstride) {
      int i = (int)(n % g.nnx), j = (int)((n / g.nnx) % g.nny), k = (int)(n / ((long long)g.nnx * g.nny));
      double rr = 0.0;
      if (!is_dir(g, a.dir, i, j, k)) {
        double Fn = (k == g.nz) ? __ldcg(a.F + (n - (long long)g.nnx * g.nny * g.nz)) : 0.0;
        rr = Fn - (double)gather_partials(g, t, a.q, a.X, nn, n, i, j, k);
      }
      a.r[n] = rr;
      v[0] += rr * rr * (double)__ldcg(a.dinv + n);
      v[1] += rr * rr;
    }
    block_reduce_store<2>(v, a.red + RS_RZ0 * a.red_stride, a.red_stride);
  }
  if (!grid_sync(a.bar)) return;
  double tot0[2];
  grid_total<2>(a.red + RS_RZ0 * a.red_stride, a.red_stride, tot0);
  double rz = tot0[0];
  const double bb = tot0[1];

  // ---- phase 2: preconditioned conjugate gradients ------------------------
  int it = 0;
  bool conv = !(bb > 0.0) || (a.tol >= 1.0);
  double rz_prev = 1.0;
  const double thresh = a.tol * a.tol * bb;
  while (!conv && it < a.max_iter) {
    const double beta = it == 0 ? 0.0 : rz / rz_prev;
    R* pold = (it & 1) ? a.p0 : a.p1;
    R* pnew = (it & 1) ? a.p1 : a.p0;
    double pq = 0.0;
    auto lam_full = [&](long long e, R (&l8)[8]) {
      R s = __ldcg(a.s_e + e), k = __ldcg(a.k_e + e);
      l8[0] = s * (R)a.Mc[0];
#pragma unroll
      for (int m = 1; m < 8; ++m) l8[m] = s * (R)a.Mc[m] + k * (R)a.Kc[m];
    };
    const R rbeta = (R)beta;
    const bool first = it == 0;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
      auto load_p = [&](long long n) -> R {
        R z = __ldcg(a.dinv + n) * (R)__ldcg(a.r + n);
        return first ? z : z + rbeta * __ldcg(pold + n);
      };
      auto emit = [&](int li, int lj, int ex, int ey, long long n, int i, int j, int k, R y, R xin) {
        int slot = window_slot(g, t, tile, i, j, k);
        store_partial(a.q, a.X, nn, n, slot, y, false);
        if (slot == 0) pnew[n] = xin;
        pq += (double)(xin * y);
      };
      apply_tile<R>(g, t, tile, sm, load_p, lam_full, emit);
    }
    {
      double v[1] = {pq};
      block_reduce_store<1>(v, a.red + RS_PQ * a.red_stride, a.red_stride);
    }
    if (!grid_sync(a.bar)) return;
    double tp[1];
    grid_total<1>(a.red + RS_PQ * a.red_stride, a.red_stride, tp);
    const double alpha = rz / tp[0];
    double v[2] = {0.0, 0.0};
    for (long long n = gtid; n < nn; n += gstride) {
      int i = (int)(n % g.nnx), j = (int)((n / g.nnx) % g.nny), k = (int)(n / ((long long)g.nnx * g.nny));
      if (is_dir(g, a.dir, i, j, k)) continue;
      double qn = (double)gather_partials(g, t, a.q, a.X, nn, n, i, j, k);
      double pn = (double)__ldcg(pnew + n);
      double un = __ldcg(a.u + n) + alpha * pn;
      double rn = __ldcg(a.r + n) - alpha * qn;
      a.u[n] = un;
      a.r[n] = rn;
      v[0] += rn * rn * (double)__ldcg(a.dinv + n);
      v[1] += rn * rn;
    }
    block_reduce_store<2>(v, a.red + RS_RZ * a.red_stride, a.red_stride);
    if (!grid_sync(a.bar)) return;
    double tr[2];
    grid_total<2>(a.red + RS_RZ * a.red_stride, a.red_stride, tr);
    rz_prev = rz;
    rz = tr[0];
    ++it;
    conv = tr[1] <= thresh;
  }
  const int lvl = a.level;
  if (!conv) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      atomicCAS(a.bar.status, 0, (int)ST_NOCONV);
      a.stats->iters[lvl] += it;
      a.stats->last_iters[lvl] = it;
    }
    return;
  }

  // ---- phase 3: update, states, energy -------------------------------------
  for (long long n = gtid; n < nn; n += gstride) a.T_out[n] = __ldcg(a.T_in + n) + __ldcg(a.u + n);
  if (a.update_state || a.energy) {
    if (!grid_sync(a.bar)) return;
    double v[3] = {0.0, 0.0, 0.0};
    for (long long e = gtid; e < ne; e += gstride) {
      int ie = (int)(e % g.nx), je = (int)((e / g.nx) % g.ny), ke = (int)(e / ((long long)g.nx * g.ny));
      if (a.update_state) {
        double s = __ldcg(a.T_out + node_id(g, ie, je, ke));
        s += __ldcg(a.T_out + node_id(g, ie + 1, je, ke));
        s += __ldcg(a.T_out + node_id(g, ie, je + 1, ke));
        s += __ldcg(a.T_out + node_id(g, ie + 1, je + 1, ke));
        s += __ldcg(a.T_out + node_id(g, ie, je, ke + 1));
        s += __ldcg(a.T_out + node_id(g, ie + 1, je, ke + 1));
        s += __ldcg(a.T_out + node_id(g, ie, je + 1, ke + 1));
        s += __ldcg(a.T_out + node_id(g, ie + 1, je + 1, ke + 1));
        const double Tb = s * 0.125;
        uint8_t* sp = a.state + ((long long)ke * a.st_sy + je + a.st_oy) * a.st_sx + ie + a.st_ox;
        uint8_t st = *sp;
        uint8_t ns = (st == POWDER) ? POWDER : SOLID;
        if (Tb > a.mat.T_melt) ns = MELTED;
        *sp = ns;
      }
      if (a.energy) {
        double us = 0.0;
#pragma unroll
        for (int c = 0; c < 8; ++c)
          us += __ldcg(a.u + node_id(g, ie + (c & 1), je + ((c >> 1) & 1), ke + (c >> 2)));
        v[0] += (double)__ldcg(a.s_e + e) * a.dt * a.vol8 * us;
      }
    }
    if (a.energy) {
      for (long long n = gtid; n < (long long)g.nnx * g.nny; n += gstride) v[1] += a.dt * __ldcg(a.F + n);
      __syncthreads();
      for (long long n = gtid; n < nn; n += gstride) {
        int i = (int)(n % g.nnx), j = (int)((n / g.nnx) % g.nny), k = (int)(n / ((long long)g.nnx * g.nny));
        if (!is_dir(g, a.dir, i, j, k)) continue;
        // reaction of a Dirichlet row: (S u + K T^{k+1})_n - F_n
        double R_n = 0.0;
        for (int dz = -1; dz <= 0; ++dz)
          for (int dy = -1; dy <= 0; ++dy)
            for (int dx = -1; dx <= 0; ++dx) {
              int ie = i + dx, je = j + dy, ke = k + dz;
              if (ie < 0 || je < 0 || ke < 0 || ie >= g.nx || je >= g.ny || ke >= g.nz) continue;
              long long e = elem_id(g, ie, je, ke);
              double se = (double)__ldcg(a.s_e + e), kk = (double)__ldcg(a.k_e + e);
              int la = (i - ie) + 2 * (j - je) + 4 * (k - ke);
              double acc = 0.0;
#pragma unroll
              for (int b = 0; b < 8; ++b) {
                long long nb = node_id(g, ie + (b & 1), je + ((b >> 1) & 1), ke + (b >> 2));
                acc += se * s_Mhat[la * 8 + b] * __ldcg(a.u + nb) + kk * s_Khat[la * 8 + b] * __ldcg(a.T_out + nb);
              }
              R_n += acc;
            }
        if (k == g.nz) R_n -= __ldcg(a.F + (n - (long long)g.nnx * g.nny * g.nz));
        v[2] += a.dt * R_n;
      }
    }
    block_reduce_store<3>(v, a.red + RS_ES * a.red_stride, a.red_stride);
    if (!grid_sync(a.bar)) return;
    if (blockIdx.x == 0) {
      double te[3];
      grid_total<3>(a.red + RS_ES * a.red_stride, a.red_stride, te);
      if (threadIdx.x == 0 && a.energy) {
        a.stats->e_stored[lvl] += te[0];
        a.stats->e_laser[lvl] += te[1];
        a.stats->e_flux[lvl] += te[2];
      }
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    a.stats->iters[lvl] += it;
    a.stats->solves[lvl] += 1;
    a.stats->last_iters[lvl] = it;
    if (it > a.stats->max_iters[lvl]) a.stats->max_iters[lvl] = it;
  }
}

// ---------------------------------------------------------------------------
// Small kernels: patch motion and fine -> coarse injection.  Defined in the
// two-level translation unit only (a unit that needs just the solve kernel
// defines TL_SOLVE_KERNEL_ONLY before including this header).
// ---------------------------------------------------------------------------
#ifndef TL_SOLVE_KERNEL_ONLY

// New fine field after the patch origin moved from (ooi, ooj) to (noi, noj)
// (coarse node indices; z fixed): nodes inside the old patch keep their
// values, the others take the trilinear interpolant of the coarse field.
__global__ void move_patch_kernel(Grid3 fg, Grid3 cg, const double* __restrict__ Tf_old,
                                  double* __restrict__ Tf_new, const double* __restrict__ Tc,
                                  int ooi, int ooj, int noi, int noj, int ok, int r) {
  const long long nn = (long long)fg.nnx * fg.nny * fg.nnz;
  for (long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x; n < nn;
       n += (long long)gridDim.x * blockDim.x) {
    int i = (int)(n % fg.nnx), j = (int)((n / fg.nnx) % fg.nny), k = (int)(n / ((long long)fg.nnx * fg.nny));
    int oi = i + (noi - ooi) * r, oj = j + (noj - ooj) * r;
    double v;
    if (oi >= 0 && oi <= fg.nx && oj >= 0 && oj <= fg.ny) {
      v = Tf_old[node_id(fg, oi, oj, k)];
    } else {
      v = trilinear_at(Tc, cg, i + noi * r, j + noj * r, k + ok * r, r);
    }
    Tf_new[n] = v;
  }
}

// inj[coarse node] = fine T at the coinciding fine node, for the box nodes.
__global__ void restrict_kernel(Grid3 fg, Grid3 cg, const double* __restrict__ Tf, double* __restrict__ inj,
                                int bi0, int bi1, int bj0, int bj1, int bk0, int bk1, int oi, int oj, int ok, int r) {
  const int bx = bi1 - bi0 + 1, by = bj1 - bj0 + 1, bz = bk1 - bk0 + 1;
  const long long nb = (long long)bx * by * bz;
  for (long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x; n < nb;
       n += (long long)gridDim.x * blockDim.x) {
    int I = bi0 + (int)(n % bx), J = bj0 + (int)((n / bx) % by), K = bk0 + (int)(n / ((long long)bx * by));
    inj[node_id(cg, I, J, K)] = Tf[node_id(fg, (I - oi) * r, (J - oj) * r, (K - ok) * r)];
  }
}

__global__ void fill_kernel(double* __restrict__ x, long long n, double v) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    x[i] = v;
}

// Initial states: POWDER iff the element centroid is within `depth` of the top.
__global__ void init_state_kernel(uint8_t* __restrict__ st, int sx, int sy, int sz, double z0, double hz,
                                  double Lz, double depth) {
  const long long n = (long long)sx * sy * sz;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    int k = (int)(e / ((long long)sx * sy));
    double zc = z0 + (k + 0.5) * hz;
    st[e] = (Lz - zc < depth) ? POWDER : SOLID;
  }
}
#endif  // TL_SOLVE_KERNEL_ONLY

}  // namespace tl
