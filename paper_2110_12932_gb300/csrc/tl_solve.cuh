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

constexpr int TXE = 16;               // max tile width in elements (x)
constexpr int TYE = 8;                // max tile depth in elements (y)
constexpr int WX = TXE + 1, WY = TYE + 1;
constexpr int NT = 160;               // threads per block: one window column each
constexpr int MIN_BLOCKS = 4;         // resident blocks per SM the register budget targets
constexpr int NRAW = 13;              // staged raw inputs per window node (CG pass: 6 + 7 partials)
constexpr int STAGE_BYTES = 2 * NRAW * NT * 8;  // dynamic shared memory: two layers in flight

// Asynchronous global -> shared copies of 4 or 8 bytes (per-thread groups).
template <int BYTES>
__device__ inline void cp_async(void* smem, const void* gmem) {
  const unsigned int sa = (unsigned int)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(sa), "l"(gmem), "n"(BYTES) : "memory");
}
__device__ inline void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ inline void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }
// 8-byte asynchronous copy of which only the first src_bytes (0, 4 or 8) are
// read; the rest of the 8 shared-memory bytes is zero-filled.
__device__ inline void cp_async8_fill(void* smem, const void* gmem, int src_bytes) {
  const unsigned int sa = (unsigned int)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(sa), "l"(gmem), "r"(src_bytes) : "memory");
}
static_assert(NT >= WX * WY, "a block must cover a tile's window columns");
static_assert(NT <= 32 * (RED_W + 1), "block_reduce_store parks the lanes of warps 1 .. RED_W");
constexpr int MAXRECT = 8;
static_assert(MAXRECT >= 3, "the load tables hold 3 (nnx + nny) values for the Gaussian");
constexpr int NXB = 7;                // exchange buffers
// Stride of the exchange planes: the node count rounded up to four, so that a
// plane starts on a 16-byte boundary (vector loads of four FP32 partials).
__host__ __device__ inline int xplane(int nn) { return (nn + 3) & ~3; }

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

// Index of the first Dirichlet set holding node (i, j, k), in the order z = 0
// face, x = 0, x = nx, y = 0, y = ny, box; -1 if the node is free.
__device__ inline int dir_set(const Grid3& g, const DirSpec& d, int i, int j, int k) {
  if ((d.faces & 16) && k == 0) return 0;
  if ((d.faces & 1) && i == 0) return 1;
  if ((d.faces & 2) && i == g.nx) return 2;
  if ((d.faces & 4) && j == 0) return 3;
  if ((d.faces & 8) && j == g.ny) return 4;
  if (i >= d.box[0] && i <= d.box[1] && j >= d.box[2] && j <= d.box[3] && k >= d.box[4] && k <= d.box[5])
    return 5;
  return -1;
}

// Calls body(n, i, j, k) once for every Dirichlet node (a node is visited by
// the first set that holds it).  The candidates go in chunks of 32 consecutive
// ones, one warp per chunk, dealt round-robin over the blocks: the boundary's
// FP64 work (interpolation, reactions) spreads over all SMs instead of
// filling the first blocks, and a warp's loads stay contiguous.  Needs
// blockDim a multiple of 32.
template <class Body>
__device__ inline void for_dirichlet(const Grid3& g, const DirSpec& d, const VGrid& vg, Body body) {
  const int bx = d.box[1] - d.box[0] + 1, by = d.box[3] - d.box[2] + 1, bz = d.box[5] - d.box[4] + 1;
  const int sz[6] = {(d.faces & 16) ? g.nnx * g.nny : 0, (d.faces & 1) ? g.nny * g.nnz : 0,
                     (d.faces & 2) ? g.nny * g.nnz : 0, (d.faces & 4) ? g.nnx * g.nnz : 0,
                     (d.faces & 8) ? g.nnx * g.nnz : 0, (bx > 0 && by > 0 && bz > 0) ? bx * by * bz : 0};
  const int total = sz[0] + sz[1] + sz[2] + sz[3] + sz[4] + sz[5];
  const int lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
  const int nchunks = (total + 31) >> 5;
  for (int c = (threadIdx.x >> 5) * vg.nblk + vg.bid; c < nchunks; c += nwarps * vg.nblk) {
    const int m = c * 32 + lane;
    if (m >= total) continue;
    int set = 0, r = m;
    while (r >= sz[set]) r -= sz[set++];
    int i, j, k;
    if (set == 0) { i = r % g.nnx; j = r / g.nnx; k = 0; }
    else if (set <= 2) { j = r % g.nny; k = r / g.nny; i = set == 1 ? 0 : g.nx; }
    else if (set <= 4) { i = r % g.nnx; k = r / g.nnx; j = set == 3 ? 0 : g.ny; }
    else { i = d.box[0] + r % bx; j = d.box[2] + (r / bx) % by; k = d.box[4] + r / (bx * by); }
    if (dir_set(g, d, i, j, k) != set) continue;
    body(i + g.nnx * (j + g.nny * k), i, j, k);
  }
}

// Dirichlet values.  kind 0 (fine patch): nodes on the plate bottom take
// T_bottom, the others the blend (1-w) I(Tc0) + w I(Tc1) of the trilinear
// interpolants of two coarse fields.  kind 1 (coarse): k = 0 takes T_bottom,
// the box nodes take the injected fine values `inj`; kind 2: the same values
// read straight from the fine field (batched path).
struct DirValues {
  int kind;
  double T_bottom, w;
  const double* Tc0;
  const double* Tc1;
  const double* inj;
  const double* Tf;  // kind 2: the fine field itself (injection fused into the solve)
  Grid3 cg, fg;
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

// (1 - w) I(Tc0) + w I(Tc1) for two coarse fields at one fine node, with the
// eight trilinear weights formed once (each sum in the order trilinear_at uses).
__device__ inline double trilinear_blend(const double* Tc0, const double* Tc1, double w, const Grid3& cg, int gi,
                                         int gj, int gk, int r) {
  int I = min(gi / r, cg.nx - 1), J = min(gj / r, cg.ny - 1), K = min(gk / r, cg.nz - 1);
  double tx = (double)(gi - I * r) / r, ty = (double)(gj - J * r) / r, tz = (double)(gk - K * r) / r;
  double a = 0.0, b = 0.0;
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    int ax = c & 1, ay = (c >> 1) & 1, az = (c >> 2) & 1;
    double wt = (ax ? tx : 1.0 - tx) * (ay ? ty : 1.0 - ty) * (az ? tz : 1.0 - tz);
    const long long n = node_id(cg, I + ax, J + ay, K + az);
    a += wt * __ldcg(Tc0 + n);
    b += wt * __ldcg(Tc1 + n);
  }
  return (1.0 - w) * a + w * b;
}

__device__ inline double dir_value(const DirValues& dv, int i, int j, int k, long long n) {
  if (dv.kind == 0) {  // fine patch
    int gi = i + dv.oi * dv.r, gj = j + dv.oj * dv.r, gk = k + dv.ok * dv.r;
    if (gk == 0) return dv.T_bottom;
    return trilinear_blend(dv.Tc0, dv.Tc1, dv.w, dv.cg, gi, gj, gk, dv.r);
  }
  if (k == 0) return dv.T_bottom;
  if (dv.kind == 2)  // coarse node (i, j, k) of the injection box: the coinciding fine node
    return __ldcg(dv.Tf + node_id(dv.fg, (i - dv.oi) * dv.r, (j - dv.oj) * dv.r, (k - dv.ok) * dv.r));
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

// The top load is separable: F(i, j) = sum_f c_f Gx_f(i) Gy_f(j) over one
// Gaussian factor or one factor per rectangle.  Phase 0 tabulates what the
// factors need, so that each transcendental is evaluated once:
//  Gaussian: entry p < w = nnx + nny holds erf(alpha (x_p - c)) and entry
//   w + p exp(-(alpha (x_p - c))^2), x_p the position of x node p (p < nnx)
//   or of y node p - nnx; after the next grid barrier entry 2w + p gets the
//   1D hat integral of that node from them (hat_gauss_tab), and F is formed
//   after the barrier after that;
//  rectangles: entry f w + idx holds the box factor of x or y node idx.
__device__ inline int load_factors(const LoadSpec& L) { return L.kind == 1 ? 1 : (L.kind == 2 ? L.nrect : 0); }

__device__ inline int load_table_size(const LoadSpec& L, const Grid3& g) {
  const int w = g.nnx + g.nny;
  return L.kind == 1 ? 2 * w : (L.kind == 2 ? L.nrect * w : 0);
}

__device__ inline double load_table_entry(const LoadSpec& L, const Grid3& g, int m) {
  const int w = g.nnx + g.nny;
  if (L.kind == 1) {
    const int p = m < w ? m : m - w;
    const bool isx = p < g.nnx;
    const int i = isx ? p : p - g.nnx;
    const double t = L.alpha * ((isx ? L.ox + g.hx * i : L.oy + g.hy * i) - (isx ? L.xc : L.yc));
    return m < w ? erf(t) : exp(-t * t);
  }
  const int f = m / w, idx = m - f * w;
  const bool isx = idx < g.nnx;
  const int i = isx ? idx : idx - g.nnx;
  return isx ? hat_box(i, g.nx, g.hx, L.ox, L.rect[f][0], L.rect[f][1])
             : hat_box(i, g.ny, g.hy, L.oy, L.rect[f][2], L.rect[f][3]);
}

// int hat_i(x) exp(-alpha^2 (x-c)^2) dx over the mesh's extent (hat of node i
// of n+1 nodes, spacing h, origin o), in closed form from the tabulated
// erf (ef) and exp (ex) values at the node positions of that direction.
__device__ inline double hat_gauss_tab(int i, int n, double h, double o, double c, double alpha, const double* ef,
                                       const double* ex) {
  const double sp = 0.88622692545275801365;  // sqrt(pi)/2
  double G = 0.0;
  if (i > 0) {  // element [x_{i-1}, x_i]; node i carries (x - a)/h
    double a = o + h * (i - 1);
    double E0 = sp / alpha * (__ldcg(ef + i) - __ldcg(ef + i - 1));
    double E1 = (__ldcg(ex + i - 1) - __ldcg(ex + i)) / (2.0 * alpha * alpha);
    G += (E1 + (c - a) * E0) / h;
  }
  if (i < n) {  // element [x_i, x_{i+1}]; node i carries (b - x)/h
    double b = o + h * (i + 1);
    double E0 = sp / alpha * (__ldcg(ef + i + 1) - __ldcg(ef + i));
    double E1 = (__ldcg(ex + i) - __ldcg(ex + i + 1)) / (2.0 * alpha * alpha);
    G += ((b - c) * E0 - E1) / h;
  }
  return G;
}

// Entry p of the Gaussian's hat table (x node p, or y node p - nnx), from the
// erf / exp entries.
__device__ inline double gauss_hat_entry(const LoadSpec& L, const Grid3& g, const double* G, int p) {
  const int w = g.nnx + g.nny;
  return p < g.nnx ? hat_gauss_tab(p, g.nx, g.hx, L.ox, L.xc, L.alpha, G, G + w)
                   : hat_gauss_tab(p - g.nnx, g.ny, g.hy, L.oy, L.yc, L.alpha, G + g.nnx, G + w + g.nnx);
}

// F(i, j) from the tables (the Gaussian: its hat table at G + 2w).
__device__ inline double top_load_tab(const LoadSpec& L, const Grid3& g, const double* G, int i, int j) {
  const int nf = load_factors(L), w = g.nnx + g.nny;
  if (L.kind == 1) {
    double F = 0.0;
    F += L.amp * __ldcg(G + 2 * w + i) * __ldcg(G + 2 * w + g.nnx + j);
    return F;
  }
  double F = 0.0;
  for (int f = 0; f < nf; ++f) F += L.rect[f][4] * __ldcg(G + f * w + i) * __ldcg(G + f * w + g.nnx + j);
  return F;
}

// Counters written by block 0 at the end of each solve (index: 0 coarse, 1 fine).
struct DevStats {
  double e_stored[2], e_laser[2], e_flux[2], e_loss[2];
  long long iters[2], solves[2], outer[2];
  int max_iters[2], last_iters[2];
  double e_last[2][4];  // the last solve's stored / laser / flux / loss terms per level (for rollback)
};

// Converts eight Hadamard factors (index = x mode + 2 y mode + 4 z mode) to
// the pair form the apply uses: (f[2m], f[2m+1]) -> (f[2m] + f[2m+1], f[2m] - f[2m+1]).
__host__ __device__ inline void to_pair_form(double (&f)[8]) {
  for (int m4 = 0; m4 < 4; ++m4) {
    const double e = f[2 * m4], o = f[2 * m4 + 1];
    f[2 * m4] = e + o;
    f[2 * m4 + 1] = e - o;
  }
}

struct Tiling {
  int ex, ey, ez;     // tile size in elements
  int ntx, nty, ntz;  // tile counts
};

// Patch motion fused into a coarse predictor solve (batched path): the new
// fine field dst takes src where the old and new patches overlap and the
// trilinear interpolant of Tc elsewhere.
struct MoveSpec {
  int active;
  const double* src;
  double* dst;
  const double* Tc;
  Grid3 fg, cg;
  int ooi, ooj, noi, noj, ok, r;
};

enum Precision : int { PREC_FP64 = 0, PREC_FP32_REFINED = 1 };

// Everything one launch needs.  FP64 arrays serve the plain path, the
// right-hand side and the outer residual of the refined path; the FP32 arrays
// (NULL in the plain path) hold the refined path's inner CG.
struct SolveArgs {
  Grid3 g;
  Tiling t;
  const double* T_in;
  double* T_out;
  // Picard iterations of the nonlinear step: the coefficients are taken at
  // T_coef (null: T_in); with T_relax set the solve writes only
  // T_relax = Tc + (T_in + u - Tc) / 2 (Tc the coefficient temperature), not
  // T_out (T_relax may equal T_coef)
  const double* T_coef;
  double* T_relax;
  double* u;     // increment T^{k+1} - T^k (Dirichlet entries prescribed)
  double* r;     // FP64 residual
  double* r2;    // its second buffer (CG pass parity)
  double* q;     // own partial of an FP64 apply
  double* X;     // NXB exchange arrays of nnode each (FP64)
  double* q2;    // second partial buffers (CG pass parity)
  double* X2;
  double* p0;
  double* p1;
  double* s0;
  double* s1;
  double* dinv;
  double* s_e;
  double* k_e;
  double* lam;   // eight Hadamard eigenvalues per element, [8][nelem]
  float* d32;    // refined path: inner correction
  float* r32;
  float* r32b;
  float* q32;
  float* X32;
  float* q32b;
  float* X32b;
  float* p0f;
  float* p1f;
  float* s0f;
  float* s1f;
  float* dinv32;
  float* sk32;   // refined path: FP32 s_e, k_e ([2][nelem]); eigenvalues rebuilt in registers
  double* F;     // top-face load, (nx+1)(ny+1)
  const double* Fx;  // extra nodal load (the flux-jump coupling's interface load), or NULL
  double* G;     // load factor tables, MAXRECT (nnx + nny)
  uint8_t* state;
  uint8_t* st_new;  // the new element states (one per element, patch order) until the commit
  int st_sx, st_sy, st_ox, st_oy;  // element (ie,je,ke) -> state[(ke st_sy + je + st_oy) st_sx + ie + st_ox]
  DirSpec dir;
  DirValues dv;
  LoadSpec ld;
  Material mat;
  double dt, tol, tol_inner;
  int max_iter, max_outer, precision;
  int wide;        // refined path: inner CG on wide tiles (two-phase pcg2, tiling tw)
  int precond;     // 0 Jacobi (pcg1 / pcg2), 1 tensor-product mass preconditioner (pcg3)
  Tiling tp;       // pcg3: node-owned tiles of the preconditioner pass (ex x ey columns, ez layers)
  Tiling tw;
  int energy, update_state, level;
  int dry;         // a timing run of the tiling tuner: no counters, nothing committed but T_out
  double Mc[8], Kc[8], Md, Kd, vol8;  // Mc, Kc: eigenvalue factors in pair form (to_pair_form)
  double Mhat[64], Khat[64];
  // heat loss through the top surface (Section 3.1): h_f (T - T_amb) per top
  // face f with h_f = h_conv + rad (T*_f^2 + T_amb^2)(T*_f + T_amb), T*_f the
  // face mean of the coefficient temperature (rad = sigma_SB emissivity on the
  // fine level, 0 on the coarse one); hf / hf32 hold h_f (nx ny, x fastest)
  int surf;        // 0: adiabatic top
  double h_conv, rad, T_amb;
  double* hf;
  float* hf32;
  double Mfx[2], Mfy[2];  // 1D mass entries of the face hats: same node h/3, other node h/6
  Barrier bar;
  double* red;   // reduction slots [RS_N][red_stride]
  float* red32;  // FP32 reduction slots of the refined path's inner CG
  int red_stride;
  DevStats* stats;
  unsigned long long* trace;  // [TRACE_CAP][2] (marker, globaltimer ns) of this solve, or NULL
  MoveSpec mv;
};

// Phase markers recorded by block 0 when tracing.
enum TraceMark : int {
  TR_START = 0, TR_PHASE0 = 1, TR_RHS = 2, TR_RESID = 3, TR_CG_PASS = 4, TR_OUTER_INIT = 5,
  TR_OUTER_APPLY = 6, TR_OUTER_END = 7, TR_UPDATE = 8, TR_END = 9, TR_CG_APPLY = 10,
  TR_RR = 11,      // value marker: second word = <r,r> of the pass (IEEE double bits)
  TR_BREAK = 12,   // value marker: CG stopped on a non-positive recurrence term
  TR_CG_UPDATE = 13,
  TR_CG_U0 = 14,   // block 0 starts its share of a CG update phase
  TR_CG_U1 = 15,   // ... and finished it (before the block reduction)
  TR_CG_PRECOND = 16,  // the preconditioner phase of a CG iteration done (grid barrier passed)
  TR_P0_ELEMS = 17,    // block 0 has done its share of phase 0's element coefficients
  TR_P0_DIR = 18,      // ... and of the Dirichlet increments
  TR_P0_LOAD = 19,     // ... and of the laser-load tables (before the grid barrier)
  TR_END_ELEMS = 20,   // block 0 has done its share of the states and stored energy
  TR_END_DIR = 21      // ... and of the Dirichlet reactions (before the reduction)
};
constexpr int TRACE_CAP = 1024;

struct Tracer {
  unsigned long long* buf;
  int bid;
  int n = 0;
  __device__ void mark(int m) {
    if (buf && bid == 0 && threadIdx.x == 0 && n < TRACE_CAP - 1) {
      buf[2 * (n + 1)] = (unsigned long long)m;
      buf[2 * (n + 1) + 1] = global_ns();
      ++n;
      buf[0] = (unsigned long long)n;
    }
  }
  __device__ void value(int m, double v) {
    if (buf && bid == 0 && threadIdx.x == 0 && n < TRACE_CAP - 1) {
      buf[2 * (n + 1)] = (unsigned long long)m;
      buf[2 * (n + 1) + 1] = (unsigned long long)__double_as_longlong(v);
      ++n;
      buf[0] = (unsigned long long)n;
    }
  }
};

template <typename R>
struct ApplySmem {
  // A window column's input values stay in its thread's registers.  Z and the
  // y-backward are separate arrays, so that a layer needs no barrier after
  // its last stage: every array's next write comes after a later barrier.
  R Z[2][WY][WX];                          // z sum / difference per node column
  struct { R L[2][TYE][WX]; R H[2][TYE][WX]; } yb;  // y-backward to low / high node row
  R Y[4][TYE][WX];                         // (y,z)-modes per element row x node column
  R XL[4][TYE][TXE];                       // x-backward to the element's left node column
  R XR[4][TYE][TXE];                       // ... and to its right node column
};

// Apply one tile of at most TXE x TYE x ez elements with NT >= (TXE+1)(TYE+1)
// threads: every thread owns at most one window node column (stages 1 and 5),
// one (element row, node column) pair (stages 2 and 4, same index) and one
// element column (stage 3), all fixed for the tile, so the index arithmetic is
// done once per tile.  For every window node n the tile emits
// emit(n, slot, y, xin): y its partial of (A x)_n, xin = x_n as consumed,
// slot = 0 if the tile owns n, else (high-x) + 2 (high-y) + 4 (high-z).
// Inputs are staged one layer ahead: fetch(n, i, j, k, owned, raw) issues
// asynchronous copies of the raw data node n needs into the thread's staging
// slots raw[s * NT], and finish(n, i, j, k, owned, raw) turns them into x_n
// (called exactly once per window node, after the copies landed).  The
// copies for layer k+2 are issued while layer k is being processed.
// lam(e, l8) fills the eight Hadamard eigenvalues of element e in pair form:
// l8[2 m4] = lam[2 m4] + lam[2 m4 + 1], l8[2 m4 + 1] = lam[2 m4] - lam[2 m4 + 1]
// (m4 = the y, z mode; the pair differs in the x mode).
// Element data (the eigenvalues' inputs) are either loaded into registers at
// the start of each layer (LAM_STAGED false: lam(e, nullptr, l8) reads
// global memory) or staged one layer ahead in slots NRAW.. of the same ring
// (LAM_STAGED true: lam_fetch(e, slots) issues the copies, lam(e, slots, l8)
// builds the eigenvalues; slots start at LSLOT).  NS = slots per buffer and thread.
template <typename R, bool LAM_STAGED, int NS, int LSLOT = NRAW, class Fetch, class Finish, class LamFetch, class Lam,
          class Emit>
__device__ inline void apply_tile(const Grid3& g, const Tiling& t, int tile, ApplySmem<R>& sm, R* stage,
                                  Fetch fetch, Finish finish, LamFetch lam_fetch, Lam lam, Emit emit) {
  const int tid = threadIdx.x;
  const int txy = t.ntx * t.nty;
  const int tiz = tile / txy, trem = tile - tiz * txy;
  const int tiy = trem / t.ntx, tix = trem - tiy * t.ntx;
  const int ie0 = tix * t.ex, je0 = tiy * t.ey, ke0 = tiz * t.ez;
  const int ex = min(t.ex, g.nx - ie0), ey = min(t.ey, g.ny - je0), ke1 = min(ke0 + t.ez, g.nz);
  const int wx = ex + 1, nwin = wx * (ey + 1);
  const int S = g.nnx * g.nny;   // node layer stride
  const int Se = g.nx * g.ny;    // element layer stride
  const bool has_w = tid < nwin;        // window node column
  const bool has_r = tid < ey * wx;     // (element row, node column) pair
  const bool has_e = tid < ey * ex;     // element column
  const int wlj = tid / wx, wli = tid - wlj * wx;
  const int ely = tid / ex, elx = tid - ely * ex;
  const int wnode = (ie0 + wli) + g.nnx * (je0 + wlj);
  const int welem = (ie0 + elx) + g.nx * (je0 + ely);
  const int wslot = ((wli == ex && ie0 + ex < g.nx) ? 1 : 0) | ((wlj == ey && je0 + ey < g.ny) ? 2 : 0);
  const int wi = ie0 + wli, wj = je0 + wlj;
  const bool z_top_owned = ke1 == g.nz;  // the tile owns its top node layer only at the plate top
  R* raw0 = stage + tid;                 // staging buffer of node layers with (k - ke0) even
  R* raw1 = stage + NS * NT + tid;       // ... odd
  auto owned_at = [&](int k) { return wslot == 0 && (k < ke1 || z_top_owned); };
  if (has_w) fetch(wnode + ke0 * S, wi, wj, ke0, owned_at(ke0), raw0);
  cp_async_commit();
  if (has_w) fetch(wnode + (ke0 + 1) * S, wi, wj, ke0 + 1, owned_at(ke0 + 1), raw1);
  // element layer k sits in the buffer of node layer k + 1
  if (LAM_STAGED && has_e) lam_fetch(welem + ke0 * Se, raw1 + LSLOT * NT);
  cp_async_commit();
  cp_async_wait<1>();
  R xcur = R(0);  // the column's value at node layer ke
  if (has_w) xcur = finish(wnode + ke0 * S, wi, wj, ke0, owned_at(ke0), raw0);
  R carry = R(0);
  for (int ke = ke0; ke < ke1; ++ke) {
    // eigenvalues of this layer's element: from registers loaded now (used in
    // stage 3), or built in stage 3 from the staged element data
    R l8[8];
    if (!LAM_STAGED && has_e) lam(welem + ke * Se, nullptr, l8);
    // stage 1: next layer (already staged), z-direction Hadamard per window column
    cp_async_wait<0>();
    R* rnext = ((ke + 1 - ke0) & 1) ? raw1 : raw0;
    R* rfree = ((ke - ke0) & 1) ? raw1 : raw0;
    const R lo = xcur;
    if (has_w) {
      const R hi = finish(wnode + (ke + 1) * S, wi, wj, ke + 1, owned_at(ke + 1), rnext);
      if (ke + 2 <= ke1) fetch(wnode + (ke + 2) * S, wi, wj, ke + 2, owned_at(ke + 2), rfree);
      xcur = hi;
      sm.Z[0][wlj][wli] = lo + hi;
      sm.Z[1][wlj][wli] = lo - hi;
    }
    if (LAM_STAGED && has_e) {
      lam(welem + ke * Se, rnext + LSLOT * NT, l8);
      if (ke + 1 < ke1) lam_fetch(welem + (ke + 1) * Se, rfree + LSLOT * NT);
    }
    cp_async_commit();
    __syncthreads();
    // stage 2: y-direction per element row and node column
    if (has_r) {
#pragma unroll
      for (int z = 0; z < 2; ++z) {
        R a = sm.Z[z][wlj][wli], b = sm.Z[z][wlj + 1][wli];
        sm.Y[2 * z][wlj][wli] = a + b;
        sm.Y[2 * z + 1][wlj][wli] = a - b;
      }
    }
    __syncthreads();
    // stage 3: per element, x-direction, eigenvalue scaling and x-backward in
    // one step: with the pair form c = lam_even + lam_odd, d = lam_even - lam_odd,
    // left = lam_even (a + b) + lam_odd (a - b) = c a + d b, right = d a + c b
    if (has_e) {
#pragma unroll
      for (int m4 = 0; m4 < 4; ++m4) {
        R a = sm.Y[m4][ely][elx], b = sm.Y[m4][ely][elx + 1];
        sm.XL[m4][ely][elx] = fma(l8[2 * m4], a, l8[2 * m4 + 1] * b);
        sm.XR[m4][ely][elx] = fma(l8[2 * m4 + 1], a, l8[2 * m4] * b);
      }
    }
    __syncthreads();
    // stage 4: gather x-backward per node column, y-backward
    if (has_r) {
      R B[4];
#pragma unroll
      for (int m4 = 0; m4 < 4; ++m4) {
        R v = wli < ex ? sm.XL[m4][wlj][wli] : R(0);
        if (wli > 0) v += sm.XR[m4][wlj][wli - 1];
        B[m4] = v;
      }
#pragma unroll
      for (int z = 0; z < 2; ++z) {
        sm.yb.L[z][wlj][wli] = B[2 * z] + B[2 * z + 1];
        sm.yb.H[z][wlj][wli] = B[2 * z] - B[2 * z + 1];
      }
    }
    __syncthreads();
    // stage 5: gather y-backward per node column, z-backward, emit layer ke
    if (has_w) {
      R C0 = wlj < ey ? sm.yb.L[0][wlj][wli] : R(0);
      R C1 = wlj < ey ? sm.yb.L[1][wlj][wli] : R(0);
      if (wlj > 0) {
        C0 += sm.yb.H[0][wlj - 1][wli];
        C1 += sm.yb.H[1][wlj - 1][wli];
      }
      emit(wnode + ke * S, wslot, carry + (C0 + C1), lo);
      carry = C0 - C1;
    }
  }
  // top node layer of the tile: only the contributions of element layer ke1-1
  if (has_w) emit(wnode + ke1 * S, wslot | (ke1 < g.nz ? 4 : 0), carry, xcur);
  cp_async_wait<0>();
  __syncthreads();
}

// Staging helpers for plain inputs: one array value per node.
template <typename R, typename T>
struct StageArray {
  const T* src;
  __device__ void operator()(int n, int, int, int, bool, R* raw) const {
    cp_async<sizeof(T)>(raw, src + n);
  }
};
template <typename R, typename T>
struct FinishArray {
  __device__ R operator()(int, int, int, int, bool, const R* raw) const {
    return (R)(*reinterpret_cast<const T*>(raw));
  }
};

// Which exchange partials a node's owner adds (the tile boundaries it lies
// on): bit 0 low-x, bit 1 low-y, bit 2 low-z of the owning tile.  Tile widths
// in x and y are powers of two whenever there is more than one tile.
__device__ inline int low_faces(const Grid3& g, const Tiling& t, int i, bool ly, bool lz) {
  const bool lx = t.ntx > 1 && i > 0 && i < g.nx && (i & (t.ex - 1)) == 0;
  return (lx ? 1 : 0) | (ly ? 2 : 0) | (lz ? 4 : 0);
}

// Full nodal value: own partial plus the neighbours' exchange partials, fixed order.
template <typename R>
__device__ inline R gather_partials(const R* prim, const R* X, int nn, int n, int lf) {
  R v = __ldcg(prim + n);
  if (lf) {
    const size_t xs = xplane(nn);
    if (lf & 1) v += __ldcg(X + 0 * xs + n);
    if (lf & 2) v += __ldcg(X + 1 * xs + n);
    if ((lf & 3) == 3) v += __ldcg(X + 2 * xs + n);
    if (lf & 4) v += __ldcg(X + 3 * xs + n);
    if ((lf & 5) == 5) v += __ldcg(X + 4 * xs + n);
    if ((lf & 6) == 6) v += __ldcg(X + 5 * xs + n);
    if (lf == 7) v += __ldcg(X + 6 * xs + n);
  }
  return v;
}

template <typename R>
__device__ inline void store_partial(R* prim, R* X, int nn, int n, int slot, R v, bool add) {
  R* dst = slot == 0 ? prim + n : X + (size_t)(slot - 1) * xplane(nn) + n;
  if (add) v += *dst;
  *dst = v;
}

// Element box of a tile: [ie0, ie0 + ex) x [je0, je0 + ey), and whether its
// element layers reach the plate top.
struct TileBox {
  int ie0, je0, ex, ey;
  bool top;
};
__device__ inline TileBox tile_box(const Grid3& g, const Tiling& t, int tile) {
  const int txy = t.ntx * t.nty;
  const int tiz = tile / txy, trem = tile - tiz * txy;
  const int tiy = trem / t.ntx, tix = trem - tiy * t.ntx;
  const int ie0 = tix * t.ex, je0 = tiy * t.ey;
  return TileBox{ie0, je0, min(t.ex, g.nx - ie0), min(t.ey, g.ny - je0), min(tiz * t.ez + t.ez, g.nz) == g.nz};
}

// Whether the node window of a tile (its elements' nodes) holds a node of one
// of the Dirichlet sets.
__device__ inline bool tile_touches_dirichlet(const Grid3& g, const Tiling& t, int tile, const DirSpec& d) {
  const int txy = t.ntx * t.nty;
  const int tiz = tile / txy, trem = tile - tiz * txy;
  const int tiy = trem / t.ntx, tix = trem - tiy * t.ntx;
  const int i0 = tix * t.ex, j0 = tiy * t.ey, k0 = tiz * t.ez;
  const int i1 = min(i0 + t.ex, g.nx), j1 = min(j0 + t.ey, g.ny), k1 = min(k0 + t.ez, g.nz);
  if (((d.faces & 1) && i0 == 0) || ((d.faces & 2) && i1 == g.nx) || ((d.faces & 4) && j0 == 0) ||
      ((d.faces & 8) && j1 == g.ny) || ((d.faces & 16) && k0 == 0))
    return true;
  return d.box[0] <= i1 && d.box[1] >= i0 && d.box[2] <= j1 && d.box[3] >= j0 && d.box[4] <= k1 && d.box[5] >= k0 &&
         d.box[0] <= d.box[1] && d.box[2] <= d.box[3] && d.box[4] <= d.box[5];
}

// The right-hand side's tiles of one block, at most RHS_ROUNDS of them
// (ntiles <= RHS_ROUNDS nblk): the tiles are ranked with the ones that touch
// Dirichlet nodes first (in tile order), then the others, and rank p goes to
// round p / nblk and, in even rounds, to block p % nblk, in odd rounds to
// block nblk - 1 - p % nblk.  Returns the block's shared list indexed by
// round (-1: no tile in that round).  All threads of the block call it; each
// scans a contiguous chunk of the tiles twice (count, then place) around one
// block-wide prefix sum of the counts.
constexpr int RHS_ROUNDS = 8;
__device__ inline int* rhs_items(const Grid3& g, const Tiling& t, const DirSpec& d, int ntiles, const VGrid& vg) {
  __shared__ int items[RHS_ROUNDS];
  __shared__ int wsum[NT / 32 + 1];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
  const int chunk = (ntiles + blockDim.x - 1) / blockDim.x;
  const int c0 = min(tid * chunk, ntiles), c1 = min(c0 + chunk, ntiles);
  int cnt = 0;
  for (int tile = c0; tile < c1; ++tile) cnt += tile_touches_dirichlet(g, t, tile, d) ? 1 : 0;
  // block-wide exclusive prefix sum of cnt (warp scans, then the warp totals)
  int incl = cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (tid < RHS_ROUNDS) items[tid] = -1;
  if (lane == 31) wsum[warp] = incl;
  __syncthreads();
  int before = 0, nd = 0;
  for (int w = 0; w < nwarps; ++w) {
    if (w < warp) before += wsum[w];
    nd += wsum[w];
  }
  int rd = before + incl - cnt;  // rank of the chunk's first Dirichlet tile
  int ri = nd + (c0 - (before + incl - cnt));  // position of its first other tile
  for (int tile = c0; tile < c1; ++tile) {
    const int p = tile_touches_dirichlet(g, t, tile, d) ? rd++ : ri++;
    const int round = p / vg.nblk, off = p - round * vg.nblk;
    if (((round & 1) ? vg.nblk - 1 - off : off) == vg.bid) items[round] = tile;
  }
  __syncthreads();
  return items;
}

// Top-surface transfer term of one tile (the Robin condition of Section 3.1):
// for every node of the tile's window on the plate's top layer, the tile's
// share sum over its top faces f next to the node of
// h_f sum_b Mf[a, b] x_b, Mf = M1x (x) M1y the consistent surface mass of the
// bilinear face hats, added to the partial the tile's apply emitted for that
// node (own or exchange slot, as the apply chose).  Returns the share of
// <x, H x>.  Called after the tile's apply with all threads of the block.
template <typename R, typename XT, typename HT>
__device__ R surface_partials(const Grid3& g, const TileBox& b, const XT* x, const HT* hf, const double (&mfx)[2],
                              const double (&mfy)[2], R* q, R* X) {
  const int wx = b.ex + 1, nwin = wx * (b.ey + 1);
  const int nn = g.nnx * g.nny * g.nnz;
  const int top = g.nnx * g.nny * g.nz;
  const R mx[2] = {(R)mfx[0], (R)mfx[1]}, my[2] = {(R)mfy[0], (R)mfy[1]};
  R vd = R(0);
  for (int w = threadIdx.x; w < nwin; w += blockDim.x) {
    const int wj = w / wx, wi = w - wj * wx;
    const int i = b.ie0 + wi, j = b.je0 + wj;
    R acc = R(0);
    for (int je = max(j - 1, b.je0); je <= min(j, b.je0 + b.ey - 1); ++je)
      for (int ie = max(i - 1, b.ie0); ie <= min(i, b.ie0 + b.ex - 1); ++ie) {
        R sf = R(0);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const int bx = c & 1, by = c >> 1;
          const R wgt = mx[ie + bx == i ? 0 : 1] * my[je + by == j ? 0 : 1];
          sf = fma(wgt, (R)__ldcg(x + top + (ie + bx) + g.nnx * (je + by)), sf);
        }
        acc = fma((R)__ldcg(hf + ie + g.nx * je), sf, acc);
      }
    const int n = top + i + g.nnx * j;
    const int slot = ((wi == b.ex && b.ie0 + b.ex < g.nx) ? 1 : 0) | ((wj == b.ey && b.je0 + b.ey < g.ny) ? 2 : 0);
    store_partial(q, X, nn, n, slot, acc, true);
    vd = fma((R)__ldcg(x + n), acc, vd);
  }
  __syncthreads();
  return vd;
}

// Row of the surface operator at top node (i, j) applied to v - shift (all
// faces next to the node), in FP64.
__device__ inline double surface_row(const Grid3& g, const double* hf, const double (&mfx)[2], const double (&mfy)[2],
                                     int i, int j, const double* T, const double* u, double shift) {
  const int top = g.nnx * g.nny * g.nz;
  double acc = 0.0;
  for (int je = max(j - 1, 0); je <= min(j, g.ny - 1); ++je)
    for (int ie = max(i - 1, 0); ie <= min(i, g.nx - 1); ++ie) {
      double sf = 0.0;
      for (int c = 0; c < 4; ++c) {
        const int bx = c & 1, by = c >> 1;
        const int nb = top + (ie + bx) + g.nnx * (je + by);
        const double v = (u ? __ldcg(T + nb) + __ldcg(u + nb) : __ldcg(T + nb)) - shift;
        sf = fma(mfx[ie + bx == i ? 0 : 1] * mfy[je + by == j ? 0 : 1], v, sf);
      }
      acc = fma(__ldcg(hf + ie + g.nx * je), sf, acc);
    }
  return acc;
}

// floor(n / d) for 0 <= n < 2^31 and a runtime divisor d >= 1, as the high
// 64 bits of n * M with M = floor(2^64 / d) + 1 (M = 2^64 / d when d is a
// power of two): the error n (d - 2^64 mod d) / (d 2^64) < 1/d cannot carry
// the quotient past an integer.  div_magic(d) computes M; d = 1 returns n.
__device__ inline unsigned long long div_magic(int d) {
  return d == 1 ? 0ull : ~0ull / (unsigned long long)d + 1ull;
}
__device__ inline int div_by(int n, int d, unsigned long long M) {
  return d == 1 ? n : (int)__umul64hi((unsigned long long)n, M);
}

// Grid-wide loop over the nodes, flat (thread gtid takes nodes gtid, gtid +
// gstride, ...): every lane has a node in every step (rows of nnx = 32 m + 1
// nodes taken by warps would leave one lane busy in every fifth step).
// body(n, i, j, k, ly, lz) with the node's low tile-face flags in y and z.
struct NodeIx {
  int i, j, k;
  bool ly, lz;  // on a low tile face in y / z
};
struct NodeDiv {
  unsigned long long mx, my, mz;
  __device__ NodeDiv(const Grid3& g, const Tiling& t)
      : mx(div_magic(g.nnx)), my(div_magic(g.nny)), mz(div_magic(t.ez)) {}
  __device__ NodeIx operator()(const Grid3& g, const Tiling& t, int n) const {
    NodeIx x;
    const int row = div_by(n, g.nnx, mx);
    x.i = n - row * g.nnx;
    x.k = div_by(row, g.nny, my);
    x.j = row - x.k * g.nny;
    x.ly = t.nty > 1 && x.j > 0 && x.j < g.ny && (x.j & (t.ey - 1)) == 0;
    x.lz = x.k > 0 && x.k < g.nz && x.k - div_by(x.k, t.ez, mz) * t.ez == 0;
    return x;
  }
};
template <class Body>
__device__ inline void for_nodes(const Grid3& g, const Tiling& t, const VGrid& vg, Body body) {
  const int nn = g.nnx * g.nny * g.nnz;
  const NodeDiv nd(g, t);
  for (int n = vg.bid * blockDim.x + threadIdx.x; n < nn; n += vg.nblk * blockDim.x) {
    const NodeIx x = nd(g, t, n);
    body(n, x.i, x.j, x.k, x.ly, x.lz);
  }
}
// Loads of a node pass batched: thread gtid takes the nodes gtid, gtid +
// gstride, ... (the order of for_nodes) NODE_BATCH at a time, first
// v = load(n, x) for all of them (the loads of one node do not wait for
// another's stores; v is a small struct kept in registers), then store(n, v)
// in node order.  NB = 1 is the plain loop (the batched kernel, whose
// register budget is tighter, measured slower with four).
constexpr int NODE_BATCH = 4;
template <int NB, class Load, class Store>
__device__ inline void for_nodes_batched(const Grid3& g, const Tiling& t, const VGrid& vg, Load load, Store store) {
  using V = decltype(load(0, NodeIx{}));
  const int nn = g.nnx * g.nny * g.nnz;
  const NodeDiv nd(g, t);
  const int gstride = vg.nblk * blockDim.x;
  for (int n0 = vg.bid * blockDim.x + threadIdx.x; n0 < nn; n0 += NB * gstride) {
    V v[NB];
#pragma unroll
    for (int m = 0; m < NB; ++m) {
      const int n = n0 + m * gstride;
      if (n < nn) v[m] = load(n, nd(g, t, n));
    }
#pragma unroll
    for (int m = 0; m < NB; ++m) {
      const int n = n0 + m * gstride;
      if (n < nn) store(n, v[m]);
    }
  }
}

// Same for elements rows (je, ke): body(e, ie, je, ke).
template <class Body>
__device__ inline void for_elems(const Grid3& g, const VGrid& vg, Body body) {
  const int lane = threadIdx.x & 31;
  const int wg = (vg.bid * blockDim.x + threadIdx.x) >> 5;
  const int nwg = (vg.nblk * blockDim.x) >> 5;
  const int rows = g.ny * g.nz;
  for (int row = wg; row < rows; row += nwg) {
    const int ke = row / g.ny, je = row - ke * g.ny;
    const int base = row * g.nx;
    for (int ie = lane; ie < g.nx; ie += 32) body(base + ie, ie, je, ke);
  }
}

enum RedSlot { RS_RZ0 = 0, RS_BB = 1, RS_PQ = 2, RS_RZ = 3, RS_RR = 4, RS_ES = 5, RS_EL = 6, RS_EF = 7, RS_EX = 8,
               RS_N = 9 };

// Buffers of one preconditioned CG on the free nodes.  Arrays that a tile
// reads on its whole window while owners update them are double-buffered by
// pass parity.
template <typename R>
struct CGBufs {
  R* x;      // solution, updated in place by the owners
  R* r[2];   // residual
  R* p[2];   // search direction
  R* s[2];   // s = A p, kept by recurrence
  R* q[2];   // own partial of w = A u
  R* X[2];   // exchange partials of w
  const R* dinv;
  const R* lam;
};

// Jacobi-preconditioned CG in the single-reduction form of Chronopoulos and
// Gear: with u = D^-1 r and w = A u,
//   p = u + beta p,  s = w + beta s,  x += alpha p,  r -= alpha s,
//   gamma = <r, u>, delta = <w, u>, beta = gamma / gamma_old,
//   alpha = gamma / (delta - beta gamma / alpha_old),
// so each iteration needs one apply and one grid reduction.  Every tile
// applies the vector update to its whole window on the fly (owners write it
// back) and feeds the new u straight into the apply: one grid barrier per
// iteration.  Starts from the residual in c.r[0] with <r,r> = rr0; stops when
// <r, r> <= thresh or after max_iter iterations.  Returns 1 converged, 0
// capped, -1 barrier failure; *iters gets the count.
template <typename R, bool LAM_STAGED, int NS, class LamFetch, class Lam>
__device__ int pcg1(const SolveArgs& a, const VGrid& vg, ApplySmem<R>& sm, R* stage, const CGBufs<R>& c,
                    LamFetch lam_fetch, Lam lam8, R thresh, int max_iter, R* red, int* iters, Tracer& tr) {
  R* s_scal = red_scalars<R>();  // broadcast of the step scalars
  const Grid3 g = a.g;
  const Tiling t = a.t;
  const int nn = g.nnx * g.nny * g.nnz;
  const int ntiles = t.ntx * t.nty * t.ntz;
  R alpha = R(0), beta = R(0), gamma = R(0);
  int it = 0;
  bool conv = false;
  // pass -1: w_0 = A u_0 (no update); passes k >= 0 update then apply w_{k+1}
  for (int k = -1; k < max_iter; ++k) {
    const int cur = k < 0 ? 0 : (k & 1), nxt = k < 0 ? 0 : (cur ^ 1);
    const bool first = k == 0;
    // reduction rows alternate by pass (see pcg2)
    R* rslots = red + (((k + 1) & 1) ? RS_ES : RS_PQ) * a.red_stride;
    // pass pointers chosen by selects (no dynamic indexing into the struct)
    const R* r_cur = cur ? c.r[1] : c.r[0];
    const R* p_cur = cur ? c.p[1] : c.p[0];
    const R* s_cur = cur ? c.s[1] : c.s[0];
    const R* q_cur = cur ? c.q[1] : c.q[0];
    const R* X_cur = cur ? c.X[1] : c.X[0];
    R* r_nxt = nxt ? c.r[1] : c.r[0];
    R* p_nxt = nxt ? c.p[1] : c.p[0];
    R* s_nxt = nxt ? c.s[1] : c.s[0];
    R* q_out = (k >= 0 && nxt) ? c.q[1] : c.q[0];
    R* X_out = (k >= 0 && nxt) ? c.X[1] : c.X[0];
    const size_t xs = xplane(nn);
    R sg = R(0), vd = R(0), vr = R(0);
    for (int tile = vg.bid; tile < ntiles; tile += vg.nblk) {
      // raw inputs of a window node: 0 dinv, 1 r, 2 own partial of w, 3 p, 4 s,
      // 5..11 the neighbours' partials of w (only on tile faces), 12 x (owner)
      auto fetch = [&](int n, int i, int j, int kk, bool owned, R* raw) {
        if (is_dir(g, a.dir, i, j, kk)) return;
        cp_async<sizeof(R)>(raw, c.dinv + n);
        cp_async<sizeof(R)>(raw + NT, r_cur + n);
        if (k < 0) return;
        cp_async<sizeof(R)>(raw + 2 * NT, q_cur + n);
        if (owned) cp_async<sizeof(R)>(raw + 12 * NT, c.x + n);
        if (!first) {
          cp_async<sizeof(R)>(raw + 3 * NT, p_cur + n);
          cp_async<sizeof(R)>(raw + 4 * NT, s_cur + n);
        }
        const bool ly = t.nty > 1 && j > 0 && j < g.ny && (j & (t.ey - 1)) == 0;
        const bool lz = kk > 0 && kk < g.nz && (kk % t.ez) == 0;
        const int lf = low_faces(g, t, i, ly, lz);
        if (lf) {
          if (lf & 1) cp_async<sizeof(R)>(raw + 5 * NT, X_cur + 0 * xs + n);
          if (lf & 2) cp_async<sizeof(R)>(raw + 6 * NT, X_cur + 1 * xs + n);
          if ((lf & 3) == 3) cp_async<sizeof(R)>(raw + 7 * NT, X_cur + 2 * xs + n);
          if (lf & 4) cp_async<sizeof(R)>(raw + 8 * NT, X_cur + 3 * xs + n);
          if ((lf & 5) == 5) cp_async<sizeof(R)>(raw + 9 * NT, X_cur + 4 * xs + n);
          if ((lf & 6) == 6) cp_async<sizeof(R)>(raw + 10 * NT, X_cur + 5 * xs + n);
          if (lf == 7) cp_async<sizeof(R)>(raw + 11 * NT, X_cur + 6 * xs + n);
        }
      };
      auto finish = [&](int n, int i, int j, int kk, bool owned, const R* raw) -> R {
        if (is_dir(g, a.dir, i, j, kk)) return R(0);
        const R dv = raw[0];
        const R rk = raw[NT];
        if (k < 0) {
          const R u = dv * rk;
          if (owned) {
            sg = fma(rk, u, sg);
            vr = fma(rk, rk, vr);
          }
          return u;
        }
        const bool ly = t.nty > 1 && j > 0 && j < g.ny && (j & (t.ey - 1)) == 0;
        const bool lz = kk > 0 && kk < g.nz && (kk % t.ez) == 0;
        const int lf = low_faces(g, t, i, ly, lz);
        R w = raw[2 * NT];  // neighbours' partials added in the order gather_partials uses
        if (lf) {
          if (lf & 1) w += raw[5 * NT];
          if (lf & 2) w += raw[6 * NT];
          if ((lf & 3) == 3) w += raw[7 * NT];
          if (lf & 4) w += raw[8 * NT];
          if ((lf & 5) == 5) w += raw[9 * NT];
          if ((lf & 6) == 6) w += raw[10 * NT];
          if (lf == 7) w += raw[11 * NT];
        }
        const R u = dv * rk;
        R pv = u, sv = w;
        if (!first) {
          pv = fma(beta, raw[3 * NT], u);
          sv = fma(beta, raw[4 * NT], w);
        }
        const R rn = fma(-alpha, sv, rk);
        const R un = dv * rn;
        if (owned) {
          p_nxt[n] = pv;
          s_nxt[n] = sv;
          r_nxt[n] = rn;
          c.x[n] = fma(alpha, pv, raw[12 * NT]);
          sg = fma(rn, un, sg);
          vr = fma(rn, rn, vr);
        }
        return un;
      };
      auto emit = [&](int n, int slot, R y, R xin) {
        store_partial(q_out, X_out, nn, n, slot, y, false);
        vd = fma(xin, y, vd);
      };
      apply_tile<R, LAM_STAGED, NS>(g, t, tile, sm, stage, fetch, finish, lam_fetch, lam8, emit);
    }
    tr.mark(TR_CG_APPLY);
    {
      R v[3] = {sg, vd, vr};
      block_reduce_store<3>(v, rslots, a.red_stride, vg);
    }
    R tot[3];
    if (!grid_sync_total<3>(a.bar, vg, rslots, a.red_stride, tot)) return -1;
    tr.mark(TR_CG_PASS);
    tr.value(TR_RR, (double)tot[2]);
    if (k >= 0) {
      ++it;
      if (tot[2] <= thresh) {
        conv = true;
        break;
      }
    }
    // next scalars, once per block
    if (threadIdx.x == 0) {
      const R gn = tot[0], dn = tot[1];
      R b = k < 0 ? R(0) : gn / gamma;
      R den = k < 0 ? dn : dn - b * gn / alpha;
      s_scal[0] = gn / den;
      s_scal[1] = b;
      s_scal[2] = (den > R(0) && gn > R(0)) ? R(1) : R(0);
    }
    __syncthreads();
    if (s_scal[2] == R(0)) {  // breakdown (no further progress possible): stop
      tr.value(TR_BREAK, (double)tot[1]);
      break;
    }
    gamma = tot[0];
    alpha = s_scal[0];
    beta = s_scal[1];
    __syncthreads();
  }
  *iters = it;
  // the converged residual sits in r[it & 1]; callers read it from there
  return conv ? 1 : 0;
}

// ---------------------------------------------------------------------------
// FP32 apply for large patches.  Tiles of up to AX x AY x ez elements; warp w
// of a block handles window node row w (w <= ey) and, for w < ey, element row
// w; lane l handles window columns 2l and 2l + 1 and the two elements that
// start there (lane 31 also column AX).  Within a row the x-direction stays in
// registers, warp shuffles and shared memory, the neighbouring node row
// passes through shared memory, and an element layer takes two block
// barriers.  Inputs arrive by cp.async two layers ahead in a four-stage ring
// of dense layers (each thread reads its pairs with 8-byte loads): the window
// values by their owners, 4 bytes a column (window rows do not start on 16
// bytes), the element data by 128 threads, 16 bytes each (zero-filled past
// the tile), which keeps the copies per thread and layer at 3 instead of 7:
// the pass is bound by issuing memory instructions, not by bytes.  Partials
// of window nodes on the tile's high faces go to the exchange arrays, as with
// apply_tile.
// ---------------------------------------------------------------------------
constexpr int AX = 64, AY = 4;
constexpr int WSTAGES = 4;
constexpr int WUX = AX + 4;  // a staged window row: AX + 1 values, padded to 16 bytes
struct WideStage {
  float u[AY + 1][WUX];      // window node values of one node layer
  float sk[2][AY][AX];       // s_e and k_e of one element layer
};
static_assert(NT == 32 * (AY + 1), "one warp per window row");
static_assert(2 * AY * AX / 4 <= NT, "one 16-byte element copy per thread");
static_assert(sizeof(WideStage) % 16 == 0, "16-byte aligned stages");
static_assert(WSTAGES * sizeof(WideStage) <= STAGE_BYTES, "staging ring fits the dynamic shared memory");

// 16-byte asynchronous copy (L2 only) of which the first src_bytes are read
// and the rest zero-filled.
__device__ inline void cp_async16_fill(void* smem, const void* gmem, int src_bytes) {
  const unsigned int sa = (unsigned int)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(sa), "l"(gmem), "r"(src_bytes) : "memory");
}
// 4-byte asynchronous copy with zero fill (src_bytes 0 or 4).
__device__ inline void cp_async4_fill(void* smem, const void* gmem, int src_bytes) {
  const unsigned int sa = (unsigned int)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(sa), "l"(gmem), "r"(src_bytes) : "memory");
}

struct WideSmem {
  float ZS[AY + 1][AX + 2];   // z-sum and z-difference of each window column (current layer pair)
  float ZD[AY + 1][AX + 2];
  float R1s[AY][AX + 2];      // y-backward of element row w to node row w + 1 (z-sum / z-difference)
  float R1d[AY][AX + 2];
};

struct WideCoef {
  float mp[8], kp[8];  // eigenvalue factors (pair form) of the mass and stiffness parts
};

// One wide tile of w = A z for the two-phase CG: stores the partials (own and
// exchange) in q / X and returns the tile's sum of z_n times its partials.
// Not inlined: the tile loop gets the kernel's whole register budget.
// Per element layer a thread does: one cp.async group for the layer two
// ahead (inputs of invalid columns and elements are zeroed once per tile),
// the z-direction of its columns, a block barrier, the y- and x-direction of
// its two elements with the eigenvalue scaling (the next column's values
// come from shared memory, so lane 31 needs no special case), the backward
// x- and y-direction (the next lane's column by shuffle, the next row by
// shared memory), a block barrier, the z-backward and the stores.
static __device__ __noinline__ float apply_wide_partials(const Grid3 g, const Tiling t, int tile, WideSmem* smp,
                                                         float* ring, const float* z, const float* sk,
                                                         const WideCoef cf, float* q, float* X) {
  constexpr unsigned FULL = 0xffffffffu;
  WideSmem& sm = *smp;
  const int lane = threadIdx.x & 31, wy = threadIdx.x >> 5;
  const int txy = t.ntx * t.nty;
  const int tiz = tile / txy, trem = tile - tiz * txy;
  const int tiy = trem / t.ntx, tix = trem - tiy * t.ntx;
  const int ie0 = tix * AX, je0 = tiy * AY, ke0 = tiz * t.ez;
  const int ex = min(AX, g.nx - ie0), ey = min(AY, g.ny - je0), ke1 = min(ke0 + t.ez, g.nz);
  const int S = g.nnx * g.nny, Se = g.nx * g.ny, ne = Se * g.nz, nn = S * g.nnz;
  const bool row_on = wy <= ey;                 // this warp has a window node row
  const bool has_el = wy < ey;                  // ... and an element row
  const int c0 = 2 * lane, c1 = c0 + 1;
  const bool v0 = row_on && c0 <= ex, v1 = row_on && c1 <= ex;
  const bool vx = row_on && lane == 31 && ex == AX;  // column AX
  const int nb = ie0 + g.nnx * (je0 + (row_on ? wy : 0));
  const float* up = z + nb;  // node (ie0, row, 0)
  // exchange slots: the tile's high-y node row; column AX is on the high-x
  // face only when another tile follows in x (a ragged last column is the
  // plate's own boundary); the top node layer adds the high-z bit
  const int ys = (wy == ey && je0 + ey < g.ny) ? 2 : 0;
  const int sx = ys | ((ie0 + AX < g.nx) ? 1 : 0);
  float* o01 = (ys ? X + (size_t)(ys - 1) * xplane(nn) : q) + nb;
  float* ox = (sx ? X + (size_t)(sx - 1) * xplane(nn) : q) + nb + AX;
  WideStage* ws = reinterpret_cast<WideStage*>(ring);
  // the thread's element copy: array ea (s or k), row er, columns 4 ec .. 4 ec + 3
  const int ea = threadIdx.x >> 6, er = (threadIdx.x >> 4) & 3, ec = threadIdx.x & 15;
  const bool ecopy = threadIdx.x < 2 * AY * AX / 4;
  const int evalid = (ecopy && er < ey) ? max(0, min(4, ex - 4 * ec)) : 0;  // columns inside the tile
  const float* eg = sk + (size_t)ea * ne + ie0 + 4 * ec + (size_t)g.nx * (je0 + er);
  // 16-byte copies need 16-byte element rows (nx a multiple of 4, aligned base)
  const bool e16 = (g.nx & 3) == 0 && ((reinterpret_cast<uintptr_t>(sk) & 15) == 0);
#pragma unroll
  for (int st = 0; st < WSTAGES; ++st) {
    if (!v0) ws[st].u[wy][c0] = 0.0f;
    if (!v1) ws[st].u[wy][c1] = 0.0f;
    if (lane == 31 && !vx) ws[st].u[wy][AX] = 0.0f;
  }
  auto issue = [&](int st) {  // stage st: z at node layer ke0 + st, s/k at element layer ke0 + st
    WideStage& w = ws[st & (WSTAGES - 1)];
    const int kn = ke0 + st;
    if (kn <= ke1) {
      const float* ub = up + (size_t)S * kn;
      if (v0) cp_async<4>(&w.u[wy][c0], ub + c0);
      if (v1) cp_async<4>(&w.u[wy][c1], ub + c1);
      if (vx) cp_async<4>(&w.u[wy][AX], ub + AX);
    }
    if (kn < ke1 && ecopy) {
      float* dst = &w.sk[ea][er][4 * ec];
      const float* src = eg + (size_t)Se * kn;
      if (e16) {
        cp_async16_fill(dst, evalid ? src : sk, 4 * evalid);
      } else {
#pragma unroll
        for (int m = 0; m < 4; ++m) cp_async4_fill(dst + m, m < evalid ? src + m : sk, m < evalid ? 4 : 0);
      }
    }
    cp_async_commit();
  };
  issue(0);
  issue(1);
  issue(2);
  cp_async_wait<2>();
  float uL0 = ws[0].u[wy][c0], uL1 = ws[0].u[wy][c1], uL2 = lane == 31 ? ws[0].u[wy][AX] : 0.0f;
  float carry0 = 0.0f, carry1 = 0.0f, carry2 = 0.0f;
  float vd = 0.0f;
  for (int ke = ke0; ke < ke1; ++ke) {
    const int j = ke - ke0;
    issue(j + 3);
    cp_async_wait<2>();  // the thread's copies of stages j and j + 1 have landed
    const WideStage& wc = ws[j & (WSTAGES - 1)];
    const WideStage& wn = ws[(j + 1) & (WSTAGES - 1)];
    const float2 uH = *reinterpret_cast<const float2*>(&wn.u[wy][c0]);
    const float uH0 = uH.x, uH1 = uH.y, uH2 = lane == 31 ? wn.u[wy][AX] : 0.0f;  // column AX: lane 31 only
    // z-direction per own column
    const float zs0 = uL0 + uH0, zs1 = uL1 + uH1, zs2 = uL2 + uH2;
    const float zd0 = uL0 - uH0, zd1 = uL1 - uH1, zd2 = uL2 - uH2;
    if (row_on) {
      *reinterpret_cast<float2*>(&sm.ZS[wy][c0]) = make_float2(zs0, zs1);
      *reinterpret_cast<float2*>(&sm.ZD[wy][c0]) = make_float2(zd0, zd1);
      if (lane == 31) {
        sm.ZS[wy][AX] = zs2;
        sm.ZD[wy][AX] = zd2;
      }
    }
    __syncthreads();
    // elements of row wy: y-forward, x-direction with scaling, y-backward
    float r0s0 = 0.0f, r0s1 = 0.0f, r0s2 = 0.0f, r0d0 = 0.0f, r0d1 = 0.0f, r0d2 = 0.0f;
    if (has_el) {
      // element data of the thread's two elements (copied by other threads:
      // read after the block barrier)
      const float2 sv = *reinterpret_cast<const float2*>(&wc.sk[0][wy][c0]);
      const float2 kv = *reinterpret_cast<const float2*>(&wc.sk[1][wy][c0]);
      const float2 ns = *reinterpret_cast<const float2*>(&sm.ZS[wy + 1][c0]);
      const float2 nd = *reinterpret_cast<const float2*>(&sm.ZD[wy + 1][c0]);
      const float s2 = sm.ZS[wy][c0 + 2], d2 = sm.ZD[wy][c0 + 2];
      const float ns2 = sm.ZS[wy + 1][c0 + 2], nd2 = sm.ZD[wy + 1][c0 + 2];
      // packed FP32 pairs (the same operations as one column at a time):
      // columns (c0, c1) of the (y, z) modes, and per mode m4 the eigenvalue
      // pairs (la, mb), (lb, ma) and the x-results of columns (c0, c0 + 2)
      const float2 M1 = make_float2(-1.0f, -1.0f);
      const float2 S0 = make_float2(zs0, zs1), D0 = make_float2(zd0, zd1);
      const float2 Yp[4] = {__fadd2_rn(S0, ns), __ffma2_rn(ns, M1, S0), __fadd2_rn(D0, nd), __ffma2_rn(nd, M1, D0)};
      const float Ys[4] = {s2 + ns2, s2 - ns2, d2 + nd2, d2 - nd2};
      float2 Be[4];  // (B[m4][c0], B[m4][c0 + 2])
      float Bm[4];   // B[m4][c0 + 1]
#pragma unroll
      for (int m4 = 0; m4 < 4; ++m4) {
        const float2 L1 = __ffma2_rn(sv, make_float2(cf.mp[2 * m4], cf.mp[2 * m4 + 1]),
                                     __fmul2_rn(kv, make_float2(cf.kp[2 * m4], cf.kp[2 * m4 + 1])));  // (la, mb)
        const float2 L2 = __ffma2_rn(sv, make_float2(cf.mp[2 * m4 + 1], cf.mp[2 * m4]),
                                     __fmul2_rn(kv, make_float2(cf.kp[2 * m4 + 1], cf.kp[2 * m4])));  // (lb, ma)
        const float a0 = Yp[m4].x, a1 = Yp[m4].y, a2 = Ys[m4];
        Be[m4] = __ffma2_rn(L1, Yp[m4], __fmul2_rn(L2, make_float2(a1, a2)));
        Bm[m4] = fmaf(L2.x, a0, fmaf(L1.x + L2.y, a1, L1.y * a2));
      }
      const float2 R0S = __fadd2_rn(Be[0], Be[1]), R0D = __fadd2_rn(Be[2], Be[3]);
      const float2 R1S = __ffma2_rn(Be[1], M1, Be[0]), R1D = __ffma2_rn(Be[3], M1, Be[2]);
      float r1s[3], r1d[3];
      r0s0 = R0S.x;
      r0s1 = Bm[0] + Bm[1];
      r0s2 = R0S.y;
      r0d0 = R0D.x;
      r0d1 = Bm[2] + Bm[3];
      r0d2 = R0D.y;
      r1s[0] = R1S.x;
      r1s[1] = Bm[0] - Bm[1];
      r1s[2] = R1S.y;
      r1d[0] = R1D.x;
      r1d[1] = Bm[2] - Bm[3];
      r1d[2] = R1D.y;
      // column 2l + 2 is the next lane's first column (lane 31 keeps it: column AX)
      const float t0 = __shfl_up_sync(FULL, r0s2, 1), t1 = __shfl_up_sync(FULL, r0d2, 1);
      const float t2 = __shfl_up_sync(FULL, r1s[2], 1), t3 = __shfl_up_sync(FULL, r1d[2], 1);
      if (lane > 0) {
        r0s0 += t0;
        r0d0 += t1;
        r1s[0] += t2;
        r1d[0] += t3;
      }
      *reinterpret_cast<float2*>(&sm.R1s[wy][c0]) = make_float2(r1s[0], r1s[1]);
      *reinterpret_cast<float2*>(&sm.R1d[wy][c0]) = make_float2(r1d[0], r1d[1]);
      if (lane == 31) {
        sm.R1s[wy][AX] = r1s[2];
        sm.R1d[wy][AX] = r1d[2];
      }
    }
    __syncthreads();
    // node row wy: own element row plus the row below, then z-backward
    if (row_on) {
      if (wy > 0) {
        const float2 ps = *reinterpret_cast<const float2*>(&sm.R1s[wy - 1][c0]);
        const float2 pd = *reinterpret_cast<const float2*>(&sm.R1d[wy - 1][c0]);
        r0s0 += ps.x;
        r0s1 += ps.y;
        r0d0 += pd.x;
        r0d1 += pd.y;
        if (lane == 31) {
          r0s2 += sm.R1s[wy - 1][AX];
          r0d2 += sm.R1d[wy - 1][AX];
        }
      }
      const float out0 = carry0 + (r0s0 + r0d0), out1 = carry1 + (r0s1 + r0d1), out2 = carry2 + (r0s2 + r0d2);
      carry0 = r0s0 - r0d0;
      carry1 = r0s1 - r0d1;
      carry2 = r0s2 - r0d2;
      const size_t lk = (size_t)S * ke;
      if (v0) {
        o01[lk + c0] = out0;
        vd = fmaf(uL0, out0, vd);
      }
      if (v1) {
        o01[lk + c1] = out1;
        vd = fmaf(uL1, out1, vd);
      }
      if (vx) {
        ox[lk] = out2;
        vd = fmaf(uL2, out2, vd);
      }
    }
    uL0 = uH0;
    uL1 = uH1;
    uL2 = uH2;
  }
  // top node layer of the tile: only the contributions of element layer ke1 - 1
  if (row_on) {
    const size_t top = (size_t)S * ke1;
    const int zb = ke1 < g.nz ? 4 : 0;
    float* t01 = ((ys | zb) ? X + (size_t)((ys | zb) - 1) * xplane(nn) : q) + nb + top;
    float* tx = ((sx | zb) ? X + (size_t)((sx | zb) - 1) * xplane(nn) : q) + nb + AX + top;
    if (v0) {
      t01[c0] = carry0;
      vd = fmaf(uL0, carry0, vd);
    }
    if (v1) {
      t01[c1] = carry1;
      vd = fmaf(uL1, carry1, vd);
    }
    if (vx) {
      tx[0] = carry2;
      vd = fmaf(uL2, carry2, vd);
    }
  }
  cp_async_wait<0>();
  __syncthreads();
  return vd;
}

// Vectors of the two-phase CG (pcg2).  Only owners touch a node in the update
// phase and the apply reads only u, so nothing is double-buffered.
template <typename R>
struct CGVecs {
  R* x;           // solution, updated in place
  R* r;           // residual
  R* p;           // search direction
  R* s;           // s = A p, kept by recurrence
  R* z;           // z = D^-1 r, the apply's input (0 on Dirichlet nodes)
  R* q;           // own partial of w = A u
  R* X;           // NXB exchange arrays of w's partials
  const R* dinv;  // Jacobi inverse diagonal, 0 on Dirichlet nodes
};

template <typename R> struct Vec16;
template <> struct Vec16<float> { using T = float4; };
template <> struct Vec16<double> { using T = double2; };
template <typename R> struct Vec2;  // two values in one access
template <> struct Vec2<float> { using T = float2; };
template <> struct Vec2<double> { using T = double2; };
template <int N> struct VecP;  // N floats in one access
template <> struct VecP<2> { using T = float2; };
template <> struct VecP<4> { using T = float4; };

template <typename R>
struct Sums2 { R a, b; };

// The update phase of the two-phase CG over all nodes, flat: each lane takes
// 16 bytes of every array at once (VEC consecutive nodes, vector loads and
// stores), so every array streams at full line width whatever the row
// length.  The lane's first node gets its (i, j, k) from two exact
// multiply-high divisions, the others by increments.  A node's low tile faces
// decide which exchange partials its owner adds; the x-, y- and z-face
// partials are loaded with the main inputs (an x face falls in every warp's
// 128 nodes, so a dependent load there would stall every step), the edge
// partials afterwards.  k < 0: z = D^-1 r only.
// Dirichlet nodes (dinv = 0) keep their r, p, s, x and get z = 0.  Returns the
// thread's sums of <r,z> and <r,r>.  Not inlined: it gets the kernel's whole
// register budget.
template <typename R>
static __device__ __noinline__ Sums2<R> cg_update(const Grid3 g, const Tiling t, const CGVecs<R> c, R alpha, R beta,
                                                  int k, int gtid, int gstride) {
  using V = typename Vec16<R>::T;
  constexpr int VEC = 16 / sizeof(R);
  const int nn = g.nnx * g.nny * g.nnz;
  const unsigned long long mx = div_magic(g.nnx), my = div_magic(g.nny), mz = div_magic(t.ez);
  const bool init = k < 0, first = k == 0;
  const int ngroups = (nn + VEC - 1) / VEC;
  const size_t xs = xplane(nn);
  R vgam = R(0), vrr = R(0);
  auto load = [&](const R* a, int n0, int cnt, R (&o)[VEC]) {
    if (cnt == VEC) {
      const V v = __ldcg(reinterpret_cast<const V*>(a + n0));
      const R* e = reinterpret_cast<const R*>(&v);
#pragma unroll
      for (int m = 0; m < VEC; ++m) o[m] = e[m];
    } else {
#pragma unroll
      for (int m = 0; m < VEC; ++m) o[m] = m < cnt ? __ldcg(a + n0 + m) : R(0);
    }
  };
  // the preconditioner's FP32 arrays, VEC values at a time (4 B x VEC)
  using VP = typename VecP<VEC>::T;
  auto loadp = [&](const float* a, int n0, int cnt, float (&o)[VEC]) {
    if (cnt == VEC) {
      const VP v = __ldcg(reinterpret_cast<const VP*>(a + n0));
      const float* e = reinterpret_cast<const float*>(&v);
#pragma unroll
      for (int m = 0; m < VEC; ++m) o[m] = e[m];
    } else {
#pragma unroll
      for (int m = 0; m < VEC; ++m) o[m] = m < cnt ? __ldcg(a + n0 + m) : 0.0f;
    }
  };
  auto storep = [&](float* a, int n0, int cnt, const float (&o)[VEC]) {
    if (cnt == VEC) {
      VP v;
      float* e = reinterpret_cast<float*>(&v);
#pragma unroll
      for (int m = 0; m < VEC; ++m) e[m] = o[m];
      *reinterpret_cast<VP*>(a + n0) = v;
    } else {
#pragma unroll
      for (int m = 0; m < VEC; ++m)
        if (m < cnt) a[n0 + m] = o[m];
    }
  };
  auto store = [&](R* a, int n0, int cnt, const R (&o)[VEC]) {
    if (cnt == VEC) {
      V v;
      R* e = reinterpret_cast<R*>(&v);
#pragma unroll
      for (int m = 0; m < VEC; ++m) e[m] = o[m];
      *reinterpret_cast<V*>(a + n0) = v;
    } else {
#pragma unroll
      for (int m = 0; m < VEC; ++m)
        if (m < cnt) a[n0 + m] = o[m];
    }
  };
  for (int q = gtid; q < ngroups; q += gstride) {
    const int n0 = q * VEC;
    const int cnt = min(VEC, nn - n0);
    R dv[VEC], rk[VEC];
    load(c.dinv, n0, cnt, dv);
    load(c.r, n0, cnt, rk);
    if (init) {
      R zn[VEC];
#pragma unroll
      for (int m = 0; m < VEC; ++m) {
        zn[m] = dv[m] * rk[m];
        if (dv[m] != R(0)) {
          vgam = fma(rk[m], zn[m], vgam);
          vrr = fma(rk[m], rk[m], vrr);
        }
      }
      store(c.z, n0, cnt, zn);
      continue;
    }
    // low tile faces of the group's nodes: the y and z faces once per row,
    // the x face per node; a group that crosses a row end (or the array end)
    // walks node by node
    int lf[VEC];
    int rowf = -1;  // the group's y / z face bits when it lies in one row, else -1
    {
      const int row = div_by(n0, g.nnx, mx);
      int i = n0 - row * g.nnx;
      int kz = div_by(row, g.nny, my);
      int j = row - kz * g.nny;
      auto row_faces = [&](int jj, int kk) {
        const bool ly = t.nty > 1 && jj > 0 && jj < g.ny && (jj & (t.ey - 1)) == 0;
        const bool lz = kk > 0 && kk < g.nz && kk - div_by(kk, t.ez, mz) * t.ez == 0;
        return (ly ? 2 : 0) | (lz ? 4 : 0);
      };
      if (cnt == VEC && i + VEC <= g.nnx) {
        rowf = row_faces(j, kz);
#pragma unroll
        for (int m = 0; m < VEC; ++m) lf[m] = rowf | low_faces(g, t, i + m, false, false);
      } else {
#pragma unroll
        for (int m = 0; m < VEC; ++m) {
          lf[m] = m < cnt ? (row_faces(j, kz) | low_faces(g, t, i, false, false)) : 0;
          if (++i == g.nnx) {
            i = 0;
            if (++j == g.nny) {
              j = 0;
              ++kz;
            }
          }
        }
      }
    }
    R w[VEC], xk[VEC], pk[VEC], sk[VEC], wy[VEC];
    load(c.q, n0, cnt, w);
    load(c.x, n0, cnt, xk);
    if (!first) {
      load(c.p, n0, cnt, pk);
      load(c.s, n0, cnt, sk);
    } else {
#pragma unroll
      for (int m = 0; m < VEC; ++m) pk[m] = sk[m] = R(0);
    }
    R wx[VEC], wz[VEC];
    if (rowf >= 0) {  // one row: whole-group y / z face partials as vectors
#pragma unroll
      for (int m = 0; m < VEC; ++m) wy[m] = wz[m] = R(0);
      if (rowf & 2) load(c.X + 1 * xs, n0, VEC, wy);
      if (rowf & 4) load(c.X + 3 * xs, n0, VEC, wz);
#pragma unroll
      for (int m = 0; m < VEC; ++m) wx[m] = (lf[m] & 1) ? __ldcg(c.X + 0 * xs + n0 + m) : R(0);
    } else {
#pragma unroll
      for (int m = 0; m < VEC; ++m) {
        wx[m] = (lf[m] & 1) ? __ldcg(c.X + 0 * xs + n0 + m) : R(0);
        wy[m] = (lf[m] & 2) ? __ldcg(c.X + 1 * xs + n0 + m) : R(0);
        wz[m] = (lf[m] & 4) ? __ldcg(c.X + 3 * xs + n0 + m) : R(0);
      }
    }
    R pn[VEC], sn[VEC], rn[VEC], xn[VEC], zn[VEC];
#pragma unroll
    for (int m = 0; m < VEC; ++m) {
      pn[m] = pk[m];
      sn[m] = sk[m];
      rn[m] = rk[m];
      xn[m] = xk[m];
      zn[m] = R(0);
      if (m >= cnt || dv[m] == R(0)) continue;
      const int n = n0 + m;
      const int f = lf[m];
      R wv = w[m];
      if (f) {  // neighbours' partials, in the order gather_partials uses
        if (f & 1) wv += wx[m];
        if (f & 2) wv += wy[m];
        if ((f & 3) == 3) wv += __ldcg(c.X + 2 * xs + n);
        if (f & 4) wv += wz[m];
        if ((f & 5) == 5) wv += __ldcg(c.X + 4 * xs + n);
        if ((f & 6) == 6) wv += __ldcg(c.X + 5 * xs + n);
        if (f == 7) wv += __ldcg(c.X + 6 * xs + n);
      }
      const R z0 = dv[m] * rk[m];
      pn[m] = first ? z0 : fma(beta, pk[m], z0);
      sn[m] = first ? wv : fma(beta, sk[m], wv);
      rn[m] = fma(-alpha, sn[m], rk[m]);
      zn[m] = dv[m] * rn[m];
      xn[m] = fma(alpha, pn[m], xk[m]);
      vgam = fma(rn[m], zn[m], vgam);
      vrr = fma(rn[m], rn[m], vrr);
    }
    store(c.p, n0, cnt, pn);
    store(c.s, n0, cnt, sn);
    store(c.r, n0, cnt, rn);
    store(c.x, n0, cnt, xn);
    store(c.z, n0, cnt, zn);
  }
  return Sums2<R>{vgam, vrr};
}

// The same single-reduction recurrences as pcg1, in two phases per iteration:
//   U  (owners, one pass over the nodes): w = own + neighbours' partials of
//      A u;  p = u + beta p;  s = w + beta s;  x += alpha p;  r -= alpha s;
//      u = D^-1 r;  block sums of <r,u> and <r,r>;
//   A  (tiles): partials of w = A u on each tile's window; block sums of
//      <w,u> (linear in the partials);
// with a grid barrier after each phase and one reduction of the three sums.
// The update streams six inputs and five outputs per node without window
// re-reads, and the apply stages a single input per window node.  Dirichlet
// nodes (dinv = 0) keep r = 0 and u = 0.  Starts from the residual in c.r
// and x = c.x; stops when <r,r> <= thresh or after max_iter iterations.
// Returns 1 converged, 0 capped, -1 barrier failure; *iters gets the count.
// apply_z(tile) applies the operator to c.z on one tile of the tiling t (whose
// faces also decide which exchange partials an owner gathers), stores the
// partials in c.q / c.X and returns the tile's share of <w, z>.
template <typename R, class ApplyZ>
__device__ int pcg2(const SolveArgs& a, const VGrid& vg, const Tiling& t, const CGVecs<R>& c, ApplyZ apply_z,
                    R thresh, int max_iter, R* red, int* iters, Tracer& tr) {
  R* s_scal = red_scalars<R>();  // broadcast of the step scalars
  const Grid3 g = a.g;
  const int ntiles = t.ntx * t.nty * t.ntz;
  R alpha = R(0), beta = R(0), gamma = R(0);
  int it = 0;
  bool conv = false;
  for (int k = -1; k < max_iter; ++k) {
    // reduction rows alternate by iteration: a block that runs ahead into the
    // next iteration never overwrites sums another block is still reading
    R* rslots = red + (((k + 1) & 1) ? RS_ES : RS_PQ) * a.red_stride;
    // ---- U: owner update of every node
    tr.mark(TR_CG_U0);
    const Sums2<R> us = cg_update<R>(g, t, c, alpha, beta, k, vg.bid * blockDim.x + threadIdx.x,
                                     vg.nblk * blockDim.x);
    tr.mark(TR_CG_U1);
    const R vgam = us.a, vrr = us.b;
    {
      R v[2] = {vgam, vrr};
      block_reduce_store<2>(v, rslots + a.red_stride, a.red_stride, vg);
    }
    if (!grid_sync(a.bar, vg)) return -1;
    tr.mark(TR_CG_UPDATE);
    // ---- A: partials of w = A u, block sums of <w, u>
    R vd = R(0);
    for (int tile = vg.bid; tile < ntiles; tile += vg.nblk) vd += apply_z(tile);
    tr.mark(TR_CG_APPLY);
    {
      R v[1] = {vd};
      block_reduce_store<1>(v, rslots, a.red_stride, vg);
    }
    R tot[3];  // <w,u>, <r,u>, <r,r>
    if (!grid_sync_total<3>(a.bar, vg, rslots, a.red_stride, tot)) return -1;
    tr.mark(TR_CG_PASS);
    tr.value(TR_RR, (double)tot[2]);
    if (k >= 0) {
      ++it;
      if (tot[2] <= thresh) {
        conv = true;
        break;
      }
    }
    if (threadIdx.x == 0) {
      const R gn = tot[1], dn = tot[0];
      R b = k < 0 ? R(0) : gn / gamma;
      R den = k < 0 ? dn : dn - b * gn / alpha;
      s_scal[0] = gn / den;
      s_scal[1] = b;
      s_scal[2] = (den > R(0) && gn > R(0)) ? R(1) : R(0);
    }
    __syncthreads();
    if (s_scal[2] == R(0)) {
      tr.value(TR_BREAK, (double)tot[0]);
      break;
    }
    gamma = tot[1];
    alpha = s_scal[0];
    beta = s_scal[1];
    __syncthreads();
  }
  *iters = it;
  return conv ? 1 : 0;
}

// ---------------------------------------------------------------------------
// CG with the tensor-product mass preconditioner (pcg3).  The operator is
// dominated by the mass part s_e M (alpha dt / h^2 ~ 1e-2 ... 1e-1), whose
// Jacobi-scaled form is close to the tensor product of the 1D matrices
// I + L/4 (L = sum of the two neighbours).  The preconditioner is
//     P^-1 = D^-1/2 (Q_x Q_y Q_z) D^-1/2,   Q_d = I - c L_d,  c = PC_C,
// a first-order Neumann approximation of that inverse (missing neighbours at
// the mesh ends are dropped, so every Q_d is symmetric and diagonally
// dominant and P^-1 is SPD on the free nodes; D^-1/2 is 0 on Dirichlet
// nodes).  c = 0.2 gave the fewest iterations on the assembled matrices of
// the 2 mm and 10 mm workloads (25 instead of 64 with Jacobi at 1e-12).
// The preconditioner runs in FP32 in both precisions (sq, v and the filter;
// u is stored in the solve's precision and <r,u> accumulated in it): it only
// has to be a fixed SPD approximation, and in an FP64 solve an FP64 filter
// was bound by the FP64 pipe.  Single-reduction recurrences as in pcg1 / pcg2
// with u = P^-1 r, in three phases per iteration, each ended by a grid
// barrier:
//   U  (owners, flat): w = own + neighbours' partials of A u; p = u + beta p;
//      s = w + beta s; x += alpha p; r -= alpha s; v = D^-1/2 r; sum <r,r>;
//   P  (flat): u = D^-1/2 Q v (27-point separable stencil); sum <r,u>;
//   A  (tiles): partials of w = A u; sum <w,u>.
// ---------------------------------------------------------------------------
constexpr double PC_C = 0.2;
// Preconditioner tiles: each thread owns two adjacent node columns of a tile
// row, so a tile is at most 64 columns wide (32 threads per row) and holds at
// most 2 NT columns; the host caps the tile height so that the stored window
// (halo one node, rows at an even pitch) has at most PC_WN_MAX entries, the
// window of a 64 x 5 tile.
constexpr int PC_CPT = 2;  // the pass reads and writes column pairs
constexpr int PC_WN_MAX = (64 + 2) * (NT / 32 + 2);
constexpr int PC_WM = (PC_WN_MAX + NT - 1) / NT;

template <typename R>
struct PCVecs {
  R* x;           // solution, updated in place
  R* r;           // residual
  R* p;           // search direction
  R* s;           // s = A p, kept by recurrence
  R* u;           // u = P^-1 r, the apply's input
  R* q;           // own partial of w = A u
  R* X;           // NXB exchange planes of w's partials
  const R* dinv;  // Jacobi inverse diagonal, 0 on Dirichlet nodes
  float* sq;      // sqrt(dinv), filled by the first update phase
  float* v;       // v = sqrt(dinv) r, the preconditioner's input
};

// Update phase of pcg3 (flat like cg_update, but two nodes per lane and step
// in both precisions: with four FP32 nodes the eleven arrays' values exceed
// the register budget and spill, measured 3.5 % slower on the 20 mm patch).
// k < 0: sq = sqrt(dinv), v = sq r.  Returns the thread's <r,r>.
template <typename R>
static __device__ __noinline__ R pc_update(const Grid3 g, const Tiling t, const PCVecs<R> c, R alpha, R beta, int k,
                                           int gtid, int gstride) {
  constexpr int VEC = 2;
  using V = typename Vec2<R>::T;
  const int nn = g.nnx * g.nny * g.nnz;
  const size_t xs = xplane(nn);
  const unsigned long long mx = div_magic(g.nnx), my = div_magic(g.nny), mz = div_magic(t.ez);
  const bool init = k < 0, first = k == 0;
  const int ngroups = (nn + VEC - 1) / VEC;
  R vrr = R(0);
  auto load = [&](const R* a, int n0, int cnt, R (&o)[VEC]) {
    if (cnt == VEC) {
      const V v = __ldcg(reinterpret_cast<const V*>(a + n0));
      const R* e = reinterpret_cast<const R*>(&v);
#pragma unroll
      for (int m = 0; m < VEC; ++m) o[m] = e[m];
    } else {
#pragma unroll
      for (int m = 0; m < VEC; ++m) o[m] = m < cnt ? __ldcg(a + n0 + m) : R(0);
    }
  };
  // the preconditioner's FP32 arrays, VEC values at a time (4 B x VEC)
  using VP = typename VecP<VEC>::T;
  auto loadp = [&](const float* a, int n0, int cnt, float (&o)[VEC]) {
    if (cnt == VEC) {
      const VP v = __ldcg(reinterpret_cast<const VP*>(a + n0));
      const float* e = reinterpret_cast<const float*>(&v);
#pragma unroll
      for (int m = 0; m < VEC; ++m) o[m] = e[m];
    } else {
#pragma unroll
      for (int m = 0; m < VEC; ++m) o[m] = m < cnt ? __ldcg(a + n0 + m) : 0.0f;
    }
  };
  auto storep = [&](float* a, int n0, int cnt, const float (&o)[VEC]) {
    if (cnt == VEC) {
      VP v;
      float* e = reinterpret_cast<float*>(&v);
#pragma unroll
      for (int m = 0; m < VEC; ++m) e[m] = o[m];
      *reinterpret_cast<VP*>(a + n0) = v;
    } else {
#pragma unroll
      for (int m = 0; m < VEC; ++m)
        if (m < cnt) a[n0 + m] = o[m];
    }
  };
  auto store = [&](R* a, int n0, int cnt, const R (&o)[VEC]) {
    if (cnt == VEC) {
      V v;
      R* e = reinterpret_cast<R*>(&v);
#pragma unroll
      for (int m = 0; m < VEC; ++m) e[m] = o[m];
      *reinterpret_cast<V*>(a + n0) = v;
    } else {
#pragma unroll
      for (int m = 0; m < VEC; ++m)
        if (m < cnt) a[n0 + m] = o[m];
    }
  };
  for (int q = gtid; q < ngroups; q += gstride) {
    const int n0 = q * VEC;
    const int cnt = min(VEC, nn - n0);
    R rk[VEC];
    float sqv[VEC], vn[VEC];
    load(c.r, n0, cnt, rk);
    if (init) {
      R dv[VEC];
      load(c.dinv, n0, cnt, dv);
#pragma unroll
      for (int m = 0; m < VEC; ++m) {
        sqv[m] = (float)sqrt(dv[m]);
        vn[m] = sqv[m] * (float)rk[m];
        if (sqv[m] != 0.0f) vrr = fma(rk[m], rk[m], vrr);
      }
      storep(c.sq, n0, cnt, sqv);
      storep(c.v, n0, cnt, vn);
      continue;
    }
    loadp(c.sq, n0, cnt, sqv);
    int lf[VEC];
    int rowf = -1;
    {
      const int row = div_by(n0, g.nnx, mx);
      int i = n0 - row * g.nnx;
      int kz = div_by(row, g.nny, my);
      int j = row - kz * g.nny;
      auto row_faces = [&](int jj, int kk) {
        const bool ly = t.nty > 1 && jj > 0 && jj < g.ny && (jj & (t.ey - 1)) == 0;
        const bool lz = kk > 0 && kk < g.nz && kk - div_by(kk, t.ez, mz) * t.ez == 0;
        return (ly ? 2 : 0) | (lz ? 4 : 0);
      };
      if (cnt == VEC && i + VEC <= g.nnx) {
        rowf = row_faces(j, kz);
#pragma unroll
        for (int m = 0; m < VEC; ++m) lf[m] = rowf | low_faces(g, t, i + m, false, false);
      } else {
#pragma unroll
        for (int m = 0; m < VEC; ++m) {
          lf[m] = m < cnt ? (row_faces(j, kz) | low_faces(g, t, i, false, false)) : 0;
          if (++i == g.nnx) {
            i = 0;
            if (++j == g.nny) {
              j = 0;
              ++kz;
            }
          }
        }
      }
    }
    R w[VEC], xk[VEC], pk[VEC], sk[VEC], uk[VEC], wx[VEC], wy[VEC], wz[VEC];
    load(c.q, n0, cnt, w);
    load(c.x, n0, cnt, xk);
    load(c.u, n0, cnt, uk);
    if (!first) {
      load(c.p, n0, cnt, pk);
      load(c.s, n0, cnt, sk);
    } else {
#pragma unroll
      for (int m = 0; m < VEC; ++m) pk[m] = sk[m] = R(0);
    }
    if (rowf >= 0) {
#pragma unroll
      for (int m = 0; m < VEC; ++m) wy[m] = wz[m] = R(0);
      if (rowf & 2) load(c.X + 1 * xs, n0, VEC, wy);
      if (rowf & 4) load(c.X + 3 * xs, n0, VEC, wz);
#pragma unroll
      for (int m = 0; m < VEC; ++m) wx[m] = (lf[m] & 1) ? __ldcg(c.X + 0 * xs + n0 + m) : R(0);
    } else {
#pragma unroll
      for (int m = 0; m < VEC; ++m) {
        wx[m] = (lf[m] & 1) ? __ldcg(c.X + 0 * xs + n0 + m) : R(0);
        wy[m] = (lf[m] & 2) ? __ldcg(c.X + 1 * xs + n0 + m) : R(0);
        wz[m] = (lf[m] & 4) ? __ldcg(c.X + 3 * xs + n0 + m) : R(0);
      }
    }
    R pn[VEC], sn[VEC], rn[VEC], xn[VEC];
#pragma unroll
    for (int m = 0; m < VEC; ++m) {
      pn[m] = pk[m];
      sn[m] = sk[m];
      rn[m] = rk[m];
      xn[m] = xk[m];
      vn[m] = 0.0f;
      if (m >= cnt || sqv[m] == 0.0f) continue;
      const int n = n0 + m;
      const int f = lf[m];
      R wv = w[m];
      if (f) {  // neighbours' partials, in the order gather_partials uses
        if (f & 1) wv += wx[m];
        if (f & 2) wv += wy[m];
        if ((f & 3) == 3) wv += __ldcg(c.X + 2 * xs + n);
        if (f & 4) wv += wz[m];
        if ((f & 5) == 5) wv += __ldcg(c.X + 4 * xs + n);
        if ((f & 6) == 6) wv += __ldcg(c.X + 5 * xs + n);
        if (f == 7) wv += __ldcg(c.X + 6 * xs + n);
      }
      pn[m] = first ? uk[m] : fma(beta, pk[m], uk[m]);
      sn[m] = first ? wv : fma(beta, sk[m], wv);
      rn[m] = fma(-alpha, sn[m], rk[m]);
      xn[m] = fma(alpha, pn[m], xk[m]);
      vn[m] = sqv[m] * (float)rn[m];
      vrr = fma(rn[m], rn[m], vrr);
    }
    store(c.p, n0, cnt, pn);
    store(c.s, n0, cnt, sn);
    store(c.r, n0, cnt, rn);
    store(c.x, n0, cnt, xn);
    storep(c.v, n0, cnt, vn);
  }
  return vrr;
}

// FP32 update phase of pcg3 (k >= 0) with its inputs staged in shared
// memory.  The same arithmetic on the same node pairs as pc_update<float>
// (thread gtid takes pairs gtid, gtid + gstride, ...; bitwise equal results),
// but a thread's inputs arrive by asynchronous copies two pairs ahead, so its
// L2 round trips overlap instead of following one another: the register
// version waits one round trip per pair, and keeping more pairs in flight in
// registers spills.  Every thread copies into and reads only its own slots
// (no block barrier).  Per stage a thread holds 8 bytes of each of 13
// arrays: r, q, x, u, p, s, sq and the x-face partials in `ra`, the y-face,
// xy-edge, z-face, xz-edge and yz-edge partials in `rb`; a partial plane no
// node of the pair gathers is zero-filled without a read, and so are p and s
// in the first iteration (p = s = 0).  The rare corner partials (x, y and z
// faces at once) are loaded directly.  Returns the thread's <r,r>.
constexpr int UST = 3, UNA = 8, UNB = 5;  // stages; arrays in ra / rb per stage
template <int NA>
struct UStage {
  float2 a[NA][NT];
};
static_assert(UST * sizeof(UStage<UNA>) <= STAGE_BYTES, "staged update inputs fit the dynamic ring");
static_assert(UST * sizeof(UStage<UNB>) <= sizeof(ApplySmem<double>), "staged partials fit the apply's buffers");
static __device__ __noinline__ float pc_update_staged(const Grid3 g, const Tiling t, const PCVecs<float> c,
                                                      float alpha, float beta, bool first, int gtid, int gstride,
                                                      UStage<UNA>* ra, UStage<UNB>* rb) {
  const int nn = g.nnx * g.nny * g.nnz;
  const size_t xs = xplane(nn);
  const unsigned long long mx = div_magic(g.nnx), my = div_magic(g.nny), mz = div_magic(t.ez);
  const int ngroups = (nn + 1) / 2;
  const int tid = threadIdx.x;
  float vrr = 0.0f;
  // low tile faces of the pair's nodes, node 0 in bits 0-2, node 1 in bits 3-5
  auto faces = [&](int q) {
    const int n0 = 2 * q;
    const int row = div_by(n0, g.nnx, mx);
    int i = n0 - row * g.nnx;
    int kz = div_by(row, g.nny, my);
    int j = row - kz * g.nny;
    auto node = [&]() {
      const bool ly = t.nty > 1 && j > 0 && j < g.ny && (j & (t.ey - 1)) == 0;
      const bool lz = kz > 0 && kz < g.nz && kz - div_by(kz, t.ez, mz) * t.ez == 0;
      return low_faces(g, t, i, ly, lz);
    };
    const int f0 = node();
    if (n0 + 1 >= nn) return f0;
    if (++i == g.nnx) {
      i = 0;
      if (++j == g.nny) {
        j = 0;
        ++kz;
      }
    }
    return f0 | (node() << 3);
  };
  auto issue = [&](int q, int st, int lf) {
    if (q < ngroups) {
      const int n0 = 2 * q;
      const int sb = min(2, nn - n0) * 4;  // bytes that lie in the arrays
      float2* A = &ra[st].a[0][tid];
      float2* B = &rb[st].a[0][tid];
      const int f0 = lf & 7, f1 = lf >> 3;
      auto any = [&](int m) { return ((f0 & m) == m || (f1 & m) == m) ? sb : 0; };
      cp_async8_fill(A + 0 * NT, c.r + n0, sb);
      cp_async8_fill(A + 1 * NT, c.q + n0, sb);
      cp_async8_fill(A + 2 * NT, c.x + n0, sb);
      cp_async8_fill(A + 3 * NT, c.u + n0, sb);
      cp_async8_fill(A + 4 * NT, c.p + n0, first ? 0 : sb);
      cp_async8_fill(A + 5 * NT, c.s + n0, first ? 0 : sb);
      cp_async8_fill(A + 6 * NT, c.sq + n0, sb);
      cp_async8_fill(A + 7 * NT, c.X + 0 * xs + n0, any(1));
      cp_async8_fill(B + 0 * NT, c.X + 1 * xs + n0, any(2));
      cp_async8_fill(B + 1 * NT, c.X + 2 * xs + n0, any(3));
      cp_async8_fill(B + 2 * NT, c.X + 3 * xs + n0, any(4));
      cp_async8_fill(B + 3 * NT, c.X + 4 * xs + n0, any(5));
      cp_async8_fill(B + 4 * NT, c.X + 5 * xs + n0, any(6));
    }
    cp_async_commit();
  };
  int q = gtid;
  int lf0 = q < ngroups ? faces(q) : 0;
  int lf1 = q + gstride < ngroups ? faces(q + gstride) : 0;
  issue(q, 0, lf0);
  issue(q + gstride, 1, lf1);
  int st = 0, st2 = 2;
  for (; q < ngroups; q += gstride) {
    const int q2 = q + 2 * gstride;
    const int lf2 = q2 < ngroups ? faces(q2) : 0;
    issue(q2, st2, lf2);
    cp_async_wait<UST - 1>();  // the pair q has landed
    const float2* A = &ra[st].a[0][tid];
    const float2* B = &rb[st].a[0][tid];
    const int n0 = 2 * q;
    const int cnt = min(2, nn - n0);
    const float2 rk2 = A[0 * NT], w2 = A[1 * NT], xk2 = A[2 * NT], uk2 = A[3 * NT];
    const float2 pk2 = A[4 * NT], sk2 = A[5 * NT], sq2 = A[6 * NT];
    const float rk[2] = {rk2.x, rk2.y}, w[2] = {w2.x, w2.y}, xk[2] = {xk2.x, xk2.y}, uk[2] = {uk2.x, uk2.y};
    const float pk[2] = {pk2.x, pk2.y}, sk[2] = {sk2.x, sk2.y}, sqv[2] = {sq2.x, sq2.y};
    float pn[2], sn[2], rn[2], xn[2], vn[2];
#pragma unroll
    for (int m = 0; m < 2; ++m) {
      pn[m] = pk[m];
      sn[m] = sk[m];
      rn[m] = rk[m];
      xn[m] = xk[m];
      vn[m] = 0.0f;
      if (m >= cnt || sqv[m] == 0.0f) continue;
      const int f = m == 0 ? (lf0 & 7) : (lf0 >> 3);
      float wv = w[m];
      if (f) {  // neighbours' partials, in the order gather_partials uses
        auto part = [&](const float2* P) { return m == 0 ? P->x : P->y; };
        if (f & 1) wv += part(A + 7 * NT);
        if (f & 2) wv += part(B + 0 * NT);
        if ((f & 3) == 3) wv += part(B + 1 * NT);
        if (f & 4) wv += part(B + 2 * NT);
        if ((f & 5) == 5) wv += part(B + 3 * NT);
        if ((f & 6) == 6) wv += part(B + 4 * NT);
        if (f == 7) wv += __ldcg(c.X + 6 * xs + n0 + m);
      }
      pn[m] = first ? uk[m] : fmaf(beta, pk[m], uk[m]);
      sn[m] = first ? wv : fmaf(beta, sk[m], wv);
      rn[m] = fmaf(-alpha, sn[m], rk[m]);
      xn[m] = fmaf(alpha, pn[m], xk[m]);
      vn[m] = sqv[m] * rn[m];
      vrr = fmaf(rn[m], rn[m], vrr);
    }
    if (cnt == 2) {
      *reinterpret_cast<float2*>(c.p + n0) = make_float2(pn[0], pn[1]);
      *reinterpret_cast<float2*>(c.s + n0) = make_float2(sn[0], sn[1]);
      *reinterpret_cast<float2*>(c.r + n0) = make_float2(rn[0], rn[1]);
      *reinterpret_cast<float2*>(c.x + n0) = make_float2(xn[0], xn[1]);
      *reinterpret_cast<float2*>(c.v + n0) = make_float2(vn[0], vn[1]);
    } else {
      c.p[n0] = pn[0];
      c.s[n0] = sn[0];
      c.r[n0] = rn[0];
      c.x[n0] = xn[0];
      c.v[n0] = vn[0];
    }
    lf0 = lf1;
    lf1 = lf2;
    st = st == UST - 1 ? 0 : st + 1;
    st2 = st2 == UST - 1 ? 0 : st2 + 1;
  }
  cp_async_wait<0>();  // no copy into the slots outlives the phase
  return vrr;
}

// Preconditioner phase of pcg3: u = sq (Q_z Q_y Q_x v) and the block's sum of
// <r,u>.  Node-owned tiles of tp.ex x tp.ey columns and tp.ez node layers;
// each thread owns two adjacent columns of a tile row (a tile step covers up
// to 2 NT nodes); a tile marches up from one layer below its range to one
// above, loads the (ex+2) x (ey+2) window of v of each layer into shared
// memory (zeros outside the mesh, which drops the missing neighbours),
// applies Q_x Q_y there, and keeps three consecutive layers of the result per
// column in registers for Q_z.  The windows (with sq and r of the owned
// nodes) arrive by cp.async several layers ahead in a ring of slots; one
// block barrier per layer.
template <typename R>
static __device__ __noinline__ R pc_apply(const Grid3 g, const Tiling tp, const PCVecs<R> c, R* win_raw,
                                          const VGrid vg) {
  const int S = g.nnx * g.nny;
  // NS ring slots, D = NS - 1 layers in flight: a tile column is narrow, so
  // several layers must be in flight to cover the memory latency.  A slot
  // holds the layer's window of v and sq of the owned columns (FP32), then r
  // of the owned columns (R).
  constexpr int NS = sizeof(R) == 4 ? 7 : 5, D = NS - 1;
  constexpr int SLOT_MAX = ((PC_WN_MAX + PC_CPT * NT) * 4 + PC_CPT * NT * (int)sizeof(R) + 15) / 16 * 16;
  static_assert(NS * SLOT_MAX <= STAGE_BYTES, "ring of the widest window fits the dynamic shared memory");
  // window rows of WXP nodes, stored with an even pitch WXPP so that a
  // thread's column pair starts on 8 bytes (the pad column is never used)
  const int TX = tp.ex, TY = tp.ey, WXP = TX + 2, WN = WXP * (TY + 2);
  const int WXPP = (WXP + 1) & ~1, WNP = WXPP * (TY + 2);
  const int TXT = (TX + PC_CPT - 1) / PC_CPT;                        // threads per tile row
  const int RB = ((WNP + PC_CPT * NT) * 4 + 15) / 16 * 16;            // byte offset of r in a slot
  const int SB = (RB + PC_CPT * NT * (int)sizeof(R) + 15) / 16 * 16;  // slot bytes
  unsigned char* ring = reinterpret_cast<unsigned char*>(win_raw);
  const int ntiles = tp.ntx * tp.nty * tp.ntz;
  const float cw = (float)PC_C;
  const int tid = threadIdx.x;
  const int ty = tid / TXT, tx0 = PC_CPT * (tid - ty * TXT);  // the thread's first column in the tile
  R gam = R(0);
  for (int tile = vg.bid; tile < ntiles; tile += vg.nblk) {
    const int txy = tp.ntx * tp.nty;
    const int tiz = tile / txy, trem = tile - tiz * txy;
    const int tiy = trem / tp.ntx, tix = trem - tiy * tp.ntx;
    const int i0 = tix * TX, j0 = tiy * TY, k0 = tiz * tp.ez, k1 = min(k0 + tp.ez, g.nnz);
    const int j = j0 + ty;
    bool own[PC_CPT];
#pragma unroll
    for (int q = 0; q < PC_CPT; ++q) own[q] = ty < TY && tx0 + q < TX && i0 + tx0 + q < g.nnx && j < g.nny;
    float tm[PC_CPT], tc[PC_CPT];  // xy-filtered values of layers L - 2, L - 1
    float sq_c[PC_CPT];            // sq, r of the columns' nodes at layer L - 1
    R r_c[PC_CPT];
#pragma unroll
    for (int q = 0; q < PC_CPT; ++q) {
      tm[q] = tc[q] = sq_c[q] = 0.0f;
      r_c[q] = R(0);
    }
    // this thread's window entries (w = tid + m NT): their in-layer node
    // offsets (-1 outside the mesh) and places in the slot; fixed for the tile
    int woff[PC_WM], soff[PC_WM];
#pragma unroll
    for (int m = 0; m < PC_WM; ++m) {
      const int w = tid + m * NT;
      const int wy = w / WXP, wx = w - wy * WXP;
      const int gi = i0 - 1 + wx, gj = j0 - 1 + wy;
      woff[m] = (w < WN && gi >= 0 && gi < g.nnx && gj >= 0 && gj < g.nny) ? gi + g.nnx * gj : -1;
      soff[m] = wy * WXPP + wx;
    }
    const int own_off = i0 + tx0 + g.nnx * j;
    // slot of layer L: async copies, zeros outside the mesh, one group per layer
    auto load_layer = [&](int L, int slot) {
      if (L >= 0 && L < g.nnz && L <= k1) {
        float* buf = reinterpret_cast<float*>(ring + slot * SB);
        const float* vL = c.v + (size_t)S * L;
#pragma unroll
        for (int m = 0; m < PC_WM; ++m) {
          const int w = tid + m * NT;
          if (woff[m] >= 0)
            cp_async<4>(buf + soff[m], vL + woff[m]);
          else if (w < WN)
            buf[soff[m]] = 0.0f;
        }
        if (L >= k0 && L < k1) {
          const size_t n = (size_t)S * L + own_off;
#pragma unroll
          for (int q = 0; q < PC_CPT; ++q)
            if (own[q]) {
              cp_async<4>(buf + WNP + PC_CPT * tid + q, c.sq + n + q);
              cp_async<sizeof(R)>(reinterpret_cast<R*>(ring + slot * SB + RB) + PC_CPT * tid + q, c.r + n + q);
            }
        }
      }
      cp_async_commit();
    };
    for (int d = 0; d < D; ++d) load_layer(k0 - 1 + d, d);
    int sl = 0;
    for (int L = k0 - 1; L <= k1; ++L) {
      cp_async_wait<D - 1>();  // layer L has landed (L + 1 .. L + D - 1 may be in flight)
      __syncthreads();         // ... for every thread; the slot of layer L - 1 is free again
      load_layer(L + D, sl == 0 ? NS - 1 : sl - 1);
      const float* buf = reinterpret_cast<const float*>(ring + sl * SB);
      float tl[PC_CPT];
#pragma unroll
      for (int q = 0; q < PC_CPT; ++q) tl[q] = 0.0f;
      if (ty < TY && L >= 0 && L < g.nnz) {
        float acc[PC_CPT];
#pragma unroll
        for (int q = 0; q < PC_CPT; ++q) acc[q] = 0.0f;
#pragma unroll
        for (int dy = 0; dy < 3; ++dy) {
          // window columns tx0 .. tx0 + 3 in two 8-byte loads (column tx0 + 3
          // may be the pad, which only the unowned column tx0 + 1 = TX uses)
          const float* row = buf + (ty + dy) * WXPP + tx0;
          const float2 ra = *reinterpret_cast<const float2*>(row);
          const float2 rb = *reinterpret_cast<const float2*>(row + 2);
          const float rv[PC_CPT + 2] = {ra.x, ra.y, rb.x, rb.y};
#pragma unroll
          for (int q = 0; q < PC_CPT; ++q) {
            const float t = fmaf(-cw, rv[q] + rv[q + 2], rv[q + 1]);
            acc[q] = dy == 1 ? acc[q] + t : fmaf(-cw, t, acc[q]);
          }
        }
#pragma unroll
        for (int q = 0; q < PC_CPT; ++q) tl[q] = own[q] ? acc[q] : 0.0f;
      }
      if (L >= k0 + 1) {  // layer L - 1 is complete
#pragma unroll
        for (int q = 0; q < PC_CPT; ++q)
          if (own[q]) {
            const int n = own_off + q + S * (L - 1);
            const R un = (R)(sq_c[q] * fmaf(-cw, tm[q] + tl[q], tc[q]));
            c.u[n] = un;
            if (sq_c[q] != 0.0f) gam = fma(r_c[q], un, gam);
          }
      }
      if (L >= k0 && L < k1) {
        using V2 = typename Vec2<R>::T;  // the thread's pair of sq and of r
        const float2 sqp = *reinterpret_cast<const float2*>(buf + WNP + PC_CPT * tid);
        const V2 rp = *reinterpret_cast<const V2*>(reinterpret_cast<const R*>(ring + sl * SB + RB) + PC_CPT * tid);
        if (own[0]) {
          sq_c[0] = sqp.x;
          r_c[0] = rp.x;
        }
        if (own[1]) {
          sq_c[1] = sqp.y;
          r_c[1] = rp.y;
        }
      }
#pragma unroll
      for (int q = 0; q < PC_CPT; ++q) {
        tm[q] = tc[q];
        tc[q] = tl[q];
      }
      sl = sl == NS - 1 ? 0 : sl + 1;
    }
    cp_async_wait<0>();
    __syncthreads();  // the window is free for the next tile
  }
  return gam;
}

// apply_z(tile) applies the operator to c.u on one tile of the tiling t, stores
// the partials in c.q / c.X and returns the tile's share of <w, u>.  Uses
// reduction rows RS_PQ..RS_RR and RS_ES..RS_EF.
template <typename R, class ApplyZ>
__device__ int pcg3(const SolveArgs& a, const VGrid& vg, const Tiling& t, const PCVecs<R>& c, ApplyZ apply_z,
                    R* win, unsigned char* aux, R thresh, int max_iter, R* red, int* iters, Tracer& tr) {
  R* s_scal = red_scalars<R>();
  const int ntiles = t.ntx * t.nty * t.ntz;
  const int gtid = vg.bid * blockDim.x + threadIdx.x, gstride = vg.nblk * blockDim.x;
  R alpha = R(0), beta = R(0), gamma = R(0);
  int it = 0;
  bool conv = false;
  for (int k = -1; k < max_iter; ++k) {
    // rows: <w,u>, <r,u>, <r,r>, alternating by iteration
    R* rslots = red + (((k + 1) & 1) ? RS_ES : RS_PQ) * a.red_stride;
    tr.mark(TR_CG_U0);
    {
      R v[1];
      if constexpr (sizeof(R) == 4) {  // FP32: staged update after the first pass
        v[0] = k < 0 ? pc_update<R>(a.g, t, c, alpha, beta, k, gtid, gstride)
                     : pc_update_staged(a.g, t, c, alpha, beta, k == 0, gtid, gstride,
                                        reinterpret_cast<UStage<UNA>*>(win), reinterpret_cast<UStage<UNB>*>(aux));
      } else {
        v[0] = pc_update<R>(a.g, t, c, alpha, beta, k, gtid, gstride);
      }
      tr.mark(TR_CG_U1);
      block_reduce_store<1>(v, rslots + 2 * a.red_stride, a.red_stride, vg);
    }
    if (!grid_sync(a.bar, vg)) return -1;
    tr.mark(TR_CG_UPDATE);
    {
      R v[1] = {pc_apply<R>(a.g, a.tp, c, win, vg)};
      block_reduce_store<1>(v, rslots + a.red_stride, a.red_stride, vg);
    }
    if (!grid_sync(a.bar, vg)) return -1;
    tr.mark(TR_CG_PRECOND);
    R vd = R(0);
    for (int tile = vg.bid; tile < ntiles; tile += vg.nblk) vd += apply_z(tile);
    tr.mark(TR_CG_APPLY);
    {
      R v[1] = {vd};
      block_reduce_store<1>(v, rslots, a.red_stride, vg);
    }
    R tot[3];  // <w,u>, <r,u>, <r,r>
    if (!grid_sync_total<3>(a.bar, vg, rslots, a.red_stride, tot)) return -1;
    tr.mark(TR_CG_PASS);
    tr.value(TR_RR, (double)tot[2]);
    if (k >= 0) {
      ++it;
      if (tot[2] <= thresh) {
        conv = true;
        break;
      }
    }
    if (threadIdx.x == 0) {
      const R gn = tot[1], dn = tot[0];
      R b = k < 0 ? R(0) : gn / gamma;
      R den = k < 0 ? dn : dn - b * gn / alpha;
      s_scal[0] = gn / den;
      s_scal[1] = b;
      s_scal[2] = (den > R(0) && gn > R(0)) ? R(1) : R(0);
    }
    __syncthreads();
    if (s_scal[2] == R(0)) {
      tr.value(TR_BREAK, (double)tot[0]);
      break;
    }
    gamma = tot[1];
    alpha = s_scal[0];
    beta = s_scal[1];
    __syncthreads();
  }
  *iters = it;
  return conv ? 1 : 0;
}

__device__ inline double elem_mean(const double* T, const Grid3& g, int ie, int je, int ke) {
  const int S = g.nnx * g.nny;
  const int n0 = ie + g.nnx * je + S * ke;
  double s = __ldcg(T + n0);
  s += __ldcg(T + n0 + 1);
  s += __ldcg(T + n0 + g.nnx);
  s += __ldcg(T + n0 + g.nnx + 1);
  s += __ldcg(T + n0 + S);
  s += __ldcg(T + n0 + S + 1);
  s += __ldcg(T + n0 + S + g.nnx);
  s += __ldcg(T + n0 + S + g.nnx + 1);
  return s * 0.125;
}

// The same mean of T + u (node by node, the values T + u rounds to), in the
// same order: equal to elem_mean of the stored sum.
__device__ inline double elem_mean_sum(const double* T, const double* u, const Grid3& g, int ie, int je, int ke) {
  const int S = g.nnx * g.nny;
  const int n0 = ie + g.nnx * je + S * ke;
  const int off[8] = {0, 1, g.nnx, g.nnx + 1, S, S + 1, S + g.nnx, S + g.nnx + 1};
  double s = __ldcg(T + n0) + __ldcg(u + n0);
#pragma unroll
  for (int c = 1; c < 8; ++c) s += __ldcg(T + n0 + off[c]) + __ldcg(u + n0 + off[c]);
  return s * 0.125;
}

// One backward-Euler solve on the block range vg (all of it or one job's slice).
// PMODE: 0 plain FP64 solves only, 1 refined solves only, 2 either (chosen by
// a.precision at run time).  Each kernel instantiates only the paths it runs,
// so the FP64 and FP32 loops do not share one register budget.
template <int PMODE, int NB = NODE_BATCH>
__device__ __forceinline__ void solve_body(const SolveArgs& a, const VGrid vg, bool first_of_launch) {
  __shared__ __align__(16) unsigned char smem_raw[sizeof(ApplySmem<double>)];
  static_assert(sizeof(WideSmem) <= sizeof(ApplySmem<double>), "wide-tile buffers share the apply's shared memory");
  extern __shared__ __align__(16) unsigned char stage_raw[];  // STAGE_BYTES of staged inputs
  ApplySmem<double>& sm64 = *reinterpret_cast<ApplySmem<double>*>(smem_raw);
  ApplySmem<float>& sm32 = *reinterpret_cast<ApplySmem<float>*>(smem_raw);
  double* stage64 = reinterpret_cast<double*>(stage_raw);
  float* stage32 = reinterpret_cast<float*>(stage_raw);
  if (first_of_launch) bar_begin(a.bar);  // later solves of a batch launch keep the block's copy
  if (ld_volatile_i32(a.bar.status) != 0) return;  // an earlier solve failed: leave state untouched
  Tracer tr{a.trace, vg.bid};
  tr.mark(TR_START);
  const Grid3 g = a.g;
  const Tiling t = a.t;
  const int nn = g.nnx * g.nny * g.nnz;
  const int ne = g.nx * g.ny * g.nz;
  const int S = g.nnx * g.nny;
  const int ntiles = t.ntx * t.nty * t.ntz;
  const bool refined = PMODE == 2 ? a.precision == PREC_FP32_REFINED : PMODE == 1;
  const int gtid = vg.bid * blockDim.x + threadIdx.x;
  const int gstride = vg.nblk * blockDim.x;

  // ---- phase 0: coefficients and eigenvalues, Dirichlet increments, load ---
  if (a.mv.active) {  // fused patch motion; independent of this (coarse) solve's data
    const MoveSpec& mv = a.mv;
    const int fnn = mv.fg.nnx * mv.fg.nny * mv.fg.nnz;
    for (int n = gtid; n < fnn; n += gstride) {
      const int i = n % mv.fg.nnx, j = (n / mv.fg.nnx) % mv.fg.nny, k = n / (mv.fg.nnx * mv.fg.nny);
      const int oi = i + (mv.noi - mv.ooi) * mv.r, oj = j + (mv.noj - mv.ooj) * mv.r;
      double v;
      if (oi >= 0 && oi <= mv.fg.nx && oj >= 0 && oj <= mv.fg.ny)
        v = __ldcg(mv.src + node_id(mv.fg, oi, oj, k));
      else
        v = trilinear_at(mv.Tc, mv.cg, i + mv.noi * mv.r, j + mv.noj * mv.r, k + mv.ok * mv.r, mv.r);
      mv.dst[n] = v;
    }
  }
  const double inv_dt = 1.0 / a.dt;  // once per thread: an FP64 division is costly here
  const double* Tcoef = a.T_coef ? a.T_coef : a.T_in;
  for_elems(g, vg, [&](int e, int ie, int je, int ke) {
    const double Tb = elem_mean(Tcoef, g, ie, je, ke);
    const uint8_t st = a.state[(ke * a.st_sy + je + a.st_oy) * a.st_sx + ie + a.st_ox];
    double rc;
    if (a.mat.chi != 0.0) {
      const double Tb0 = a.T_coef ? elem_mean(a.T_in, g, ie, je, ke) : Tb;
      rc = a.mat.rho * (a.mat.c0 + a.mat.c1 * (Tb - a.mat.Tref) + a.mat.chi * fpc_secant(a.mat, Tb, Tb0));
    } else {
      rc = a.mat.rho * (a.mat.c0 + a.mat.c1 * (Tb - a.mat.Tref));
    }
    double k = a.mat.k0 + a.mat.k1 * (Tb - a.mat.Tref);
    if (st == POWDER) k = a.mat.powder_factor * k;
    const double se = rc * inv_dt;
    a.s_e[e] = se;
    a.k_e[e] = k;
    // the element's share of the Jacobi diagonal, parked in r (unused until
    // the residual phase, which comes after the next grid barrier)
    a.r[e] = fma(se, a.Md, k * a.Kd);
#pragma unroll
    for (int m = 0; m < 8; ++m) a.lam[m * ne + e] = se * a.Mc[m] + k * a.Kc[m];
    if (refined) {
      a.sk32[e] = (float)se;
      a.sk32[ne + e] = (float)k;
    }
  });
  if (a.surf) {  // transfer coefficient per top face at the face mean of the coefficient temperature
    const int top = S * g.nz;
    for (int f = gtid; f < g.nx * g.ny; f += gstride) {
      const int je = f / g.nx, ie = f - je * g.nx;
      const int n0 = top + ie + g.nnx * je;
      double tf = __ldcg(Tcoef + n0);
      tf += __ldcg(Tcoef + n0 + 1);
      tf += __ldcg(Tcoef + n0 + g.nnx);
      tf += __ldcg(Tcoef + n0 + g.nnx + 1);
      tf *= 0.25;
      const double ta = a.T_amb;
      const double h = a.h_conv + a.rad * (tf * tf + ta * ta) * (tf + ta);
      a.hf[f] = h;
      if (refined) a.hf32[f] = (float)h;
    }
  }
  tr.mark(TR_P0_ELEMS);
  // increments: 0 on free nodes, g - T^k on Dirichlet nodes (disjoint writes)
  for_nodes(g, t, vg, [&](int n, int i, int j, int k, bool, bool) {
    if (!is_dir(g, a.dir, i, j, k)) a.u[n] = 0.0;
  });
  for_dirichlet(g, a.dir, vg, [&](int n, int i, int j, int k) {
    a.u[n] = dir_value(a.dv, i, j, k, n) - __ldcg(a.T_in + n);
  });
  tr.mark(TR_P0_DIR);
  {
    // the load tables (see load_table_entry), in chunks of 32 entries, one
    // warp per chunk, dealt round-robin over the blocks
    const int ne_tab = load_table_size(a.ld, g);
    const int lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
    for (int c = (threadIdx.x >> 5) * vg.nblk + vg.bid; c * 32 < ne_tab; c += nwarps * vg.nblk) {
      const int m = c * 32 + lane;
      if (m < ne_tab) a.G[m] = load_table_entry(a.ld, g, m);
    }
  }
  tr.mark(TR_P0_LOAD);
  if (!grid_sync(a.bar, vg)) return;
  tr.mark(TR_PHASE0);

  // ---- phase 1: Jacobi diagonal and right-hand side partials --------------
  if (a.ld.kind == 1) {  // the Gaussian's 1D hat integrals (chunks of 32, round-robin)
    const int w = g.nnx + g.nny;
    const int lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
    for (int c = (threadIdx.x >> 5) * vg.nblk + vg.bid; c * 32 < w; c += nwarps * vg.nblk) {
      const int p = c * 32 + lane;
      if (p < w) a.G[2 * w + p] = gauss_hat_entry(a.ld, g, a.G, p);
    }
  }
  // the precision form needs only the FP32 diagonal (its FP64 solves are
  // applies and residual updates, and the FP64 residual norm is <r,r>)
  for_nodes(g, t, vg, [&](int n, int i, int j, int k, bool, bool) {
    double d = 0.0;
    if (!is_dir(g, a.dir, i, j, k)) {
      for (int dz = -1; dz <= 0; ++dz)
        for (int dy = -1; dy <= 0; ++dy)
          for (int dx = -1; dx <= 0; ++dx) {
            int ie = i + dx, je = j + dy, ke = k + dz;
            if (ie < 0 || je < 0 || ke < 0 || ie >= g.nx || je >= g.ny || ke >= g.nz) continue;
            d += __ldcg(a.r + ie + g.nx * (je + g.ny * ke));
          }
      if (a.surf && k == g.nz)
        for (int je = max(j - 1, 0); je <= min(j, g.ny - 1); ++je)
          for (int ie = max(i - 1, 0); ie <= min(i, g.nx - 1); ++ie)
            d += __ldcg(a.hf + ie + g.nx * je) * a.Mfx[0] * a.Mfy[0];
    }
    if (refined)
      a.dinv32[n] = d > 0.0 ? 1.0f / (float)d : 0.0f;
    else
      a.dinv[n] = d > 0.0 ? 1.0 / d : 0.0;
  });
  {
    // partials of A u_D (u holds the Dirichlet increments, 0 elsewhere) + K T^k
    auto lam_full = [&](int e, const double*, double (&l8)[8]) {
#pragma unroll
      for (int m = 0; m < 8; ++m) l8[m] = __ldcg(a.lam + m * ne + e);
    };
    auto lam_k = [&](int e, const double*, double (&l8)[8]) {
      const double k = __ldcg(a.k_e + e);
#pragma unroll
      for (int m = 0; m < 8; ++m) l8[m] = k * a.Kc[m];
    };
    auto emit1 = [&](int n, int slot, double y, double) { store_partial(a.q, a.X, nn, n, slot, y, false); };
    auto emit2 = [&](int n, int slot, double y, double) { store_partial(a.q, a.X, nn, n, slot, y, true); };
    const FinishArray<double, double> fin;
    auto no_lam_fetch = [](int, double*) {};
    auto rhs_tile = [&](int tile) {
      const TileBox tb = tile_box(g, t, tile);
      apply_tile<double, false, NRAW>(g, t, tile, sm64, stage64, StageArray<double, double>{a.T_in}, fin,
                                      no_lam_fetch, lam_k, emit1);
      // the surface term of T^k too: its ambient part enters the load below
      if (a.surf && tb.top) surface_partials<double>(g, tb, a.T_in, a.hf, a.Mfx, a.Mfy, a.q, a.X);
      // u holds the Dirichlet increments and zeros: A u is zero on tiles whose
      // window holds no Dirichlet node
      if (tile_touches_dirichlet(g, t, tile, a.dir)) {
        apply_tile<double, false, NRAW>(g, t, tile, sm64, stage64, StageArray<double, double>{a.u}, fin,
                                        no_lam_fetch, lam_full, emit2);
        if (a.surf && tb.top) surface_partials<double>(g, tb, a.u, a.hf, a.Mfx, a.Mfy, a.q, a.X);
      }
    };
    if (ntiles <= RHS_ROUNDS * vg.nblk) {
      // a tile with Dirichlet nodes costs two applies: deal the tiles with
      // them first, then the others, in snake order over the blocks, so no
      // block gets two heavy tiles while another has fewer tiles
      int* items = rhs_items(g, t, a.dir, ntiles, vg);
      const int rounds = (ntiles + vg.nblk - 1) / vg.nblk;
      for (int m = 0; m < rounds; ++m)
        if (items[m] >= 0) rhs_tile(items[m]);
    } else {
      for (int tile = vg.bid; tile < ntiles; tile += vg.nblk) rhs_tile(tile);
    }
  }
  if (!grid_sync(a.bar, vg)) return;
  tr.mark(TR_RHS);
  {
    double v[2] = {0.0, 0.0};
    struct ResidV {
      double rr, Fn, dinv;
      bool top;
    };
    for_nodes_batched<NB>(
        g, t, vg,
        [&](int n, const NodeIx& x) {
          ResidV o{0.0, 0.0, 0.0, x.k == g.nz};
          double Fa = 0.0;  // ambient part of the surface term: T_amb sum_f h_f int_f phi_n dA
          if (o.top) {      // the top-face load, kept for the energy account
            o.Fn = top_load_tab(a.ld, g, a.G, x.i, x.j);
            if (a.surf) {
              double hs = 0.0;
              for (int je = max(x.j - 1, 0); je <= min(x.j, g.ny - 1); ++je)
                for (int ie = max(x.i - 1, 0); ie <= min(x.i, g.nx - 1); ++ie) hs += __ldcg(a.hf + ie + g.nx * je);
              Fa = a.T_amb * hs * (0.25 * g.hx * g.hy);
            }
          }
          const double Fxn = a.Fx ? __ldcg(a.Fx + n) : 0.0;
          if (!is_dir(g, a.dir, x.i, x.j, x.k))
            o.rr = ((o.Fn + Fa) + Fxn) - gather_partials((const double*)a.q, (const double*)a.X, nn, n,
                                                         low_faces(g, t, x.i, x.ly, x.lz));
          if (!refined) o.dinv = __ldcg(a.dinv + n);
          return o;
        },
        [&](int n, const ResidV& o) {
          if (o.top) a.F[n - S * g.nz] = o.Fn;
          a.r[n] = o.rr;
          if (!refined) v[0] += o.rr * o.rr * o.dinv;
          v[1] += o.rr * o.rr;
        });
    block_reduce_store<2>(v, a.red + RS_RZ0 * a.red_stride, a.red_stride, vg);
  }
  double tot0[2];
  if (!grid_sync_total<2>(a.bar, vg, a.red + RS_RZ0 * a.red_stride, a.red_stride, tot0)) return;
  tr.mark(TR_RESID);
  const double bb = tot0[1];
  const double thresh = a.tol * a.tol * bb;

  // ---- phase 2: solve ------------------------------------------------------
  int it = 0, outer = 0;
  bool conv = !(bb > 0.0) || (a.tol >= 1.0);
  if (!conv && !refined) {
    CGBufs<double> c{a.u, {a.r, a.r2}, {a.p0, a.p1}, {a.s0, a.s1}, {a.q, a.q2}, {a.X, a.X2}, a.dinv, a.lam};
    auto lam64 = [&](int e, const double*, double (&l8)[8]) {
#pragma unroll
      for (int m = 0; m < 8; ++m) l8[m] = __ldcg(a.lam + m * ne + e);
    };
    auto no_fetch64 = [](int, double*) {};
    int res;
    if (a.precond == 1) {
      // the FP32 preconditioner arrays live in the first halves of s1 and p1
      // (FP64 arrays of the node count, unused by this CG form)
      PCVecs<double> c3{a.u, a.r, a.p0, a.s0, a.r2, a.q, a.X, a.dinv, reinterpret_cast<float*>(a.s1),
                        reinterpret_cast<float*>(a.p1)};
      auto apply_z = [&](int tile) {
        double vd = 0.0;
        auto emit = [&](int n, int slot, double y, double xin) {
          store_partial(c3.q, c3.X, nn, n, slot, y, false);
          vd = fma(xin, y, vd);
        };
        apply_tile<double, false, 1, 1>(g, t, tile, sm64, stage64, StageArray<double, double>{c3.u},
                                        FinishArray<double, double>{}, no_fetch64, lam64, emit);
        if (a.surf) {
          const TileBox tb = tile_box(g, t, tile);
          if (tb.top) vd += surface_partials<double>(g, tb, c3.u, a.hf, a.Mfx, a.Mfy, c3.q, c3.X);
        }
        return vd;
      };
      res = pcg3<double>(a, vg, t, c3, apply_z, stage64, smem_raw, thresh, a.max_iter, a.red, &it, tr);
    } else {
      res = pcg1<double, false, NRAW>(a, vg, sm64, stage64, c, no_fetch64, lam64, thresh, a.max_iter, a.red, &it,
                                      tr);
    }
    if (res < 0) return;
    conv = res == 1;
  }
  // refined: FP32 CG for the correction d of the FP64 residual, FP64 update of
  // u and of the residual r -= A d, until ||r|| <= tol ||r_0||.  The inner
  // problem is scaled to unit residual norm (r / sigma with sigma = ||r||), so
  // FP32 neither underflows on nearly converged or barely loaded solves nor
  // overflows on hot ones; the correction is sigma d.
  double rr64 = bb;
  while (!conv && refined && outer < a.max_outer) {
    const double sigma = sqrt(rr64);
    const double isig = 1.0 / sigma;
    {
      float v[2] = {0.0f, 0.0f};
      for_nodes(g, t, vg, [&](int n, int, int, int, bool, bool) {
        float rf = (float)(__ldcg(a.r + n) * isig);
        a.r32[n] = rf;
        a.d32[n] = 0.0f;
        v[0] = fmaf(rf * rf, __ldcg(a.dinv32 + n), v[0]);
        v[1] = fmaf(rf, rf, v[1]);
      });
      block_reduce_store<2>(v, a.red32 + RS_RZ0 * a.red_stride, a.red_stride, vg);
    }
    float t32[2];
    if (!grid_sync_total<2>(a.bar, vg, a.red32 + RS_RZ0 * a.red_stride, a.red_stride, t32)) return;
    tr.mark(TR_OUTER_INIT);
    int inner = 0;
    CGBufs<float> c{a.d32, {a.r32, a.r32b}, {a.p0f, a.p1f}, {a.s0f, a.s1f}, {a.q32, a.q32b}, {a.X32, a.X32b},
                    a.dinv32, nullptr};
    float mcf[8], kcf[8];
#pragma unroll
    for (int m = 0; m < 8; ++m) {
      mcf[m] = (float)a.Mc[m];
      kcf[m] = (float)a.Kc[m];
    }
    // element data staged one layer ahead: two consecutive slots (s_e, k_e)
    auto fetch32 = [&](int e, float* slots) {
      cp_async<4>(slots, a.sk32 + e);
      cp_async<4>(slots + NT, a.sk32 + ne + e);
    };
    auto lam32 = [&](int e, const float* slots, float (&l8)[8]) {
      const float se = slots[0], ke = slots[NT];
#pragma unroll
      for (int m = 0; m < 8; ++m) l8[m] = fmaf(se, mcf[m], ke * kcf[m]);
    };
    const float ti = (float)a.tol_inner;
    int res;
    if (a.precond == 1) {
      PCVecs<float> c3{a.d32, a.r32, a.p0f, a.s0f, a.r32b, a.q32, a.X32, a.dinv32, a.s1f, a.p1f};
      if (a.wide) {
        WideSmem* smw = reinterpret_cast<WideSmem*>(smem_raw);
        WideCoef cf;
#pragma unroll
        for (int m = 0; m < 8; ++m) {
          cf.mp[m] = mcf[m];
          cf.kp[m] = kcf[m];
        }
        auto apply_z = [&](int tile) {
          float vd = apply_wide_partials(g, a.tw, tile, smw, stage32, c3.u, a.sk32, cf, c3.q, c3.X);
          if (a.surf) {
            const TileBox tb = tile_box(g, a.tw, tile);
            if (tb.top) vd += surface_partials<float>(g, tb, c3.u, a.hf32, a.Mfx, a.Mfy, c3.q, c3.X);
          }
          return vd;
        };
        res = pcg3<float>(a, vg, a.tw, c3, apply_z, stage32, smem_raw, ti * ti * t32[1], a.max_iter, a.red32,
                          &inner, tr);
      } else {
        auto apply_z = [&](int tile) {
          float vd = 0.0f;
          auto emit = [&](int n, int slot, float y, float xin) {
            store_partial(c3.q, c3.X, nn, n, slot, y, false);
            vd = fmaf(xin, y, vd);
          };
          // staging slots: 0 the window value, 1 and 2 the element data
          apply_tile<float, true, 3, 1>(g, t, tile, sm32, stage32, StageArray<float, float>{c3.u},
                                        FinishArray<float, float>{}, fetch32, lam32, emit);
          if (a.surf) {
            const TileBox tb = tile_box(g, t, tile);
            if (tb.top) vd += surface_partials<float>(g, tb, c3.u, a.hf32, a.Mfx, a.Mfy, c3.q, c3.X);
          }
          return vd;
        };
        res = pcg3<float>(a, vg, t, c3, apply_z, stage32, smem_raw, ti * ti * t32[1], a.max_iter, a.red32, &inner, tr);
      }
    } else if (a.wide) {
      CGVecs<float> c2{a.d32, a.r32, a.p0f, a.s0f, a.r32b, a.q32, a.X32, a.dinv32};
      WideSmem* smw = reinterpret_cast<WideSmem*>(smem_raw);
      WideCoef cf;
#pragma unroll
      for (int m = 0; m < 8; ++m) {
        cf.mp[m] = mcf[m];
        cf.kp[m] = kcf[m];
      }
      auto apply_z = [&](int tile) {
        return apply_wide_partials(g, a.tw, tile, smw, stage32, c2.z, a.sk32, cf, c2.q, c2.X);
      };
      res = pcg2<float>(a, vg, a.tw, c2, apply_z, ti * ti * t32[1], a.max_iter, a.red32, &inner, tr);
    } else {
      res = pcg1<float, true, NRAW + 2>(a, vg, sm32, stage32, c, fetch32, lam32, ti * ti * t32[1], a.max_iter,
                                        a.red32, &inner, tr);
    }
    if (res < 0) return;
    it += inner;
    ++outer;
    // FP64 apply of the correction (exact in FP64: d is an FP32 vector)
    auto lam_full = [&](int e, const double*, double (&l8)[8]) {
#pragma unroll
      for (int m = 0; m < 8; ++m) l8[m] = __ldcg(a.lam + m * ne + e);
    };
    auto no_lam_fetch = [](int, double*) {};
    auto emit = [&](int n, int slot, double y, double) { store_partial(a.q, a.X, nn, n, slot, y, false); };
    for (int tile = vg.bid; tile < ntiles; tile += vg.nblk) {
      apply_tile<double, false, NRAW>(g, t, tile, sm64, stage64, StageArray<double, float>{a.d32},
                                      FinishArray<double, float>{}, no_lam_fetch, lam_full, emit);
      if (a.surf) {
        const TileBox tb = tile_box(g, t, tile);
        if (tb.top) surface_partials<double>(g, tb, a.d32, a.hf, a.Mfx, a.Mfy, a.q, a.X);
      }
    }
    if (!grid_sync(a.bar, vg)) return;
    tr.mark(TR_OUTER_APPLY);
    double v[1] = {0.0};
    struct CorrV {
      double y, rk, uk;
      float dk;
      bool free;
    };
    for_nodes_batched<NB>(
        g, t, vg,
        [&](int n, const NodeIx& x) {
          CorrV o{0.0, 0.0, 0.0, 0.0f, !is_dir(g, a.dir, x.i, x.j, x.k)};
          if (o.free) {
            o.y = gather_partials((const double*)a.q, (const double*)a.X, nn, n, low_faces(g, t, x.i, x.ly, x.lz));
            o.rk = __ldcg(a.r + n);
            o.uk = __ldcg(a.u + n);
            o.dk = __ldcg(a.d32 + n);
          }
          return o;
        },
        [&](int n, const CorrV& o) {
          if (!o.free) return;
          const double rn = fma(-sigma, o.y, o.rk);  // partials are of A d; the correction is sigma d
          a.r[n] = rn;
          a.u[n] = fma(sigma, (double)o.dk, o.uk);
          v[0] += rn * rn;
        });
    block_reduce_store<1>(v, a.red + RS_RR * a.red_stride, a.red_stride, vg);
    double trr[1];
    if (!grid_sync_total<1>(a.bar, vg, a.red + RS_RR * a.red_stride, a.red_stride, trr)) return;
    tr.mark(TR_OUTER_END);
    rr64 = trr[0];
    conv = trr[0] <= thresh;
  }
  const int lvl = a.level;
  if (!conv) {
    if (vg.bid == 0 && threadIdx.x == 0 && !a.dry) {
      atomicCAS(a.bar.status, 0, (int)ST_NOCONV);
      a.stats->iters[lvl] += it;
      a.stats->outer[lvl] += outer;
      a.stats->last_iters[lvl] = it;
    }
    return;
  }

  // ---- phase 3: states and energy, then the commit ----------------------------
  // Everything that outlives the launch (T_out or T_relax, the element states,
  // the counters) is written after the solve's last grid barrier, which either
  // releases every block or none: a launch that fails at any barrier leaves
  // the problem's state as it was.  The new states and the energy terms are
  // formed from T^k + u, the same values T_out receives.
  tr.mark(TR_UPDATE);
  double te[3] = {0.0, 0.0, 0.0}, tloss[1] = {0.0};
  if (a.update_state || a.energy) {
    double v[3] = {0.0, 0.0, 0.0}, vl[1] = {0.0};
    for_elems(g, vg, [&](int e, int ie, int je, int ke) {
      if (a.update_state) {
        const double Tb = elem_mean_sum(a.T_in, a.u, g, ie, je, ke);
        const uint8_t st = a.state[(ke * a.st_sy + je + a.st_oy) * a.st_sx + ie + a.st_ox];
        uint8_t ns = (st == POWDER) ? POWDER : SOLID;
        if (Tb > a.mat.T_melt) ns = MELTED;
        a.st_new[e] = ns;
      }
      if (a.energy) {
        const int n0 = ie + g.nnx * je + S * ke;
        double us = __ldcg(a.u + n0);
        us += __ldcg(a.u + n0 + 1);
        us += __ldcg(a.u + n0 + g.nnx);
        us += __ldcg(a.u + n0 + g.nnx + 1);
        us += __ldcg(a.u + n0 + S);
        us += __ldcg(a.u + n0 + S + 1);
        us += __ldcg(a.u + n0 + S + g.nnx);
        us += __ldcg(a.u + n0 + S + g.nnx + 1);
        v[0] += __ldcg(a.s_e + e) * a.dt * a.vol8 * us;
      }
    });
    tr.mark(TR_END_ELEMS);
    if (a.energy) {
      for (int n = gtid; n < S; n += gstride) v[1] += a.dt * __ldcg(a.F + n);
      if (a.Fx)  // the interface load counts as heat through the boundary
        for (int n = gtid; n < nn; n += gstride) v[2] += a.dt * __ldcg(a.Fx + n);
      if (a.surf) {  // heat lost through the top: dt 1^T H (T^{k+1} - T_amb), face by face
        const int top = S * g.nz;
        for (int f = gtid; f < g.nx * g.ny; f += gstride) {
          const int je = f / g.nx, ie = f - je * g.nx;
          const int n0 = top + ie + g.nnx * je;
          const int off[4] = {0, 1, g.nnx, g.nnx + 1};
          double sv = 0.0;
#pragma unroll
          for (int c = 0; c < 4; ++c) sv += __ldcg(a.T_in + n0 + off[c]) + __ldcg(a.u + n0 + off[c]) - a.T_amb;
          vl[0] += a.dt * __ldcg(a.hf + f) * (0.25 * g.hx * g.hy) * sv;
        }
      }
      for_dirichlet(g, a.dir, vg, [&](int n, int i, int j, int k) {
        // reaction of a Dirichlet row: (S u + K T^{k+1})_n - F_n, T^{k+1} = T^k + u
        double R_n = 0.0;
        for (int dz = -1; dz <= 0; ++dz)
          for (int dy = -1; dy <= 0; ++dy)
            for (int dx = -1; dx <= 0; ++dx) {
              int ie = i + dx, je = j + dy, ke = k + dz;
              if (ie < 0 || je < 0 || ke < 0 || ie >= g.nx || je >= g.ny || ke >= g.nz) continue;
              int e = ie + g.nx * (je + g.ny * ke);
              double se = __ldcg(a.s_e + e), kk = __ldcg(a.k_e + e);
              int la = (i - ie) + 2 * (j - je) + 4 * (k - ke);
              double am = 0.0, ak = 0.0;  // row la of M^ u and of K^ T^{k+1}
#pragma unroll
              for (int b = 0; b < 8; ++b) {
                int nb = (ie + (b & 1)) + g.nnx * (je + ((b >> 1) & 1)) + S * (ke + (b >> 2));
                const double ub = __ldcg(a.u + nb);
                am = fma(a.Mhat[la * 8 + b], ub, am);
                ak = fma(a.Khat[la * 8 + b], __ldcg(a.T_in + nb) + ub, ak);
              }
              R_n += se * am + kk * ak;
            }
        if (k == g.nz) {
          R_n -= __ldcg(a.F + (n - S * g.nz));
          if (a.surf) R_n += surface_row(g, a.hf, a.Mfx, a.Mfy, i, j, a.T_in, a.u, a.T_amb);
        }
        v[2] += a.dt * R_n;
      });
    }
    tr.mark(TR_END_DIR);
    block_reduce_store<3>(v, a.red + RS_ES * a.red_stride, a.red_stride, vg);
    if (a.surf) block_reduce_store<1>(vl, a.red + RS_EX * a.red_stride, a.red_stride, vg);
    if (!grid_sync_total<3>(a.bar, vg, a.red + RS_ES * a.red_stride, a.red_stride, te)) return;
    if (a.surf) grid_total<1>(a.red + RS_EX * a.red_stride, a.red_stride, tloss, vg);
  }
  // the commit: no barrier follows
  if (a.T_relax) {  // an intermediate Picard solve: only the next coefficient temperature
    for (int n = gtid; n < nn; n += gstride) {
      const double ts = __ldcg(Tcoef + n);
      a.T_relax[n] = ts + 0.5 * (__ldcg(a.T_in + n) + __ldcg(a.u + n) - ts);
    }
  } else {  // four nodes per thread and step, loads first (element-wise, so T_out may be T_in)
    int n = gtid;
    for (; n + 3 * gstride < nn; n += 4 * gstride) {
      double v[4];
#pragma unroll
      for (int m = 0; m < 4; ++m) v[m] = __ldcg(a.T_in + n + m * gstride) + __ldcg(a.u + n + m * gstride);
#pragma unroll
      for (int m = 0; m < 4; ++m) a.T_out[n + m * gstride] = v[m];
    }
    for (; n < nn; n += gstride) a.T_out[n] = __ldcg(a.T_in + n) + __ldcg(a.u + n);
  }
  if (a.update_state)
    for_elems(g, vg, [&](int e, int ie, int je, int ke) {
      a.state[(ke * a.st_sy + je + a.st_oy) * a.st_sx + ie + a.st_ox] = __ldcg(a.st_new + e);
    });
  tr.mark(TR_END);
  if (vg.bid == 0 && threadIdx.x == 0 && !a.dry) {
    if (a.energy) {
      a.stats->e_stored[lvl] += te[0];
      a.stats->e_laser[lvl] += te[1];
      a.stats->e_flux[lvl] += te[2];
      a.stats->e_loss[lvl] += tloss[0];
      a.stats->e_last[lvl][0] = te[0];
      a.stats->e_last[lvl][1] = te[1];
      a.stats->e_last[lvl][2] = te[2];
      a.stats->e_last[lvl][3] = tloss[0];
    }
    a.stats->iters[lvl] += it;
    a.stats->outer[lvl] += outer;
    a.stats->solves[lvl] += 1;
    a.stats->last_iters[lvl] = it;
    if (it > a.stats->max_iters[lvl]) a.stats->max_iters[lvl] = it;
  }
}


// Internal linkage: every translation unit that launches the solve compiles its
// own copy (the two-level path and the allocation-free single step).
template <int PMODE>
static __global__ void __launch_bounds__(NT, MIN_BLOCKS) solve_kernel(const SolveArgs a) {
  solve_body<PMODE>(a, VGrid{(int)blockIdx.x, (int)gridDim.x}, true);
}

// A batch of independent jobs in one cooperative launch: job j runs on the
// blocks [first[j], first[j+1]) and performs its next nsolves[j] solves back
// to back (job-local grid barrier in between), each with its own barrier
// words, reduction slots and buffers, so jobs meet only at the launch's end.
// The arguments of job j's s-th solve are jobs[j * per_job + s]; each is
// copied to shared memory once per block.  At the end the job's first block
// writes the job's status word into st_out[j] (nonzero: a solve failed and
// the job's later solves were skipped).
constexpr int BATCH_MAX = 512;
struct BatchTable {
  int njobs, per_job;
  int first[BATCH_MAX + 1];
  int nsolves[BATCH_MAX];
};

template <int PMODE>
static __global__ void __launch_bounds__(NT, MIN_BLOCKS) solve_batch_kernel(const BatchTable* __restrict__ tab,
                                                                  const SolveArgs* __restrict__ jobs,
                                                                  int* __restrict__ st_out) {
  __shared__ SolveArgs s_args;
  __shared__ int s_job;
  if (threadIdx.x == 0) {
    int lo = 0, hi = tab->njobs - 1;
    while (lo < hi) {  // last job whose first block <= blockIdx.x
      const int mid = (lo + hi + 1) / 2;
      if (tab->first[mid] <= (int)blockIdx.x) lo = mid; else hi = mid - 1;
    }
    s_job = lo;
  }
  __syncthreads();
  const int j = s_job;
  if (tab->njobs <= 0 || (int)blockIdx.x >= tab->first[tab->njobs]) return;  // block not assigned
  const int b0 = tab->first[j], nb = tab->first[j + 1] - b0;
  if (nb <= 0) return;
  const VGrid vg{(int)blockIdx.x - b0, nb};
  const int ns = tab->nsolves[j];
  for (int sv = 0; sv < ns; ++sv) {
    const int* src = reinterpret_cast<const int*>(jobs + (size_t)j * tab->per_job + sv);
    int* dst = reinterpret_cast<int*>(&s_args);
    __syncthreads();  // the previous solve is done with s_args
    for (int w = threadIdx.x; w < (int)(sizeof(SolveArgs) / sizeof(int)); w += blockDim.x) dst[w] = src[w];
    __syncthreads();
    solve_body<PMODE, 1>(s_args, vg, sv == 0);
    if (sv + 1 < ns) {
      if (!grid_sync(s_args.bar, vg)) break;  // the next solve reads this one's results
      if (ld_volatile_i32(s_args.bar.status) != 0) break;
    }
  }
  if (vg.bid == 0 && threadIdx.x == 0) st_out[j] = ld_volatile_i32(s_args.bar.status);
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

// Flux-jump coupling (Section 3, Eqs. deltaDef and globalPbmAlternate): the
// interface load G_I = int_gamma (kappa_+ - kappa_-) dT-/dn phi_I dA of every
// coarse node of the patch's bounding box [oi, oi + pnx] x [oj, oj + pny] x
// [ok, nz] (zero elsewhere: the caller clears G).  gamma = the patch faces
// immersed in the plate (faces bit 0 x-, 1 x+, 2 y-, 3 y+, 4 bottom); n the
// local domain's outward normal; dT-/dn the normal derivative of the fine
// trilinear field (T- = Tf, at the end of the macro step) inside the fine
// element next to the face; kappa_- that element's conductivity (element mean
// of Tf, fine state after the step), kappa_+ the conductivity of the coarse
// element just outside the patch (element mean of the coarse field Tc at t_n,
// coarse state).  Each fine face's integrand is a product of two bilinear
// functions, integrated by 2 x 2 Gauss points; one thread per coarse node
// sums its faces in a fixed order.
struct IfaceSpec {
  Grid3 fg, cg;
  int oi, oj, ok, r, pnx, pny, pnz, faces;
  const double* Tf;
  const double* Tc;
  const uint8_t* st_f;  // plate-wide fine state map, (sx, sy) plane strides
  int st_sx, st_sy;
  const uint8_t* st_c;
  Material mat;
  double* G;
};

__device__ inline double iface_k(const Material& m, double Tb, uint8_t st) {
  double k = m.k0 + m.k1 * (Tb - m.Tref);
  return st == POWDER ? m.powder_factor * k : k;
}

__global__ void interface_load_kernel(IfaceSpec s) {
  const int bx = s.pnx + 1, by = s.pny + 1, bz = s.cg.nz - s.ok + 1;
  const long long nb = (long long)bx * by * bz;
  const double gq[2] = {0.21132486540518711775, 0.78867513459481288225};  // (1 -+ 1/sqrt 3) / 2
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < nb;
       q += (long long)gridDim.x * blockDim.x) {
    const int ci[3] = {s.oi + (int)(q % bx), s.oj + (int)((q / bx) % by), s.ok + (int)(q / ((long long)bx * by))};
    const int o[3] = {s.oi, s.oj, s.ok}, pn[3] = {s.pnx, s.pny, s.pnz};
    const int nf[3] = {s.fg.nx, s.fg.ny, s.fg.nz};
    const double hf[3] = {s.fg.hx, s.fg.hy, s.fg.hz};
    double Gsum = 0.0;
    for (int plane = 0; plane < 5; ++plane) {
      if (!((s.faces >> plane) & 1)) continue;
      const int d = plane / 2, side = plane & 1;  // plane 4: z, low side
      const int a1 = d == 0 ? 1 : 0, a2 = d == 2 ? 1 : 2;
      if (ci[d] != o[d] + (side ? pn[d] : 0)) continue;
      const int lo1 = o[a1], hi1 = o[a1] + pn[a1], lo2 = o[a2], hi2 = o[a2] + pn[a2];
      const double sign = side ? 1.0 : -1.0;
      const int ed = side ? nf[d] - 1 : 0;                // fine element layer next to the plane
      for (int c2 = max(ci[a2] - 1, lo2); c2 <= min(ci[a2], hi2 - 1); ++c2)
        for (int c1 = max(ci[a1] - 1, lo1); c1 <= min(ci[a1], hi1 - 1); ++c1) {
          // the coarse element outside the patch across this coarse face
          int ce[3];
          ce[d] = side ? o[d] + pn[d] : o[d] - 1;
          ce[a1] = c1;
          ce[a2] = c2;
          const double Tcb = elem_mean(s.Tc, s.cg, ce[0], ce[1], ce[2]);
          const double kp = iface_k(s.mat, Tcb, s.st_c[ce[0] + s.cg.nx * (ce[1] + s.cg.ny * ce[2])]);
          for (int f2 = 0; f2 < s.r; ++f2)
            for (int f1 = 0; f1 < s.r; ++f1) {
              int fe[3];
              fe[d] = ed;
              fe[a1] = (c1 - o[a1]) * s.r + f1;
              fe[a2] = (c2 - o[a2]) * s.r + f2;
              const double Tfb = elem_mean(s.Tf, s.fg, fe[0], fe[1], fe[2]);
              const uint8_t stf = s.st_f[(size_t)s.st_sx * s.st_sy * fe[2] + (size_t)s.st_sx * (fe[1] + o[1] * s.r) +
                                         fe[0] + o[0] * s.r];
              const double jump = kp - iface_k(s.mat, Tfb, stf);
              for (int g2 = 0; g2 < 2; ++g2)
                for (int g1 = 0; g1 < 2; ++g1) {
                  const double xi1 = gq[g1], xi2 = gq[g2];
                  double grad = 0.0;
                  for (int b2 = 0; b2 < 2; ++b2)
                    for (int b1 = 0; b1 < 2; ++b1) {
                      const double w = (b1 ? xi1 : 1.0 - xi1) * (b2 ? xi2 : 1.0 - xi2);
                      int lo[3], hi[3];
                      lo[d] = fe[d];
                      hi[d] = fe[d] + 1;
                      lo[a1] = hi[a1] = fe[a1] + b1;
                      lo[a2] = hi[a2] = fe[a2] + b2;
                      grad += w * (__ldcg(s.Tf + node_id(s.fg, hi[0], hi[1], hi[2])) -
                                   __ldcg(s.Tf + node_id(s.fg, lo[0], lo[1], lo[2]))) / hf[d];
                    }
                  // the coarse hat of node ci on this coarse face, bilinear in the plane
                  const double t1 = (f1 + xi1) / s.r, t2 = (f2 + xi2) / s.r;
                  const double phi = (c1 == ci[a1] - 1 ? t1 : 1.0 - t1) * (c2 == ci[a2] - 1 ? t2 : 1.0 - t2);
                  Gsum += jump * (sign * grad) * 0.25 * hf[a1] * hf[a2] * phi;
                }
            }
        }
    }
    s.G[node_id(s.cg, ci[0], ci[1], ci[2])] = Gsum;
  }
}

// Takes the last solve of a level out of the energy account (a solve the
// iterated coupling supersedes).  One thread.
__global__ void energy_rollback_kernel(DevStats* s, int lvl) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    s->e_stored[lvl] -= s->e_last[lvl][0];
    s->e_laser[lvl] -= s->e_last[lvl][1];
    s->e_flux[lvl] -= s->e_last[lvl][2];
    s->e_loss[lvl] -= s->e_last[lvl][3];
  }
}

// out[0] = max |a - b|, out[1] = max |a| as IEEE bit patterns (the order of
// non-negative doubles is the order of their patterns, so the atomic maximum
// is exact and independent of the schedule).  out must start at zero.
__global__ void max_diff_kernel(const double* __restrict__ a, const double* __restrict__ b, long long n,
                                unsigned long long* out) {
  double d = 0.0, m = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double x = a[i];
    d = fmax(d, fabs(x - b[i]));
    m = fmax(m, fabs(x));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    d = fmax(d, __shfl_down_sync(0xffffffffu, d, o));
    m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(out, (unsigned long long)__double_as_longlong(d));
    atomicMax(out + 1, (unsigned long long)__double_as_longlong(m));
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
