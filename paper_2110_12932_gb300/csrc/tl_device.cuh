// Device-side building blocks of the two-level LPBF heat solve (sm_103a).
//
// Discretisation: one backward-Euler step of the heat equation (Section 2.1,
// Eq. thermalEqn, without the latent term) on a uniform mesh of trilinear
// hexahedra, with element-constant s_e = rho c_e / dt and k_e:
//     (sum_e s_e Mhat + k_e Khat) T^{k+1} = (sum_e s_e Mhat) T^k + F.
// On a box element both element matrices are Kronecker products of the 1D
// matrices M1 = (h/6)[[2,1],[1,2]] and K1 = (1/h)[[1,-1],[-1,1]], which share
// the eigenvectors [1,1] and [1,-1].  With the 2-point Hadamard transform H the
// element operator is therefore H3 diag(lambda_e) H3 with eight eigenvalues
//     lambda_e[m] = s_e Mc[m] + k_e Kc[m]   (the 1/8 of H3^-1 folded in),
// so a matrix-free apply costs one forward and one backward separable
// Hadamard transform plus eight multiplies per element.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace tl {

enum : uint8_t { POWDER = 0, SOLID = 1, MELTED = 2 };

enum Status : int {
  ST_OK = 0,
  ST_NOCONV = -3,
  ST_TIMEOUT = -6,
};

struct Material {
  double rho, c0, c1, k0, k1, Tref, powder_factor, T_melt;
  double chi, S, Tm;  // latent heat [J/kg] (0: none), sigmoid sharpness [1/K], centre [K]
};

// Latent heat per element (the phase-change term of Eq. thermalEqn under
// backward Euler, chi rho (f_pc(T^{k+1}) - f_pc(T^k)) / dt): the secant
// (f_pc(Tb) - f_pc(Tb0)) / (Tb - Tb0) of the sigmoid
// f_pc(T) = (1 + tanh(S (T - Tm))) / 2 between the element means Tb (where the
// coefficients are taken) and Tb0 (the step's start); its derivative
// (S/2)(1 - tanh^2(S (T - Tm))) at the midpoint when |S (Tb - Tb0)| < 1e-3.
__device__ inline double fpc_secant(const Material& m, double Tb, double Tb0) {
  const double d = Tb - Tb0;
  if (fabs(m.S * d) < 1e-3) {
    const double th = tanh(m.S * (0.5 * (Tb + Tb0) - m.Tm));
    return 0.5 * m.S * (1.0 - th * th);
  }
  const double f1 = 0.5 * (1.0 + tanh(m.S * (Tb - m.Tm)));
  const double f0 = 0.5 * (1.0 + tanh(m.S * (Tb0 - m.Tm)));
  return (f1 - f0) / d;
}

struct Grid3 {
  int nx, ny, nz;     // elements
  int nnx, nny, nnz;  // nodes (n* = elements + 1)
  double hx, hy, hz;
};

__host__ __device__ inline long long node_id(const Grid3& g, int i, int j, int k) {
  return (long long)i + (long long)g.nnx * ((long long)j + (long long)g.nny * k);
}
__host__ __device__ inline long long elem_id(const Grid3& g, int i, int j, int k) {
  return (long long)i + (long long)g.nx * ((long long)j + (long long)g.ny * k);
}

// Balanced split of n items into parts: part a covers [a n / parts, (a+1) n / parts).
__host__ __device__ inline int split_lo(int n, int parts, int a) {
  return (int)(((long long)a * n) / parts);
}

// ---------------------------------------------------------------------------
// Time-limited grid barrier for cooperative (co-resident) launches.  One
// 64-bit word holds the arrivals (low half) and the generation (high half):
// every block arrives with one atomic add; the block whose add completes the
// count releases the next generation with a second add that also clears the
// count.  (Measured on GB300 with 152 to 608 blocks: 2.2 - 2.4 us per
// barrier for the one-counter scheme, against 2.9 - 3.2 us with a two-level
// tree of 32-block groups; the arrivals on one word do not queue noticeably
// at this block count.)
// A barrier either releases every block or none: a block whose wait exceeds
// the time limit withdraws its arrival (compare-and-swap, possible only while
// some block has not arrived, so the count can no longer complete), records
// ST_TIMEOUT and returns false; a waiting block that sees ST_TIMEOUT returns
// false too, so that all blocks leave the kernel at the same barrier and no
// block runs a phase that another skipped.  Once the count is complete no
// block gives up: the release follows.
// Word layout (BAR_WORDS unsigned ints, zero at creation): [0..1] the 64-bit
// arrival / generation word, [BAR_STATUS] the sticky status word.
// ---------------------------------------------------------------------------
// The block range a solve runs on: a whole cooperative grid, or one job's
// slice of a batched grid.  bid is the block's index within the slice.
struct VGrid {
  int bid, nblk;
};

constexpr int BAR_STATUS = 2;
constexpr int BAR_WORDS = 4;
constexpr unsigned long long BAR_DEFAULT_LIMIT_NS = 1000000000ull;

struct Barrier {
  unsigned long long* word;  // arrivals | generation << 32
  int* status;               // sticky device status word
  unsigned long long limit_ns;  // time limit of every wait
};

__device__ inline unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ inline unsigned long long ld_acquire_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ inline void atom_add_release_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
// Arrival: one RMW with acquire and release semantics.  Every arrival and the
// release are RMWs of the same word, so they form one release sequence: the
// last arrival acquires every earlier block's writes, and a waiter that
// acquires the released generation sees all of them (no separate fences).
__device__ inline unsigned long long atom_add_acqrel_u64(unsigned long long* p, unsigned long long v) {
  unsigned long long o;
  asm volatile("atom.acq_rel.gpu.global.add.u64 %0, [%1], %2;" : "=l"(o) : "l"(p), "l"(v) : "memory");
  return o;
}
__device__ inline int ld_volatile_i32(const int* p) {
  return *(volatile const int*)p;
}
// The barriers' result flag, shared by all of a kernel's barrier calls.
__device__ inline int* bar_ok_flag() {
  __shared__ int ok;
  return &ok;
}

// Each block keeps the generation of its next barrier in shared memory (thread
// 0 reads and writes it), read once per launch by bar_begin (at a launch's
// start every reset of the previous launch has been applied): every use of a
// barrier moves the generation by exactly one, so the copy stays exact, and
// the arrival path needs no read of the word.
__device__ inline unsigned int* bar_gen_local() {
  __shared__ unsigned int gen;
  return &gen;
}
__device__ inline void bar_begin(const Barrier& b) {
  if (threadIdx.x == 0) *bar_gen_local() = (unsigned int)(ld_acquire_u64(b.word) >> 32);
  __syncthreads();
}

// Arrivals still counted in the word for barrier g (the block's local
// generation) when the word reads w: the generation part of w may lag g by
// the resets not yet applied, each of which will take nblk away.
__device__ inline unsigned int bar_count(unsigned long long w, unsigned int g, int nblk) {
  return (unsigned int)w - (g - (unsigned int)(w >> 32)) * (unsigned int)nblk;
}

// Waits (thread 0) until barrier g is complete; false if the time limit
// passed (the arrival is withdrawn and the time-out recorded) or another block
// recorded a time-out.  The barrier is complete once its count reaches nblk
// or its reset (generation g + 1) has been applied.  Once complete, the wait
// never gives up.  The status word and the clock are looked at every 16th
// poll, or at every poll under a limit shorter than a millisecond.
__device__ inline bool bar_wait(const Barrier& b, unsigned int g, int nblk) {
  const unsigned long long t0 = global_ns();
  const bool every = b.limit_ns < 1000000ull;
  for (unsigned int poll = 1;; ++poll) {
    unsigned long long w = ld_acquire_u64(b.word);
    if ((unsigned int)(w >> 32) == g + 1u || bar_count(w, g, nblk) >= (unsigned int)nblk) return true;
    if (every || (poll & 15) == 0) {
      if (ld_volatile_i32(b.status) == ST_TIMEOUT) return false;
      if (global_ns() - t0 > b.limit_ns) {
        for (;;) {  // withdraw the arrival while the count is incomplete
          if ((unsigned int)(w >> 32) == g + 1u || bar_count(w, g, nblk) >= (unsigned int)nblk) return true;
          const unsigned long long prev = atomicCAS(b.word, w, w - 1ull);
          if (prev == w) {
            atomicExch(b.status, (int)ST_TIMEOUT);
            return false;
          }
          w = prev;
        }
      }
    }
    __nanosleep(32);
  }
}

// All arrivals are RMWs of one word (acquire-release), so a waiter that
// acquires a value at or after the last arrival sees every block's writes.
// Waiters pass as soon as the count is complete; the last arrival then resets
// the count and moves the generation with one more add, which may land after
// blocks have already arrived at the next barrier (bar_count accounts for it).
__device__ inline bool grid_sync(const Barrier& b, const VGrid& vg) {
  int* s_ok = bar_ok_flag();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned int g = *bar_gen_local();
    bool ok = true;
    // the block barrier above orders the block's writes before thread 0's
    // release (cumulativity)
    const unsigned long long old = atom_add_acqrel_u64(b.word, 1ull);
    if (bar_count(old, g, vg.nblk) == (unsigned int)vg.nblk - 1u) {
      atom_add_release_u64(b.word, (1ull << 32) - (unsigned long long)(unsigned int)vg.nblk);
    } else {
      ok = bar_wait(b, g, vg.nblk);
    }
    *bar_gen_local() = g + 1u;
    *s_ok = ok;
  }
  __syncthreads();
  return *s_ok != 0;
}

// ---------------------------------------------------------------------------
// Deterministic reductions in the solve's own precision: per-thread partial ->
// block sum in a fixed order (block_reduce_store) -> one slot per block ->
// after a grid barrier every block forms the grid totals from the slots
// (grid_sync_total), bitwise equal in all blocks.  On GB300 an FP64 warp
// instruction occupies the SM sub-partition's FP64 unit for ~64 cycles, so
// the block sums keep FP64 additions few and the grid totals of FP64 slots
// are formed exactly in integer arithmetic; FP32 solves reduce in FP32.
// ---------------------------------------------------------------------------
// Reductions carry at most RED_NV values at once, over at most
// MAX_GRID_BLOCKS block slots (the exact FP64 totals rely on it).
constexpr int RED_NV = 3;
constexpr int MAX_GRID_BLOCKS = 2048;
// One shared scratch for all reductions of a kernel (a static array in a
// template would be allocated once per instantiation): the lane values of
// warps 1 .. RED_W (block_reduce_store) or per-warp partials (the grid
// totals), RED_NV totals, and a few scalars (red_scalars) that the CG
// broadcasts after a reduction.  The users never overlap in time.
constexpr int RED_W = 4;  // blocks of up to 32 (RED_W + 1) threads
__device__ inline double* red_scratch() {
  __shared__ double buf[RED_W * 32 + RED_NV + 4];
  return buf;
}
template <typename T>
__device__ inline T* red_totals() {
  return reinterpret_cast<T*>(red_scratch() + RED_W * 32);
}
template <typename T>
__device__ inline T* red_scalars() {
  return reinterpret_cast<T*>(red_scratch() + RED_W * 32 + RED_NV);
}

// Sum of one value over a warp, in a fixed shuffle tree (lane 0 holds it).
template <typename T>
__device__ inline T warp_sum(T x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
  return x;
}

// Block sums of NV values into slot vg.bid of NV rows.  Warps 1 .. RED_W park
// their lane values in shared memory and warp 0 alone adds: per value it adds
// those columns to its own lanes, then runs one shuffle tree (RED_W + 5 warp
// additions instead of a tree per warp; FP64 additions are the cost).
template <int NV, typename T>
__device__ inline void block_reduce_store(T (&v)[NV], T* slots, int stride, const VGrid& vg) {
  static_assert(NV <= RED_NV && sizeof(T) <= sizeof(double), "reduction scratch");
  T (*s_lane)[32] = reinterpret_cast<T (*)[32]>(red_scratch());
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarps = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int a = 0; a < NV; ++a) {
    if (a > 0) __syncthreads();  // warp 0 has read the previous value's columns
    if (warp > 0) s_lane[warp - 1][lane] = v[a];
    __syncthreads();
    if (warp == 0) {
      T x = v[a];
      for (int w = 1; w < nwarps; ++w) x += s_lane[w - 1][lane];
      x = warp_sum(x);
      if (lane == 0) slots[(size_t)a * stride + vg.bid] = x;
    }
  }
  __syncthreads();
}

// FP32 grid totals: every thread of the block loads up to four slots per
// value at once (one L2 round trip for grids of up to 4 x blockDim blocks),
// then the block sums them in a fixed tree.
template <int NV>
__device__ inline void grid_total(const float* slots, int stride, float (&out)[NV], const VGrid& vg) {
  static_assert(NV <= RED_NV && RED_W >= NV, "reduction scratch");
  float (*s_part)[32] = reinterpret_cast<float (*)[32]>(red_scratch());
  float* s_tot = red_totals<float>();
  constexpr int U = 4;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarps = (blockDim.x + 31) >> 5;
  float x[NV];
#pragma unroll
  for (int a = 0; a < NV; ++a) x[a] = 0.0f;
  for (int s0 = threadIdx.x; s0 < vg.nblk; s0 += U * blockDim.x) {
    float v[NV][U];
#pragma unroll
    for (int a = 0; a < NV; ++a)
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int s = s0 + u * blockDim.x;
        v[a][u] = s < vg.nblk ? __ldcg(slots + (size_t)a * stride + s) : 0.0f;
      }
#pragma unroll
    for (int a = 0; a < NV; ++a)
#pragma unroll
      for (int u = 0; u < U; ++u) x[a] += v[a][u];
  }
#pragma unroll
  for (int a = 0; a < NV; ++a) {
    x[a] = warp_sum(x[a]);
    if (lane == 0) s_part[a][warp] = x[a];
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int a = 0; a < NV; ++a) {
      float y = lane < nwarps ? s_part[a][lane] : 0.0f;
      y = warp_sum(y);
      if (lane == 0) s_tot[a] = y;
    }
  }
  __syncthreads();
#pragma unroll
  for (int a = 0; a < NV; ++a) out[a] = s_tot[a];
  __syncthreads();
}

// Biased exponent of a double given by its bits, 1 for subnormals (their
// scale), 0 for zeros.
__device__ inline int exp_eff(long long b) {
  const int e = (int)((b >> 52) & 0x7FF);
  return (e == 0 && (b & 0xFFFFFFFFFFFFFll) != 0) ? 1 : e;
}

// FP64 grid totals, summed exactly in integers.  For each value row, Emax is
// the largest biased exponent among the slots; every slot x = +-m 2^(e-1075)
// (m the 53-bit significand; subnormals: e = 1, no implicit bit) becomes the
// signed integer +-(m >> (Emax - e + 1)), a multiple of the unit
// 2^(Emax - 1074) truncated towards zero (each loses less than one unit, at
// most 2^-51 of the largest magnitude).  Each such integer is below 2^52, so
// the sum of up to 2^11 slots is exact in 64 bits and independent of the
// order of the additions; it is rounded to double once and scaled back.  The
// error, at most n units plus that rounding, is of the order of a plain FP64
// summation's bound, every block gets the same bits, and all the work runs
// on the integer pipes.  Warp sums use the 32-bit reduction instruction on
// three 21-bit limbs of each per-thread integer.  A non-finite slot makes the
// total NaN.
template <int NV>
__device__ inline void grid_total(const double* slots, int stride, double (&out)[NV], const VGrid& vg) {
  static_assert(NV <= RED_NV, "reduction scratch");
  constexpr int U = 4;  // slots a thread holds in registers; larger grids are read twice
  int* s_emax = reinterpret_cast<int*>(red_scratch());  // [RED_W + 1][RED_NV]
  int* s_limb = s_emax + (RED_W + 1) * RED_NV;           // [RED_W + 1][RED_NV][3]
  double* s_tot = red_totals<double>();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarps = (blockDim.x + 31) >> 5;
  const bool one_pass = vg.nblk <= U * (int)blockDim.x;
  long long bits[NV][U];  // zero (adds nothing) where the thread holds no slot
  int emax[NV];
#pragma unroll
  for (int a = 0; a < NV; ++a) {
    emax[a] = 0;
#pragma unroll
    for (int u = 0; u < U; ++u) bits[a][u] = 0ll;
  }
  for (int s0 = threadIdx.x; s0 < vg.nblk; s0 += U * blockDim.x) {
#pragma unroll
    for (int a = 0; a < NV; ++a)
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int s = s0 + u * blockDim.x;
        bits[a][u] = s < vg.nblk ? __double_as_longlong(__ldcg(slots + (size_t)a * stride + s)) : 0ll;
        emax[a] = max(emax[a], exp_eff(bits[a][u]));
      }
  }
#pragma unroll
  for (int a = 0; a < NV; ++a) {
    const int m = (int)__reduce_max_sync(0xffffffffu, (unsigned int)emax[a]);
    if (lane == 0) s_emax[warp * RED_NV + a] = m;
  }
  __syncthreads();
#pragma unroll
  for (int a = 0; a < NV; ++a) {
    int m = 0;
    for (int w = 0; w < nwarps; ++w) m = max(m, s_emax[w * RED_NV + a]);
    emax[a] = m;
  }
  // the thread's integers (exact: below 2^52 each, at most 2^11 of them)
  long long acc[NV];
#pragma unroll
  for (int a = 0; a < NV; ++a) acc[a] = 0;
  auto add = [&](int a, long long b) {
    const int e = (int)((b >> 52) & 0x7FF);
    if (e == 0x7FF) return;  // non-finite: Emax = 0x7FF, handled below
    const long long frac = b & 0xFFFFFFFFFFFFFll;
    const long long m = e ? (frac | (1ll << 52)) : frac;  // subnormal: no implicit bit, exponent 1
    const int sh = emax[a] - max(e, 1) + 1;
    const long long q = sh < 63 ? (m >> sh) : 0ll;
    acc[a] += b < 0 ? -q : q;
  };
  if (one_pass) {
#pragma unroll
    for (int a = 0; a < NV; ++a)
#pragma unroll
      for (int u = 0; u < U; ++u) add(a, bits[a][u]);
  } else {
    for (int s = threadIdx.x; s < vg.nblk; s += blockDim.x)
#pragma unroll
      for (int a = 0; a < NV; ++a) add(a, __double_as_longlong(__ldcg(slots + (size_t)a * stride + s)));
  }
  // limbs: acc = l0 + 2^21 l1 + 2^42 l2 with l0, l1 in [0, 2^21) and l2 signed
#pragma unroll
  for (int a = 0; a < NV; ++a) {
    const int l0 = (int)(acc[a] & 0x1FFFFF), l1 = (int)((acc[a] >> 21) & 0x1FFFFF), l2 = (int)(acc[a] >> 42);
    const int w0 = (int)__reduce_add_sync(0xffffffffu, (unsigned int)l0);
    const int w1 = (int)__reduce_add_sync(0xffffffffu, (unsigned int)l1);
    const int w2 = __reduce_add_sync(0xffffffffu, l2);
    if (lane == 0) {
      int* L = s_limb + (warp * RED_NV + a) * 3;
      L[0] = w0;
      L[1] = w1;
      L[2] = w2;
    }
  }
  __syncthreads();
  if (threadIdx.x < NV) {
    const int a = threadIdx.x;
    long long t = 0;
    for (int w = 0; w < nwarps; ++w) {
      const int* L = s_limb + (w * RED_NV + a) * 3;
      t += (long long)L[0] + ((long long)L[1] << 21) + ((long long)L[2] << 42);
    }
    double r;
    if (emax[a] == 0x7FF)
      r = __longlong_as_double(0x7FF8000000000000ll);
    else if (emax[a] == 0)
      r = 0.0;
    else
      r = ldexp(__ll2double_rn(t), emax[a] - 1074);
    s_tot[a] = r;
  }
  __syncthreads();
#pragma unroll
  for (int a = 0; a < NV; ++a) out[a] = s_tot[a];
  __syncthreads();
}

// Grid barrier followed by the grid totals of NV reduction rows (each block's
// slot values stored by block_reduce_store before the call).  Same time limit
// and error behaviour as grid_sync; on false the totals are undefined.
template <int NV, typename T>
__device__ inline bool grid_sync_total(const Barrier& b, const VGrid& vg, const T* slots, int stride, T (&out)[NV]) {
  if (!grid_sync(b, vg)) return false;
  grid_total<NV>(slots, stride, out, vg);
  return true;
}

}  // namespace tl
