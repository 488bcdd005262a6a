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
};

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
// Time-limited grid barrier for cooperative (co-resident) launches.
// Two-level arrival: blocks arrive on the counter of their group of
// BAR_GROUP consecutive blocks; the last of a group arrives on the root
// counter; the last group releases the generation word.  Every wait gives up
// after `limit_ns` of global time, records ST_TIMEOUT and returns false; a
// block that sees an error recorded by another returns false too, so that all
// blocks leave the kernel.
// Word layout (BAR_WORDS unsigned ints, zero at creation): [0] root counter,
// [1 .. BAR_MAXG] group counters, [BAR_GEN] generation, [BAR_STATUS] status.
// ---------------------------------------------------------------------------
// The block range a solve runs on: a whole cooperative grid, or one job's
// slice of a batched grid.  bid is the block's index within the slice.
struct VGrid {
  int bid, nblk;
};

constexpr int BAR_GROUP = 32;
constexpr int BAR_MAXG = 64;
constexpr int BAR_GEN = BAR_MAXG + 1;
constexpr int BAR_STATUS = BAR_MAXG + 2;
constexpr int BAR_WORDS = BAR_MAXG + 3;

struct Barrier {
  unsigned int* count;  // root counter followed by the group counters
  unsigned int* gen;
  int* status;          // sticky device status word
};

__device__ inline unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ inline unsigned int ld_acquire_u32(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ inline void st_release_u32(unsigned int* p, unsigned int v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ inline int ld_volatile_i32(const int* p) {
  return *(volatile const int*)p;
}

__device__ inline bool grid_sync(const Barrier& b, const VGrid& vg, unsigned long long limit_ns = 1000000000ull) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    const unsigned int g = ld_acquire_u32(b.gen);
    __threadfence();
    const unsigned int grp = (unsigned int)vg.bid / BAR_GROUP;
    const unsigned int ngroups = ((unsigned int)vg.nblk + BAR_GROUP - 1) / BAR_GROUP;
    const unsigned int gsize = min((unsigned int)BAR_GROUP, (unsigned int)vg.nblk - grp * BAR_GROUP);
    bool released = false;
    if (atomicAdd(b.count + 1 + grp, 1u) == gsize - 1) {
      __threadfence();  // acquire side: the group's arrivals
      atomicExch(b.count + 1 + grp, 0u);
      if (atomicAdd(b.count, 1u) == ngroups - 1) {
        __threadfence();  // acquire side: every group's arrival
        atomicExch(b.count, 0u);
        st_release_u32(b.gen, g + 1u);
        released = true;
      }
    }
    if (!released) {
      const unsigned long long t0 = global_ns();
      while (ld_acquire_u32(b.gen) == g) {
        if (ld_volatile_i32(b.status) == ST_TIMEOUT) { ok = 0; break; }
        if (global_ns() - t0 > limit_ns) {
          atomicExch(b.status, (int)ST_TIMEOUT);
          ok = 0;
          break;
        }
        __nanosleep(32);
      }
    }
    if (ld_volatile_i32(b.status) == ST_TIMEOUT) ok = 0;
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// ---------------------------------------------------------------------------
// Deterministic reductions in the solve's own precision: per-thread partial ->
// warp sum (fixed shuffle tree) -> per-warp partials in shared memory -> one
// warp sums them -> one slot per block; after a grid barrier warp 0 of every
// block sums the slots in the same fixed order, so all blocks hold bitwise
// equal totals.  On GB300 an FP64 warp instruction occupies the SM
// sub-partition's FP64 unit for ~64 cycles, so FP32 solves reduce in FP32.
// ---------------------------------------------------------------------------
// One shared scratch for all reductions of a kernel (a static array in a
// template would be allocated once per instantiation): per-warp partials of up
// to RED_NV values, the block totals, and a few scalars (red_scalars) that the
// CG broadcasts after a reduction.  The users never overlap in time.
constexpr int RED_NV = 3;
__device__ inline double* red_scratch() {
  __shared__ double buf[RED_NV * 32 + RED_NV + 4];
  return buf;
}
template <typename T>
__device__ inline T* red_scalars() {
  return reinterpret_cast<T*>(red_scratch() + RED_NV * 32 + RED_NV);
}

template <int NV, typename T>
__device__ inline void block_reduce_store(T (&v)[NV], T* slots, int stride, const VGrid& vg) {
  static_assert(NV <= RED_NV && sizeof(T) <= sizeof(double), "reduction scratch");
  T (*s_part)[32] = reinterpret_cast<T (*)[32]>(red_scratch());
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarps = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int a = 0; a < NV; ++a) {
    T x = v[a];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if (lane == 0) s_part[a][warp] = x;
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int a = 0; a < NV; ++a) {
      T x = lane < nwarps ? s_part[a][lane] : T(0);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
      if (lane == 0) slots[(size_t)a * stride + vg.bid] = x;
    }
  }
  __syncthreads();
}

// Every thread of the block loads up to four slots per value at once (one L2
// round trip for grids of up to 4 x blockDim blocks), then the block sums them
// in a fixed tree.
template <int NV, typename T>
__device__ inline void grid_total(const T* slots, int stride, T (&out)[NV], const VGrid& vg) {
  static_assert(NV <= RED_NV && sizeof(T) <= sizeof(double), "reduction scratch");
  T (*s_part)[32] = reinterpret_cast<T (*)[32]>(red_scratch());
  T* s_tot = reinterpret_cast<T*>(red_scratch() + RED_NV * 32);
  constexpr int U = 4;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarps = (blockDim.x + 31) >> 5;
  T x[NV];
#pragma unroll
  for (int a = 0; a < NV; ++a) x[a] = T(0);
  for (int s0 = threadIdx.x; s0 < vg.nblk; s0 += U * blockDim.x) {
    T v[NV][U];
#pragma unroll
    for (int a = 0; a < NV; ++a)
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int s = s0 + u * blockDim.x;
        v[a][u] = s < vg.nblk ? __ldcg(slots + (size_t)a * stride + s) : T(0);
      }
#pragma unroll
    for (int a = 0; a < NV; ++a)
#pragma unroll
      for (int u = 0; u < U; ++u) x[a] += v[a][u];
  }
#pragma unroll
  for (int a = 0; a < NV; ++a) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x[a] += __shfl_down_sync(0xffffffffu, x[a], o);
    if (lane == 0) s_part[a][warp] = x[a];
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int a = 0; a < NV; ++a) {
      T y = lane < nwarps ? s_part[a][lane] : T(0);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) y += __shfl_down_sync(0xffffffffu, y, o);
      if (lane == 0) s_tot[a] = y;
    }
  }
  __syncthreads();
#pragma unroll
  for (int a = 0; a < NV; ++a) out[a] = s_tot[a];
  __syncthreads();
}

}  // namespace tl
