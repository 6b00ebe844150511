// Shared device-side building blocks: model constants, periodic indexing,
// warp/block reductions and the deterministic grid reduction used by every
// kernel that produces a scalar.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "moto.h"

namespace moto {

constexpr int kThreads = 256;         // block size of the streaming kernels
constexpr int kSMs = 152;             // GB300: 2 dies x 76 SMs
constexpr int kStreamBlocks = 2 * kSMs;  // persistent-style grid of the vector kernels

// Device copy of the model.  Shell offsets are compile-time constants in
// stencil.cuh; only strengths and sizes travel here.  A general pair-list
// model (npairs > 0) replaces the shells and the Neel DMI: pairs holds
// npairs records [d1, d2, J, Dx, Dy, Dz] in device memory, reach the largest
// |d1|, |d2| (kernels_pairs.cu).
struct ModelDev {
  int L1, L2, N, n_shells;
  double J[3];
  double D, K, muB;
  const double* pairs = nullptr;
  int npairs = 0, reach = 0;
};

// Status bits written by kernels into the context's status word.
enum : int {
  kStatusNonfinite = 1,
  kStatusBreakdown = 2,
  kStatusNotSPD = 4,
  kStatusTimeout = 8,
};

// Walker batches: a launch may serve several walkers whose scratch and fields
// lie at equal offsets of equally sized slices of one allocation.  The walker
// is blockIdx.z; its pointers are the first walker's plus z * ws bytes
// (ws == 0: a single walker, pointers unchanged).
template <typename P>
__device__ __forceinline__ P* wofs(P* p, size_t ws) {
  return (ws != 0 && p != nullptr) ? reinterpret_cast<P*>(reinterpret_cast<uintptr_t>(p) + (size_t)blockIdx.z * ws)
                                   : p;
}

__device__ __forceinline__ int wrap(int a, int L) {
  a %= L;
  return a < 0 ? a + L : a;
}

// ---------------------------------------------------------------------------
// reductions
// ---------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Sum of NV values over the block in a fixed order; result valid in thread 0.
// scratch: at least NV * (blockDim/32) doubles of shared memory.
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double* scratch) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int j = 0; j < NV; ++j) v[j] = warp_sum(v[j]);
  if (lane == 0) {
#pragma unroll
    for (int j = 0; j < NV; ++j) scratch[j * nw + wid] = v[j];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int j = 0; j < NV; ++j) {
      double a = 0.0;
      for (int w = 0; w < nw; ++w) a += scratch[j * nw + w];
      v[j] = a;
    }
  }
  __syncthreads();
}

__device__ __forceinline__ double block_max(double v, double* scratch) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = warp_max(v);
  if (lane == 0) scratch[wid] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = scratch[0];
    for (int w = 1; w < nw; ++w) a = fmax(a, scratch[w]);
    v = a;
  }
  __syncthreads();
  return v;
}

// Deterministic grid reduction.  Every block has written `nv` partial values at
// part[blockIdx.x * nv + j] (thread 0, before calling).  The last block to
// arrive reduces them in block-index order (sum, or max where is_max[j]) and
// returns true in all of its threads with the totals in `tot` (shared memory,
// nv doubles); it also resets the arrival counter for the next launch.
__device__ __forceinline__ bool grid_last_block(unsigned* counter) {
  __shared__ bool last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned t = atomicAdd(counter, 1u);
    last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (last) __threadfence();
  return last;
}

// Inside the last block: tot[j] = sum_b part[b * nv + j] in an order fixed by
// (nblocks, nv, blockDim), so the result does not depend on which block came
// last.  Few blocks: a thread per entry adds the blocks in index order (loads
// issued eight at a time); many blocks and few entries: a warp per entry, lane
// l adding blocks l, l + 32, ... in order, then a fixed shuffle tree.
__device__ __forceinline__ void grid_sum_entries(const double* part, int nblocks, int nv, double* tot) {
  if (nblocks <= 256 || nv >= (int)blockDim.x) {
    for (int j = threadIdx.x; j < nv; j += blockDim.x) {
      double a = 0.0;
      int b = 0;
      for (; b + 8 <= nblocks; b += 8) {
        double v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = __ldcg(part + (size_t)(b + u) * nv + j);
#pragma unroll
        for (int u = 0; u < 8; ++u) a += v[u];
      }
      for (; b < nblocks; ++b) a += __ldcg(part + (size_t)b * nv + j);
      tot[j] = a;
    }
  } else {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int j = wid; j < nv; j += nw) {
      double a = 0.0;
      for (int b = lane; b < nblocks; b += 32) a += __ldcg(part + (size_t)b * nv + j);
      a = warp_sum(a);
      if (lane == 0) tot[j] = a;
    }
  }
}

// Two-float numbers hi + lo (|lo| <= ulp(hi) / 2) and their sum after
// Knuth's TwoSum (the rounding error of hi + hi carried into lo): about 44
// significant bits in FP32 instructions.  Reductions of FP32 fields with
// thousands of additions a block (tens of thousands in the last block) use
// them instead of FP64, whose pipe on GB300 is a small fraction of FP32's.
struct F2 {
  float hi, lo;
};
__device__ __forceinline__ F2 f2_of(float a) { return F2{a, 0.f}; }
__device__ __forceinline__ F2 radd(F2 a, F2 b) {
  const float s = a.hi + b.hi;
  const float bb = s - a.hi;
  float e = (a.hi - (s - bb)) + (b.hi - bb);
  e += a.lo + b.lo;
  const float hi = s + e;
  return F2{hi, e - (hi - s)};
}
__device__ __forceinline__ double radd(double a, double b) { return a + b; }
__device__ __forceinline__ F2 rshfl(F2 a, int o) {
  return F2{__shfl_xor_sync(0xffffffffu, a.hi, o), __shfl_xor_sync(0xffffffffu, a.lo, o)};
}
__device__ __forceinline__ double rshfl(double a, int o) { return __shfl_xor_sync(0xffffffffu, a, o); }

// Last block: out[j] = sum over the blocks b of part[b * nv + j] (two-float),
// in an order fixed by (nb, nv, blockDim): C chunks of consecutive blocks per
// entry (C = blockDim / nv, 1 to 8) are summed by separate threads with eight
// loads in flight, then the chunks in order.  scratch: C * nv entries.
__device__ __forceinline__ void grid_sum_f2(const F2* part, int nb, int nv, double* out, F2* scratch) {
  int C = (int)blockDim.x / nv;
  C = C < 1 ? 1 : (C > 8 ? 8 : C);
  const int S = (nb + C - 1) / C;
  for (int t = threadIdx.x; t < nv * C; t += blockDim.x) {
    const int j = t % nv, c = t / nv;
    const int b1 = min(nb, (c + 1) * S);
    F2 a = F2{0.f, 0.f};
    int b = c * S;
    for (; b + 8 <= b1; b += 8) {
      float2 v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) v[u] = __ldcg(reinterpret_cast<const float2*>(part + (size_t)(b + u) * nv + j));
#pragma unroll
      for (int u = 0; u < 8; ++u) a = radd(a, F2{v[u].x, v[u].y});
    }
    for (; b < b1; ++b) {
      const float2 v = __ldcg(reinterpret_cast<const float2*>(part + (size_t)b * nv + j));
      a = radd(a, F2{v.x, v.y});
    }
    scratch[t] = a;
  }
  __syncthreads();
  for (int j = threadIdx.x; j < nv; j += blockDim.x) {
    F2 a = scratch[j];
    for (int c = 1; c < C; ++c) a = radd(a, scratch[c * nv + j]);
    out[j] = (double)a.hi + (double)a.lo;
  }
}

__device__ __forceinline__ void grid_max_entries(const double* part, int nblocks, int nv, double* tot) {
  for (int j = threadIdx.x; j < nv; j += blockDim.x) {
    double a = -1.0 / 0.0;
    for (int b = 0; b < nblocks; ++b) a = fmax(a, __ldcg(part + (size_t)b * nv + j));
    tot[j] = a;
  }
}

template <typename T>
__device__ __forceinline__ bool finite3(T a, T b, T c) {
  return isfinite((double)a) && isfinite((double)b) && isfinite((double)c);
}

}  // namespace moto
