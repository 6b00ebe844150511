// Explorer front-end (Results, "Multi-objective initial-configuration
// explorer"): masked perturbations x = R_x0(P_Omega P_x0 delta) of a reference
// configuration, and the pairwise L1 distances of a population that its
// diversity objective is built from.
//
// Pairwise L1: a block streams tiles of kTE elements of every candidate
// through shared memory; thread (block pair, slice) owns the 4 x 4 distances
// between candidates 4i .. 4i+3 and 4j .. 4j+3 (i <= j) and adds |x_a - x_b|
// over every nslice-th element of a tile, so each staged value feeds four
// distances.  FP32 sums are promoted to FP64 every kFlushT tiles; slices,
// blocks and the grid are summed in FP64 in a fixed order.
#include <algorithm>

#include "internal.h"

namespace moto {

namespace {
constexpr int kTE = 128;      // elements per staged tile
constexpr int kSX = kTE + 1;  // staged row stride: rows of one column fall in different banks
constexpr int kFlushT = 32;   // tiles between FP32 -> FP64 promotions
constexpr int kPThreads = 256;
// staged values per thread per tile: populations of up to 24 / up to 64
constexpr int kPrefetchSmall = 24 * kTE / kPThreads, kPrefetchLarge = 4 * ((MOTO_MAX_POP + 3) / 4) * kTE / kPThreads;
}  // namespace

template <typename T>
__global__ void __launch_bounds__(kThreads) perturb_kernel(const T* __restrict__ x0, const unsigned char* mask,
                                                           const T* __restrict__ delta, size_t ldd, int count,
                                                           T* out, size_t ldo, int N) {
  const int j = blockIdx.y;
  if (j >= count) return;
  const T* dj = delta + (size_t)j * ldd;
  T* oj = out + (size_t)j * ldo;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    T m0 = x0[i], m1 = x0[N + i], m2 = x0[2 * (size_t)N + i];
    if (!mask || mask[i]) {
      T d0 = dj[i], d1 = dj[N + i], d2 = dj[2 * (size_t)N + i];
      const T p = m0 * d0 + m1 * d1 + m2 * d2;
      d0 -= p * m0;
      d1 -= p * m1;
      d2 -= p * m2;
      // Rodrigues rotation by the tangent step, then unit length
      const T th = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
      if (th > (T)0) {
        T sn, cs;
        if constexpr (sizeof(T) == 4) {
          sincosf(th, &sn, &cs);
        } else {
          sincos(th, &sn, &cs);
        }
        const T f = sn / th;
        m0 = m0 * cs + d0 * f;
        m1 = m1 * cs + d1 * f;
        m2 = m2 * cs + d2 * f;
      }
      const T inv = (T)1 / sqrt(m0 * m0 + m1 * m1 + m2 * m2);
      m0 *= inv;
      m1 *= inv;
      m2 *= inv;
    }
    oj[i] = m0;
    oj[N + i] = m1;
    oj[2 * (size_t)N + i] = m2;
  }
}

template <typename T, int kPrefetch>
__global__ void __launch_bounds__(kPThreads) pairwise_l1_kernel(const T* __restrict__ X, size_t ldx, int P,
                                                                size_t n, double* part, unsigned* counter,
                                                                double* D) {
  extern __shared__ __align__(16) unsigned char ex_raw[];
  T* Xs = reinterpret_cast<T*>(ex_raw);  // [4 nb][kSX]
  const int nb = (P + 3) / 4, nbp = nb * (nb + 1) / 2;
  const int nsl = blockDim.x / nbp;
  const int tid = threadIdx.x, bp = tid % nbp, slice = tid / nbp;
  const bool active = slice < nsl;
  // block pair bp -> (bi, bj), bi <= bj, row-major over the upper triangle
  int bi = 0, bj = 0;
  {
    int r = bp;
    while (r >= nb - bi) {
      r -= nb - bi;
      ++bi;
    }
    bj = bi + r;
  }
  float acc[4][4];
  double dacc[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      acc[r][c] = 0.f;
      dacc[r][c] = 0.0;
    }
  const size_t ntiles = (n + kTE - 1) / kTE;
  const int total = 4 * nb * kTE;  // staged values per tile, <= kPrefetch * kPThreads
  // the next tile's values wait in registers while the current one is used
  T nxt[kPrefetch];
  auto fetch = [&](size_t t) {
#pragma unroll
    for (int u = 0; u < kPrefetch; ++u) {
      const int idx = tid + u * kPThreads;
      if (idx < total) {
        const int a = idx / kTE, e = idx - a * kTE;
        const size_t g = t * kTE + e;
        nxt[u] = (a < P && g < n) ? X[(size_t)a * ldx + g] : (T)0;
      }
    }
  };
  if (blockIdx.x < ntiles) fetch(blockIdx.x);
  int since = 0;
  for (size_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    __syncthreads();
#pragma unroll
    for (int u = 0; u < kPrefetch; ++u) {
      const int idx = tid + u * kPThreads;
      if (idx < total) {
        const int a = idx / kTE, e = idx - a * kTE;
        Xs[a * kSX + e] = nxt[u];
      }
    }
    __syncthreads();
    if (t + gridDim.x < ntiles) fetch(t + gridDim.x);
    if (active) {
      for (int e = slice; e < kTE; e += nsl) {
        T xa[4], xb[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          xa[r] = Xs[(4 * bi + r) * kSX + e];
          xb[r] = Xs[(4 * bj + r) * kSX + e];
        }
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            if constexpr (sizeof(T) == 4)
              acc[r][c] += fabsf(xa[r] - xb[c]);
            else
              dacc[r][c] += fabs((double)xa[r] - (double)xb[c]);
          }
      }
      if (sizeof(T) == 4 && ++since == kFlushT) {
        since = 0;
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            dacc[r][c] += (double)acc[r][c];
            acc[r][c] = 0.f;
          }
      }
    }
  }
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) dacc[r][c] += (double)acc[r][c];
  // slices of a block pair summed in slice order, then the block's partials
  __syncthreads();
  double* red = reinterpret_cast<double*>(ex_raw);  // [nsl][nbp][16]
  if (active)
#pragma unroll
    for (int q = 0; q < 16; ++q) red[((size_t)slice * nbp + bp) * 16 + q] = dacc[q >> 2][q & 3];
  __syncthreads();
  const int nent = nbp * 16;
  for (int o = tid; o < nent; o += blockDim.x) {
    double a = 0.0;
    for (int s = 0; s < nsl; ++s) a += red[(size_t)s * nent + o];
    part[(size_t)blockIdx.x * nent + o] = a;
  }
  if (!grid_last_block(counter)) return;
  __syncthreads();
  grid_sum_entries(part, gridDim.x, nent, red);
  __syncthreads();
  for (int o = tid; o < nent; o += blockDim.x) {
    const int p = o >> 4, q = o & 15;
    int i = 0, r = p;
    while (r >= nb - i) {
      r -= nb - i;
      ++i;
    }
    const int j = i + r;
    const int a = 4 * i + (q >> 2), b = 4 * j + (q & 3);
    if (a < P && b < P && a < b) {
      D[a * P + b] = red[o];
      D[b * P + a] = red[o];
    }
    if (a < P && a == b) D[a * P + a] = 0.0;
  }
  if (tid == 0) *counter = 0u;
}

template <typename T>
void launch_perturb(const T* x0, const unsigned char* mask, const T* delta, size_t ldd, int count, T* out,
                    size_t ldo, int N, cudaStream_t st) {
  size_t b = ((size_t)N + kThreads - 1) / kThreads;
  const size_t cap = (size_t)kSMs * 4;
  if (b > cap) b = cap;
  if (b < 1) b = 1;
  const dim3 grid((unsigned)b, (unsigned)count);
  perturb_kernel<T><<<grid, kThreads, 0, st>>>(x0, mask, delta, ldd, count, out, ldo, N);
}

template <typename T>
bool launch_pairwise_l1(const T* X, size_t ldx, int P, size_t n, double* part, size_t part_cap, unsigned* counter,
                        double* D, cudaStream_t st) {
  if (P < 2 || P > MOTO_MAX_POP) return false;
  const int nb = (P + 3) / 4, nbp = nb * (nb + 1) / 2, nent = nbp * 16;
  const int nsl = kPThreads / nbp;
  size_t smem = (size_t)4 * nb * kSX * sizeof(T);
  smem = std::max(smem, ((size_t)nsl * nent) * sizeof(double));
  smem = std::max(smem, (size_t)nent * sizeof(double));
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(pairwise_l1_kernel<T, kPrefetchSmall>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         96 * 1024);
    cudaFuncSetAttribute(pairwise_l1_kernel<T, kPrefetchLarge>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         96 * 1024);
    attr = true;
  }
  if (smem > 96 * 1024) return false;
  const size_t ntiles = (n + kTE - 1) / kTE;
  size_t g = std::min<size_t>(ntiles, (size_t)kSMs * 2);
  g = std::min<size_t>(g, part_cap / (size_t)nent);
  if (g < 1) return false;
  if (4 * nb * kTE <= kPrefetchSmall * kPThreads)
    pairwise_l1_kernel<T, kPrefetchSmall><<<(int)g, kPThreads, smem, st>>>(X, ldx, P, n, part, counter, D);
  else
    pairwise_l1_kernel<T, kPrefetchLarge><<<(int)g, kPThreads, smem, st>>>(X, ldx, P, n, part, counter, D);
  return true;
}

#define INST(T)                                                                                                  \
  template void launch_perturb<T>(const T*, const unsigned char*, const T*, size_t, int, T*, size_t, int,       \
                                  cudaStream_t);                                                                 \
  template bool launch_pairwise_l1<T>(const T*, size_t, int, size_t, double*, size_t, unsigned*, double*,       \
                                      cudaStream_t);
INST(float)
INST(double)
#undef INST

}  // namespace moto
