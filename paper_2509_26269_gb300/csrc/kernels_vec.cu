// Vector-field kernels of the Krylov solvers and the L-BFGS ascent/descent:
// skinny Gram products (FP64-accumulated), site-wise combinations with
// tangent projection, Ritz finishing, and the small dense FP64 steps
// (Cholesky QR factors, Jacobi eigensolver, L-BFGS two-loop in coefficient
// space) that run in a single block.
#include <float.h>
#include <stdlib.h>
#include <string.h>

#include <type_traits>

#include "internal.h"

namespace moto {

// packed FP32 FMA on (x, y) pairs: each half rounds exactly like fma.rn.f32
__device__ __forceinline__ float2 ffma2v(float2 a, float2 b, float2 c) {
  unsigned long long d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;"
      : "=l"(d)
      : "l"(*reinterpret_cast<unsigned long long*>(&a)), "l"(*reinterpret_cast<unsigned long long*>(&b)),
        "l"(*reinterpret_cast<unsigned long long*>(&c)));
  return *reinterpret_cast<float2*>(&d);
}

// ===========================================================================
// Gram:  out[r][c] = X_r . Y_c
// ===========================================================================
constexpr int kGramKT = 64;  // elements per shared-memory tile

int gram_blocks() { return kStreamBlocks; }

template <typename T, int NY>
__global__ void __launch_bounds__(kThreads) gram_kernel(const T* __restrict__ X, size_t ldx, int nx,
                                                        const T* __restrict__ Y, size_t ldy, int ny, size_t n,
                                                        double* out, double* part, unsigned* counter,
                                                        const int* gate, int mask, size_t ws) {
  X = wofs(X, ws);
  Y = wofs(Y, ws);
  out = wofs(out, ws);
  part = wofs(part, ws);
  counter = wofs(counter, ws);
  gate = wofs(gate, ws);
  if (gate && (*gate & mask)) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int npairs = (nx + 1) >> 1;
  const int nxp = 2 * npairs + 2;  // padded row of the transposed X tile
  T* Xs = reinterpret_cast<T*>(smem_raw);
  T* Ys = Xs + kGramKT * nxp;
  const int nkg = blockDim.x / npairs;
  const int q = threadIdx.x % npairs, kg = threadIdx.x / npairs;
  const bool worker = kg < nkg;

  double acc64[2][NY];
  T mid[2][NY];
#pragma unroll
  for (int j = 0; j < 2; ++j)
#pragma unroll
    for (int c = 0; c < NY; ++c) {
      acc64[j][c] = 0.0;
      mid[j][c] = (T)0;
    }
  const size_t ntiles = (n + kGramKT - 1) / kGramKT;
  int since_flush = 0;
  for (size_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const size_t e0 = t * kGramKT;
    const int len = (int)min((size_t)kGramKT, n - e0);
    __syncthreads();
    for (int idx = threadIdx.x; idx < nx * kGramKT; idx += blockDim.x) {
      const int r = idx / kGramKT, k = idx - r * kGramKT;
      Xs[k * nxp + r] = k < len ? X[(size_t)r * ldx + e0 + k] : (T)0;
    }
    for (int idx = threadIdx.x; idx < kGramKT * nxp; idx += blockDim.x) {
      // zero the padding columns (r >= nx) once per tile
      const int k = idx / nxp, r = idx - k * nxp;
      if (r >= nx) Xs[idx] = (T)0;
      (void)k;
    }
    for (int idx = threadIdx.x; idx < NY * kGramKT; idx += blockDim.x) {
      const int c = idx / kGramKT, k = idx - c * kGramKT;
      Ys[k * NY + c] = (c < ny && k < len) ? Y[(size_t)c * ldy + e0 + k] : (T)0;
    }
    __syncthreads();
    if (worker) {
      T tacc[2][NY];
#pragma unroll
      for (int j = 0; j < 2; ++j)
#pragma unroll
        for (int c = 0; c < NY; ++c) tacc[j][c] = (T)0;
      for (int k = kg; k < kGramKT; k += nkg) {
        const T x0 = Xs[k * nxp + 2 * q], x1 = Xs[k * nxp + 2 * q + 1];
#pragma unroll
        for (int c = 0; c < NY; ++c) {
          const T y = Ys[k * NY + c];
          tacc[0][c] += x0 * y;
          tacc[1][c] += x1 * y;
        }
      }
#pragma unroll
      for (int j = 0; j < 2; ++j)
#pragma unroll
        for (int c = 0; c < NY; ++c) mid[j][c] += tacc[j][c];
      if (++since_flush == 16) {
        since_flush = 0;
#pragma unroll
        for (int j = 0; j < 2; ++j)
#pragma unroll
          for (int c = 0; c < NY; ++c) {
            acc64[j][c] += (double)mid[j][c];
            mid[j][c] = (T)0;
          }
      }
    }
  }
#pragma unroll
  for (int j = 0; j < 2; ++j)
#pragma unroll
    for (int c = 0; c < NY; ++c) acc64[j][c] += (double)mid[j][c];
  // block reduction over k-groups, fixed order
  __syncthreads();
  double* red = reinterpret_cast<double*>(smem_raw);  // nkg * npairs * 2 * NY doubles
  if (worker) {
#pragma unroll
    for (int j = 0; j < 2; ++j)
#pragma unroll
      for (int c = 0; c < NY; ++c) red[((size_t)kg * npairs + q) * 2 * NY + j * NY + c] = acc64[j][c];
  }
  __syncthreads();
  const int nout = nx * ny;
  for (int o = threadIdx.x; o < nout; o += blockDim.x) {
    const int r = o / ny, c = o - r * ny;
    const int qq = r >> 1, jj = r & 1;
    double a = 0.0;
    for (int g = 0; g < nkg; ++g) a += red[((size_t)g * npairs + qq) * 2 * NY + jj * NY + c];
    part[(size_t)blockIdx.x * nout + o] = a;
  }
  if (!grid_last_block(counter)) return;
  grid_sum_entries(part, gridDim.x, nout, out);
  if (threadIdx.x == 0) *counter = 0u;
}

template <typename T, int NY>
static void gram_launch_ny(const T* X, size_t ldx, int nx, const T* Y, size_t ldy, int ny, size_t n, double* out,
                           double* part, unsigned* counter, const int* gate, int mask, cudaStream_t st) {
  const int npairs = (nx + 1) / 2;
  const int nxp = 2 * npairs + 2;
  const int nkg = kThreads / npairs;
  size_t tile = (size_t)kGramKT * (nxp + NY) * sizeof(T);
  size_t red = (size_t)nkg * npairs * 2 * NY * sizeof(double);
  size_t smem = tile > red ? tile : red;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(gram_kernel<T, NY>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr = true;
  }
  const size_t ntiles = (n + kGramKT - 1) / kGramKT;
  const int grid = (int)(ntiles < (size_t)kStreamBlocks ? ntiles : (size_t)kStreamBlocks);
  gram_kernel<T, NY><<<wgrid(grid), kThreads, smem, st>>>(X, ldx, nx, Y, ldy, ny, n, out, part, counter, gate, mask, walker_ws());
}

static int* g_gram_status = nullptr;
void set_gram_status(int* status) { g_gram_status = status; }

template <typename T>
void launch_gram(const T* X, size_t ldx, int nx, const T* Y, size_t ldy, int ny, size_t n, double* out,
                 double* part, unsigned* counter, const int* gate, int mask, cudaStream_t st) {
  if (launch_tile<T>(0, X, ldx, nx, 0, 0, Y, ldy, ny, n, nullptr, nullptr, 0, out, part, counter, gate, mask,
                    g_gram_status, st))
    return;
  if (ny <= 1)
    gram_launch_ny<T, 1>(X, ldx, nx, Y, ldy, ny, n, out, part, counter, gate, mask, st);
  else if (ny <= 2)
    gram_launch_ny<T, 2>(X, ldx, nx, Y, ldy, ny, n, out, part, counter, gate, mask, st);
  else if (ny <= 4)
    gram_launch_ny<T, 4>(X, ldx, nx, Y, ldy, ny, n, out, part, counter, gate, mask, st);
  else
    gram_launch_ny<T, 8>(X, ldx, nx, Y, ldy, ny, n, out, part, counter, gate, mask, st);
}

// ===========================================================================
// Combination:  out_c = beta Y_c + sigma sum_r X_r C[r][c]   (site-wise)
// ===========================================================================
template <typename T, int NY>
__global__ void __launch_bounds__(kThreads) combine_kernel(const T* __restrict__ X, size_t ldx, int nx,
                                                           const int* nx_dev, const double* __restrict__ C, int ny,
                                                           const T* Y, size_t ldy, T beta, T sigma, T* out,
                                                           size_t ldo, const T* __restrict__ m, int N,
                                                           const int* gate, int mask, size_t ws) {
  X = wofs(X, ws);
  nx_dev = wofs(nx_dev, ws);
  C = wofs(C, ws);
  Y = wofs(Y, ws);
  out = wofs(out, ws);
  m = wofs(m, ws);
  gate = wofs(gate, ws);
  if (gate && (*gate & mask)) return;
  if (nx_dev) nx = min(*nx_dev, nx);
  __shared__ T Cs[MOTO_MAX_BASIS * NY];
  for (int idx = threadIdx.x; idx < nx * NY; idx += blockDim.x) {
    const int r = idx / NY, c = idx - r * NY;
    Cs[idx] = c < ny ? (T)((double)sigma * C[r * ny + c]) : (T)0;
  }
  __syncthreads();
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    T acc[NY][3];
#pragma unroll
    for (int c = 0; c < NY; ++c) {
      if (c < ny && beta != (T)0) {
        acc[c][0] = beta * Y[(size_t)c * ldy + i];
        acc[c][1] = beta * Y[(size_t)c * ldy + N + i];
        acc[c][2] = beta * Y[(size_t)c * ldy + 2 * (size_t)N + i];
      } else {
        acc[c][0] = acc[c][1] = acc[c][2] = (T)0;
      }
    }
    for (int r = 0; r < nx; ++r) {
      const T* xr = X + (size_t)r * ldx;
      const T x0 = __ldg(xr + i), x1 = __ldg(xr + N + i), x2 = __ldg(xr + 2 * (size_t)N + i);
#pragma unroll
      for (int c = 0; c < NY; ++c) {
        const T w = Cs[r * NY + c];
        acc[c][0] += x0 * w;
        acc[c][1] += x1 * w;
        acc[c][2] += x2 * w;
      }
    }
    T m0 = 0, m1 = 0, m2 = 0;
    if (m) {
      m0 = __ldg(m + i);
      m1 = __ldg(m + N + i);
      m2 = __ldg(m + 2 * (size_t)N + i);
    }
#pragma unroll
    for (int c = 0; c < NY; ++c) {
      if (c >= ny) continue;
      T a0 = acc[c][0], a1 = acc[c][1], a2 = acc[c][2];
      if (m) {
        const T p = m0 * a0 + m1 * a1 + m2 * a2;
        a0 -= p * m0;
        a1 -= p * m1;
        a2 -= p * m2;
      }
      out[(size_t)c * ldo + i] = a0;
      out[(size_t)c * ldo + N + i] = a1;
      out[(size_t)c * ldo + 2 * (size_t)N + i] = a2;
    }
  }
}

// Blocks of a site-wise kernel: in FP32 four sites a thread at least (a
// block's set-up and, where there is one, its reduction are then amortised on
// small lattices, e.g. the walkers of a batch); in FP64, whose arithmetic
// GB300 runs at a small fraction of the FP32 rate, one site a thread; at
// most eight blocks an SM.
static int stream_grid(size_t sites, size_t per_thread) {
  size_t b = (sites + per_thread * kThreads - 1) / (per_thread * kThreads);
  const size_t cap = (size_t)kSMs * 8;
  return (int)(b < cap ? (b > 0 ? b : 1) : cap);
}
template <typename T>
static int stream_grid(size_t sites) {
  return stream_grid(sites, sizeof(T) == 4 ? 4 : 1);
}

// Long FP32 combinations out = X C (nx >= 16 fields into ny <= 8, no Y term,
// no projection: the Ritz vectors of a block Lanczos basis).  Such a
// combination reads nx fields at once; a thread of combine_kernel keeps one
// field's loads in registers at a time, too few bytes in flight to cover the
// memory latency.  Here each thread owns quads of 4 consecutive elements of
// the flattened fields and copies its quad of 4 fields at a time into its
// own slots of a shared-memory ring with 16-byte cp.async (kCombRing groups,
// three in flight while one is used), so the bytes in flight do not cost
// registers.  Only the issuing thread reads its slots, so cp.async.wait_group
// is the only synchronisation.  Each output element is the same FMA chain
// over the fields in order as in combine_kernel, so the results are
// bit-identical.  (thread, group) steps run through one pipeline across the
// thread's quads.  Slots are field-major, thread-minor: a warp's 16-byte
// reads are conflict-free.
constexpr int kCombRing = 4;  // a power of two (slot = step & (kCombRing - 1))
static_assert((kCombRing & (kCombRing - 1)) == 0, "ring size");
constexpr int kCombThreads = 160;  // 40 KB of static shared memory a block

__device__ __forceinline__ void cp_async16_cg(void* smem_dst, const void* gsrc) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(smem_dst)),
               "l"(gsrc)
               : "memory");
}

template <int NY>
__global__ void __launch_bounds__(kCombThreads) combine_long_kernel(const float* __restrict__ X, size_t ldx, int nx,
                                                                    const int* nx_dev, const double* __restrict__ C,
                                                                    int ny, double sigma, float* out, size_t ldo,
                                                                    size_t n, const int* gate, int mask, size_t ws) {
  X = wofs(X, ws);
  nx_dev = wofs(nx_dev, ws);
  C = wofs(C, ws);
  out = wofs(out, ws);
  gate = wofs(gate, ws);
  if (gate && (*gate & mask)) return;
  if (nx_dev) nx = min(*nx_dev, nx);
  __shared__ __align__(16) float Cs[MOTO_MAX_BASIS * NY];  // row r: the NY weights of field r
  __shared__ __align__(16) float4 ring[kCombRing * 4 * kCombThreads];
  for (int idx = threadIdx.x; idx < nx * NY; idx += blockDim.x) {
    const int r = idx / NY, c = idx - r * NY;
    Cs[idx] = c < ny ? (float)(sigma * C[r * ny + c]) : 0.f;
  }
  __syncthreads();
  const size_t nq = (n + 3) / 4;
  const int G = nx > 4 ? (nx + 3) / 4 : 1;  // groups of 4 fields (nx = 0: the outputs are zero)
  const size_t tq = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  const size_t qstride = (size_t)gridDim.x * blockDim.x;
  // the thread's quads: tq, tq + qstride, ...; step s = (quad index i, group g)
  const size_t nmine = tq < nq ? (nq - 1 - tq) / qstride + 1 : 0;
  const size_t nsteps = nmine * (size_t)G;
  // the issue position runs kCombRing - 1 steps ahead of the consume
  // position; both walk (quad, group) with counters (no divisions)
  size_t iq = 0;  // issue: quad index and group
  int ig = 0;
  auto issue = [&](size_t step) {
    if (step < nsteps) {
      const size_t e0 = 4 * (tq + iq * qstride);
      const int slot = (int)(step & (kCombRing - 1));
#pragma unroll
      for (int f = 0; f < 4; ++f) {
        const int r = 4 * ig + f;
        if (r < nx) cp_async16_cg(&ring[(slot * 4 + f) * kCombThreads + threadIdx.x], X + (size_t)r * ldx + e0);
      }
      if (++ig == G) {
        ig = 0;
        ++iq;
      }
    }
    asm volatile("cp.async.commit_group;" ::: "memory");  // empty groups keep the count uniform
  };
#pragma unroll
  for (int k = 0; k < kCombRing - 1; ++k) issue(k);
  float acc[NY][4];
  size_t cq = 0;  // consume: quad index and group
  int g = 0;
  for (size_t step = 0; step < nsteps; ++step) {
    issue(step + kCombRing - 1);
    asm volatile("cp.async.wait_group %0;" ::"n"(kCombRing - 1) : "memory");
    if (g == 0) {
#pragma unroll
      for (int c = 0; c < NY; ++c) acc[c][0] = acc[c][1] = acc[c][2] = acc[c][3] = 0.f;
    }
    const int slot = (int)(step & (kCombRing - 1));
    // a field's NY weights in NY / 4 16-byte loads; full groups skip the
    // per-field test
    auto field = [&](int f) {
      const int r = 4 * g + f;
      const float4 x = ring[(slot * 4 + f) * kCombThreads + threadIdx.x];
      float w[NY];
#pragma unroll
      for (int c4 = 0; c4 < NY; c4 += 4) {
        const float4 w4 = *reinterpret_cast<const float4*>(&Cs[r * NY + c4]);
        w[c4] = w4.x;
        w[c4 + 1] = w4.y;
        w[c4 + 2] = w4.z;
        w[c4 + 3] = w4.w;
      }
#pragma unroll
      for (int c = 0; c < NY; ++c) {
        acc[c][0] = fmaf(x.x, w[c], acc[c][0]);
        acc[c][1] = fmaf(x.y, w[c], acc[c][1]);
        acc[c][2] = fmaf(x.z, w[c], acc[c][2]);
        acc[c][3] = fmaf(x.w, w[c], acc[c][3]);
      }
    };
    if (4 * g + 4 <= nx) {
#pragma unroll
      for (int f = 0; f < 4; ++f) field(f);
    } else {
      for (int f = 0; f < 4; ++f)
        if (4 * g + f < nx) field(f);
    }
    if (g == G - 1) {
      const size_t e0 = 4 * (tq + cq * qstride);
      if (e0 + 4 <= n) {
#pragma unroll
        for (int c = 0; c < NY; ++c)
          if (c < ny)
            *reinterpret_cast<float4*>(out + (size_t)c * ldo + e0) =
                make_float4(acc[c][0], acc[c][1], acc[c][2], acc[c][3]);
      } else {
#pragma unroll
        for (int c = 0; c < NY; ++c)
          if (c < ny)
            for (int u = 0; u < 4 && e0 + u < n; ++u) out[(size_t)c * ldo + e0 + u] = acc[c][u];
      }
    }
    if (++g == G) {
      g = 0;
      ++cq;
    }
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
}

template <typename T>
void launch_combine(const T* X, size_t ldx, int nx, const int* nx_dev, const double* C, int ny, const T* Y,
                    size_t ldy, double beta, double sigma, T* out, size_t ldo, const T* m, int N, const int* gate,
                    int mask, cudaStream_t st) {
  if constexpr (sizeof(T) == 4) {
    // long combinations: the cp.async ring (needs 16-byte aligned fields:
    // the quads of the last field may read up to 3 elements past 3N, inside
    // its padding, and those elements are never stored)
    const size_t n = 3 * (size_t)N;
    const bool al = ((uintptr_t)X % 16 == 0) && ((uintptr_t)out % 16 == 0) && ldx % 4 == 0 && ldo % 4 == 0 &&
                    ldx >= (n + 3) / 4 * 4 && walker_ws() % 16 == 0;
    static const bool ring_on = [] {
      const char* e = getenv("MOTO_COMBINE_RING");  // "0": always combine_kernel (a diagnostic switch)
      return !(e && strcmp(e, "0") == 0);
    }();
    if (ring_on && nx >= 16 && !Y && !m && beta == 0.0 && al) {
      // one wave of as many blocks an SM as fit (shared memory carveout at its
      // maximum; queried once per kernel)
      static int bps4 = 0, bps8 = 0;
      int& bps = ny <= 4 ? bps4 : bps8;
      if (bps == 0) {
        auto kern = ny <= 4 ? combine_long_kernel<4> : combine_long_kernel<8>;
        cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kern, kCombThreads, 0) != cudaSuccess || bps < 1) bps = 1;
      }
      const size_t nq = (n + 3) / 4;
      const size_t want = (nq + kCombThreads - 1) / kCombThreads;
      const int g = (int)std::min<size_t>(want, (size_t)kSMs * bps);
      if (ny <= 4)
        combine_long_kernel<4><<<wgrid(g), kCombThreads, 0, st>>>(X, ldx, nx, nx_dev, C, ny, sigma, out, ldo, n, gate,
                                                                mask, walker_ws());
      else
        combine_long_kernel<8><<<wgrid(g), kCombThreads, 0, st>>>(X, ldx, nx, nx_dev, C, ny, sigma, out, ldo, n, gate,
                                                                mask, walker_ws());
      return;
    }
  }
  const int g = stream_grid<T>(N);
  if (ny <= 1)
    combine_kernel<T, 1><<<wgrid(g), kThreads, 0, st>>>(X, ldx, nx, nx_dev, C, ny, Y, ldy, (T)beta, (T)sigma, out, ldo, m,
                                                 N, gate, mask, walker_ws());
  else if (ny <= 2)
    combine_kernel<T, 2><<<wgrid(g), kThreads, 0, st>>>(X, ldx, nx, nx_dev, C, ny, Y, ldy, (T)beta, (T)sigma, out, ldo, m,
                                                 N, gate, mask, walker_ws());
  else if (ny <= 4)
    combine_kernel<T, 4><<<wgrid(g), kThreads, 0, st>>>(X, ldx, nx, nx_dev, C, ny, Y, ldy, (T)beta, (T)sigma, out, ldo, m,
                                                 N, gate, mask, walker_ws());
  else
    combine_kernel<T, 8><<<wgrid(g), kThreads, 0, st>>>(X, ldx, nx, nx_dev, C, ny, Y, ldy, (T)beta, (T)sigma, out, ldo, m,
                                                 N, gate, mask, walker_ws());
}

namespace {
constexpr int kUpdSelf = 36;  // upper-triangle entries of an 8 x 8 Gram
}  // namespace

// ===========================================================================
// Cholesky QR applied twice without storing the first factor's product.
// t = X P (X: nx <= 8 fields, P = R1^{-1}, upper triangular) is formed per
// element in registers by t_c = fma(x_c, P[c][c], ... fma(x_0, P[0][c], 0))
// (rows past nx are zero), the same chain in both kernels below, so the Gram
// of the second pass and the final combination see bit-identical t (a packed
// fma.rn.f32x2 rounds each half exactly like fma.rn.f32):
//   chol2_gram: out = t^T t;
//   combine2:   Q = t P2 (P2 = R2^{-1}, upper triangular), projected on the
//               tangent planes of m when m is given.
// ===========================================================================
namespace {

// t = x P over the upper triangle: t[c] takes rows r = 0 .. c in order
template <typename T>
__device__ __forceinline__ void tri_mul(const T (&x)[8], const T* Ps, T (&t)[8]) {
#pragma unroll
  for (int c = 0; c < 8; ++c) t[c] = (T)0;
#pragma unroll
  for (int r = 0; r < 8; ++r)
#pragma unroll
    for (int c = r; c < 8; ++c) t[c] = fma(x[r], Ps[r * 8 + c], t[c]);
}
// P rows are re-read from shared memory (volatile loads: hoisting all 36
// entries into registers out of a streaming loop would cost more than the
// broadcast loads)
__device__ __forceinline__ void tri_mul2(const float2 (&x)[8], const float* Ps, float2 (&t)[8]) {
  const uint32_t pa = (uint32_t)__cvta_generic_to_shared(Ps);
#pragma unroll
  for (int c = 0; c < 8; ++c) t[c] = make_float2(0.f, 0.f);
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    float p[8];
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(p[0]), "=f"(p[1]), "=f"(p[2]), "=f"(p[3])
                 : "r"(pa + 32u * r));
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(p[4]), "=f"(p[5]), "=f"(p[6]), "=f"(p[7])
                 : "r"(pa + 32u * r + 16u));
#pragma unroll
    for (int c = r; c < 8; ++c) t[c] = ffma2v(x[r], make_float2(p[c], p[c]), t[c]);
  }
}

template <typename T>
__device__ __forceinline__ void stage_tri(T* Ps, const double* P, int nx) {
  for (int i = threadIdx.x; i < 64; i += blockDim.x) {
    const int r = i >> 3, c = i & 7;
    Ps[i] = (r < nx && c < nx && r <= c) ? (T)P[r * nx + c] : (T)0;
  }
}
}  // namespace

// FP32: a thread owns element pairs (8-byte loads, packed FMAs for t, the
// next pair loading while one is multiplied); FP64: single elements.
template <typename T>
__global__ void __launch_bounds__(kThreads, 2) chol2_gram_kernel(const T* __restrict__ X, size_t ldx, int nx,
                                                                 const double* __restrict__ P, size_t n,
                                                                 double* out, double* part, unsigned* counter,
                                                                 const int* gate, int mask, size_t ws) {
  X = wofs(X, ws);
  P = wofs(P, ws);
  out = wofs(out, ws);
  part = wofs(part, ws);
  counter = wofs(counter, ws);
  gate = wofs(gate, ws);
  if (gate && (*gate & mask)) return;
  __shared__ __align__(16) T Ps[64];
  __shared__ double red[kThreads / 32][kUpdSelf];
  stage_tri(Ps, P, nx);
  __syncthreads();
  T sacc[kUpdSelf];
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  if constexpr (sizeof(T) == 4) {
    // the next element pair is in flight while one is multiplied
#pragma unroll
    for (int q = 0; q < kUpdSelf; ++q) sacc[q] = 0.f;
    const size_t np = (n + 1) / 2;
    auto load = [&](size_t v, float2 (&x)[8]) {
      const size_t e = 2 * v;
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        x[r] = make_float2(0.f, 0.f);
        if (r < nx && v < np) {
          if (e + 2 <= n)
            x[r] = __ldg(reinterpret_cast<const float2*>(X + (size_t)r * ldx + e));
          else
            x[r].x = X[(size_t)r * ldx + e];
        }
      }
    };
    auto accumulate = [&](const float2 (&x)[8]) {
      float2 t[8];
      tri_mul2(x, Ps, t);
      int q = 0;
#pragma unroll
      for (int c1 = 0; c1 < 8; ++c1)
#pragma unroll
        for (int c2 = c1; c2 < 8; ++c2, ++q) sacc[q] = fmaf(t[c1].y, t[c2].y, fmaf(t[c1].x, t[c2].x, sacc[q]));
    };
    size_t v = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    float2 xa[8], xb[8];
    load(v, xa);
    load(v + stride, xb);
    for (; v < np; v += 2 * stride) {
      accumulate(xa);  // xb in flight
      load(v + 2 * stride, xa);
      if (v + stride >= np) break;
      accumulate(xb);  // xa in flight
      load(v + 3 * stride, xb);
    }
  } else {
#pragma unroll
    for (int q = 0; q < kUpdSelf; ++q) sacc[q] = (T)0;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += stride) {
      T x[8];
#pragma unroll
      for (int r = 0; r < 8; ++r) x[r] = r < nx ? __ldg(X + (size_t)r * ldx + e) : (T)0;
      T t[8];
      tri_mul<T>(x, Ps, t);
      int q = 0;
#pragma unroll
      for (int c1 = 0; c1 < 8; ++c1)
#pragma unroll
        for (int c2 = c1; c2 < 8; ++c2, ++q) sacc[q] = fma(t[c1], t[c2], sacc[q]);
    }
  }
  // warp sums in the field precision (a fixed butterfly over 32 partials of
  // a few tens of products each); block and grid sums in two-float
  // arithmetic for FP32 fields, FP64 for FP64 fields
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < kUpdSelf; ++q) {
    T v = sacc[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    sacc[q] = v;
  }
  // FP32: block and grid sums in two-float arithmetic (F2, 8 bytes like the
  // FP64 partials of FP64 fields)
  typedef typename std::conditional<sizeof(T) == 4, F2, double>::type RT;
  RT(*rred)[kUpdSelf] = reinterpret_cast<RT(*)[kUpdSelf]>(red);
#pragma unroll
  for (int q = 0; q < kUpdSelf; ++q)
    if (lane == (q & 31)) {
      if constexpr (sizeof(T) == 4)
        rred[wid][q] = f2_of(sacc[q]);
      else
        rred[wid][q] = sacc[q];
    }
  __syncthreads();
  if (threadIdx.x < kUpdSelf) {
    RT acc = rred[0][threadIdx.x];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) acc = radd(acc, rred[w][threadIdx.x]);
    reinterpret_cast<RT*>(part)[(size_t)blockIdx.x * kUpdSelf + threadIdx.x] = acc;
  }
  if (!grid_last_block(counter)) return;
  __syncthreads();
  __shared__ double tot[kUpdSelf];
  if constexpr (sizeof(T) == 4)
    grid_sum_f2(reinterpret_cast<const F2*>(part), gridDim.x, kUpdSelf, tot, reinterpret_cast<F2*>(red));
  else
    grid_sum_entries(part, gridDim.x, kUpdSelf, tot);
  __syncthreads();
  if (threadIdx.x < kUpdSelf) {
    const double acc = tot[threadIdx.x];
    int c1 = 0, rem = threadIdx.x;
    while (rem >= 8 - c1) {
      rem -= 8 - c1;
      ++c1;
    }
    const int c2 = c1 + rem;
    if (c2 < nx) {
      out[c1 * nx + c2] = acc;
      out[c2 * nx + c1] = acc;
    }
  }
  if (threadIdx.x == 0) *counter = 0u;
}

// Site-based: a thread loads all its fields first (24 per site), then forms
// t and Q per component.  PAIR (FP32, N even): two adjacent sites per thread
// with 8-byte loads and packed FMAs.
template <typename T, bool PAIR>
__global__ void __launch_bounds__(kThreads) combine2_kernel(const T* __restrict__ X, size_t ldx, int nx,
                                                            const double* __restrict__ P1,
                                                            const double* __restrict__ P2, T* out, size_t ldo,
                                                            const T* __restrict__ m, int N, const int* gate,
                                                            int mask, size_t ws) {
  X = wofs(X, ws);
  P1 = wofs(P1, ws);
  P2 = wofs(P2, ws);
  out = wofs(out, ws);
  m = wofs(m, ws);
  gate = wofs(gate, ws);
  if (gate && (*gate & mask)) return;
  __shared__ __align__(16) T P1s[64], P2s[64];
  stage_tri(P1s, P1, nx);
  stage_tri(P2s, P2, nx);
  __syncthreads();
  if constexpr (PAIR) {
    const int np = N / 2;
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < np; v += gridDim.x * blockDim.x) {
      const size_t i = 2 * (size_t)v;
      float2 x[3][8];
#pragma unroll
      for (int comp = 0; comp < 3; ++comp)
#pragma unroll
        for (int r = 0; r < 8; ++r)
          x[comp][r] = r < nx ? __ldg(reinterpret_cast<const float2*>(X + (size_t)r * ldx + (size_t)comp * N + i))
                              : make_float2(0.f, 0.f);
      float2 mm[3];
#pragma unroll
      for (int comp = 0; comp < 3; ++comp)
        mm[comp] = m ? __ldg(reinterpret_cast<const float2*>(m + (size_t)comp * N + i)) : make_float2(0.f, 0.f);
      float2 q[3][8];
#pragma unroll
      for (int comp = 0; comp < 3; ++comp) {
        float2 t[8];
        tri_mul2(x[comp], P1s, t);
        tri_mul2(t, P2s, q[comp]);
      }
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        if (c >= nx) continue;
        float2 a0 = q[0][c], a1 = q[1][c], a2 = q[2][c];
        if (m) {
          const float2 p = make_float2(mm[0].x * a0.x + mm[1].x * a1.x + mm[2].x * a2.x,
                                       mm[0].y * a0.y + mm[1].y * a1.y + mm[2].y * a2.y);
          a0.x -= p.x * mm[0].x;
          a0.y -= p.y * mm[0].y;
          a1.x -= p.x * mm[1].x;
          a1.y -= p.y * mm[1].y;
          a2.x -= p.x * mm[2].x;
          a2.y -= p.y * mm[2].y;
        }
        *reinterpret_cast<float2*>(out + (size_t)c * ldo + i) = a0;
        *reinterpret_cast<float2*>(out + (size_t)c * ldo + N + i) = a1;
        *reinterpret_cast<float2*>(out + (size_t)c * ldo + 2 * (size_t)N + i) = a2;
      }
    }
  } else {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
      T x[3][8];
#pragma unroll
      for (int comp = 0; comp < 3; ++comp)
#pragma unroll
        for (int r = 0; r < 8; ++r) x[comp][r] = r < nx ? __ldg(X + (size_t)r * ldx + (size_t)comp * N + i) : (T)0;
      T m0 = 0, m1 = 0, m2 = 0;
      if (m) {
        m0 = __ldg(m + i);
        m1 = __ldg(m + N + i);
        m2 = __ldg(m + 2 * (size_t)N + i);
      }
      T q[3][8];
#pragma unroll
      for (int comp = 0; comp < 3; ++comp) {
        T t[8];
        tri_mul<T>(x[comp], P1s, t);
        tri_mul<T>(t, P2s, q[comp]);
      }
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        if (c >= nx) continue;
        T a0 = q[0][c], a1 = q[1][c], a2 = q[2][c];
        if (m) {
          const T p = m0 * a0 + m1 * a1 + m2 * a2;
          a0 -= p * m0;
          a1 -= p * m1;
          a2 -= p * m2;
        }
        out[(size_t)c * ldo + i] = a0;
        out[(size_t)c * ldo + N + i] = a1;
        out[(size_t)c * ldo + 2 * (size_t)N + i] = a2;
      }
    }
  }
}

template <typename T>
bool launch_chol2(const T* X, size_t ldx, int nx, const double* P1, const double* P2, T* Q, size_t ldq, const T* m,
                  int N, double* S2, double* part, unsigned* counter, const int* gate, int mask, bool gram,
                  cudaStream_t st) {
  if (nx < 1 || nx > 8) return false;
  if (gram) {
    if (((uintptr_t)X % (2 * sizeof(T))) || (ldx % 2)) return false;
    const size_t n = 3 * (size_t)N;
    // at least 64 KB of FP32 fields a block (small fields: fewer blocks);
    // FP64 arithmetic is slow on GB300, so FP64 blocks take 8 KB
    const size_t per_block = sizeof(T) == 4 ? 65536 : 8192;
    size_t g = (nx * n * sizeof(T) + per_block - 1) / per_block;
    const size_t cap = (size_t)kSMs * 2;  // one wave at two blocks per SM
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    chol2_gram_kernel<T><<<wgrid((int)g), kThreads, 0, st>>>(X, ldx, nx, P1, n, S2, part, counter, gate, mask, walker_ws());
  } else {
    const bool pair = sizeof(T) == 4 && N % 2 == 0 && ldx % 2 == 0 && ldq % 2 == 0 && (uintptr_t)X % 8 == 0 &&
                      (uintptr_t)Q % 8 == 0 && (!m || (uintptr_t)m % 8 == 0);
    if constexpr (sizeof(T) == 4) {
      if (pair) {
        combine2_kernel<T, true><<<wgrid(stream_grid<T>(N / 2)), kThreads, 0, st>>>(X, ldx, nx, P1, P2, Q, ldq, m, N, gate,
                                                                          mask, walker_ws());
        return true;
      }
    }
    combine2_kernel<T, false><<<wgrid(stream_grid<T>(N)), kThreads, 0, st>>>(X, ldx, nx, P1, P2, Q, ldq, m, N, gate, mask, walker_ws());
  }
  return true;
}

// ===========================================================================
// projection and Ritz finishing
// ===========================================================================
template <typename T>
__global__ void project_kernel(const T* __restrict__ m, const T* in, size_t ldi, T* out, size_t ldo, int nvec, int N,
                               const int* gate, int mask, size_t ws) {
  m = wofs(m, ws);
  in = wofs(in, ws);
  out = wofs(out, ws);
  gate = wofs(gate, ws);
  if (gate && (*gate & mask)) return;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    const T m0 = m[i], m1 = m[N + i], m2 = m[2 * (size_t)N + i];
    for (int j = 0; j < nvec; ++j) {
      const T* a = in + (size_t)j * ldi;
      T* b = out + (size_t)j * ldo;
      const T a0 = a[i], a1 = a[N + i], a2 = a[2 * (size_t)N + i];
      const T p = m0 * a0 + m1 * a1 + m2 * a2;
      b[i] = a0 - p * m0;
      b[N + i] = a1 - p * m1;
      b[2 * (size_t)N + i] = a2 - p * m2;
    }
  }
}

template <typename T>
void launch_project(const T* m, const T* in, size_t ldi, T* out, size_t ldo, int nvec, int N, const int* gate,
                    int mask, cudaStream_t st) {
  project_kernel<T><<<wgrid(stream_grid<T>(N)), kThreads, 0, st>>>(m, in, ldi, out, ldo, nvec, N, gate, mask, walker_ws());
}

// argmax with ties to the lowest index: (abs, idx) pairs
__device__ __forceinline__ void amax_merge(double& a, double& ai, double& av, double b, double bi, double bv) {
  if (b > a || (b == a && bi < ai)) {
    a = b;
    ai = bi;
    av = bv;
  }
}

// pass 1: partials per block and vector of P(V_c) (computed, not stored):
// |P V_c|^2, max |entry|, its flat index, its signed value.  Per-thread shares are kept in the field
// precision (a thread sees ~160 entries; comparisons of |entries| are exact in
// either precision) and promoted to FP64 for the cross-thread reductions.
template <typename A>
__device__ __forceinline__ void amax_merge_t(A& a, int& ai, A& av, A b, int bi, A bv) {
  if (b > a || (b == a && bi < ai)) {
    a = b;
    ai = bi;
    av = bv;
  }
}

template <typename T>
__global__ void __launch_bounds__(kThreads) finish1_kernel(const T* __restrict__ m, const T* __restrict__ V,
                                                           size_t ldv, int k, int N, double* part, unsigned* counter,
                                                           double* scal, const int* gate, int mask, size_t ws) {
  m = wofs(m, ws);
  V = wofs(V, ws);
  part = wofs(part, ws);
  counter = wofs(counter, ws);
  scal = wofs(scal, ws);
  gate = wofs(gate, ws);
  if (gate && (*gate & mask)) return;
  T nrm_t[MOTO_MAX_K], amx_t[MOTO_MAX_K], aval_t[MOTO_MAX_K];
  int aidx_t[MOTO_MAX_K];
#pragma unroll
  for (int c = 0; c < MOTO_MAX_K; ++c) {
    nrm_t[c] = (T)0;
    amx_t[c] = (T)-1;
    aidx_t[c] = 0x7fffffff;
    aval_t[c] = (T)0;
  }
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    const T m0 = m[i], m1 = m[N + i], m2 = m[2 * (size_t)N + i];
    // every load of the site first (predicated, not a loop exit), so that
    // they are all in flight together
    T va[MOTO_MAX_K][3];
#pragma unroll
    for (int c = 0; c < MOTO_MAX_K; ++c) {
      const T* v = V + (size_t)c * ldv;
      va[c][0] = c < k ? __ldg(v + i) : (T)0;
      va[c][1] = c < k ? __ldg(v + N + i) : (T)0;
      va[c][2] = c < k ? __ldg(v + 2 * (size_t)N + i) : (T)0;
    }
#pragma unroll
    for (int c = 0; c < MOTO_MAX_K; ++c) {
      if (c >= k) break;
      T a0 = va[c][0], a1 = va[c][1], a2 = va[c][2];
      const T p = m0 * a0 + m1 * a1 + m2 * a2;
      a0 -= p * m0;
      a1 -= p * m1;
      a2 -= p * m2;
      nrm_t[c] += a0 * a0 + a1 * a1 + a2 * a2;
      amax_merge_t<T>(amx_t[c], aidx_t[c], aval_t[c], fabs(a0), i, a0);
      amax_merge_t<T>(amx_t[c], aidx_t[c], aval_t[c], fabs(a1), N + i, a1);
      amax_merge_t<T>(amx_t[c], aidx_t[c], aval_t[c], fabs(a2), 2 * N + i, a2);
    }
  }
  __shared__ double sh[MOTO_MAX_K][kThreads / 32][4];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int c = 0; c < MOTO_MAX_K; ++c) {
    if (c >= k) break;
    // warp level in the field precision: the sum by a fixed butterfly, the
    // largest entry (ties: lowest index) in any order
    T sT = nrm_t[c], aT = amx_t[c], avT = aval_t[c];
    int aiT = aidx_t[c];
    for (int o = 16; o > 0; o >>= 1) {
      sT += __shfl_xor_sync(0xffffffffu, sT, o);
      const T b = __shfl_xor_sync(0xffffffffu, aT, o);
      const int bi = __shfl_xor_sync(0xffffffffu, aiT, o);
      const T bv = __shfl_xor_sync(0xffffffffu, avT, o);
      amax_merge_t<T>(aT, aiT, avT, b, bi, bv);
    }
    if (lane == 0) {
      sh[c][wid][0] = (double)sT;
      sh[c][wid][1] = (double)aT;
      sh[c][wid][2] = aiT == 0x7fffffff ? 1e300 : (double)aiT;
      sh[c][wid][3] = (double)avT;
    }
  }
  __syncthreads();
  // thread c merges vector c over the warps in order
  if (threadIdx.x < k) {
    const int c = threadIdx.x;
    double S = 0.0, A = -1.0, AI = 1e300, AV = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      S += sh[c][w][0];
      amax_merge(A, AI, AV, sh[c][w][1], sh[c][w][2], sh[c][w][3]);
    }
    double* p = part + ((size_t)blockIdx.x * MOTO_MAX_K + c) * 4;
    p[0] = S;
    p[1] = A;
    p[2] = AI;
    p[3] = AV;
  }
  if (!grid_last_block(counter)) return;
  // warp c reduces vector c: lane l takes blocks l, l + 32, ... in order (four
  // blocks' loads in flight at a time); the sums meet in a fixed shuffle tree,
  // the largest entry in any order (ties go to the lowest index, a total order)
  if (wid < k) {
    const int c = wid;
    double S = 0.0, A = -1.0, AI = 1e300, AV = 0.0;
    int b = lane;
    for (; b + 96 < (int)gridDim.x; b += 128) {
      double4 q[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const double* p = part + ((size_t)(b + 32 * u) * MOTO_MAX_K + c) * 4;
        q[u] = make_double4(__ldcg(p), __ldcg(p + 1), __ldcg(p + 2), __ldcg(p + 3));
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        S += q[u].x;
        amax_merge(A, AI, AV, q[u].y, q[u].z, q[u].w);
      }
    }
    for (; b < (int)gridDim.x; b += 32) {
      const double* p = part + ((size_t)b * MOTO_MAX_K + c) * 4;
      S += __ldcg(p);
      amax_merge(A, AI, AV, __ldcg(p + 1), __ldcg(p + 2), __ldcg(p + 3));
    }
    S = warp_sum(S);
    for (int o = 16; o > 0; o >>= 1) {
      const double b = __shfl_xor_sync(0xffffffffu, A, o);
      const double bi = __shfl_xor_sync(0xffffffffu, AI, o);
      const double bv = __shfl_xor_sync(0xffffffffu, AV, o);
      amax_merge(A, AI, AV, b, bi, bv);
    }
    if (lane == 0) {
      const double nrm_ = sqrt(S);
      scal[c] = (nrm_ > 0.0 ? 1.0 / nrm_ : 0.0) * (AV < 0.0 ? -1.0 : 1.0);
    }
  }
  if (threadIdx.x == 0) *counter = 0u;
}

// pass 2: V_c <- scal_c P(V_c) (the projection recomputed exactly as in pass 1)
template <typename T>
__global__ void __launch_bounds__(kThreads) finish2_kernel(const T* __restrict__ m, T* V, size_t ldv, int k, int N,
                                                           const double* scal, const int* gate, int mask, size_t ws) {
  m = wofs(m, ws);
  V = wofs(V, ws);
  scal = wofs(scal, ws);
  gate = wofs(gate, ws);
  if (gate && (*gate & mask)) return;
  __shared__ T sc[MOTO_MAX_K];
  if (threadIdx.x < MOTO_MAX_K) sc[threadIdx.x] = threadIdx.x < k ? (T)scal[threadIdx.x] : (T)0;
  __syncthreads();
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    const T m0 = m[i], m1 = m[N + i], m2 = m[2 * (size_t)N + i];
#pragma unroll
    for (int c = 0; c < MOTO_MAX_K; ++c) {
      if (c >= k) break;
      T* v = V + (size_t)c * ldv;
      T a0 = v[i], a1 = v[N + i], a2 = v[2 * (size_t)N + i];
      const T p = m0 * a0 + m1 * a1 + m2 * a2;
      a0 -= p * m0;
      a1 -= p * m1;
      a2 -= p * m2;
      const T f = sc[c];
      v[i] = a0 * f;
      v[N + i] = a1 * f;
      v[2 * (size_t)N + i] = a2 * f;
    }
  }
}

template <typename T>
void launch_finish(const T* m, T* V, size_t ldv, int k, int N, double* part, unsigned* counter, double* scal,
                   const int* gate, int mask, cudaStream_t st) {
  const int g = stream_grid<T>(N);
  // two blocks an SM for the reducing pass: fewer partials for its last block
  const int g1 = g < 2 * kSMs ? g : 2 * kSMs;
  finish1_kernel<T><<<wgrid(g1), kThreads, 0, st>>>(m, V, ldv, k, N, part, counter, scal, gate, mask, walker_ws());
  finish2_kernel<T><<<wgrid(g), kThreads, 0, st>>>(m, V, ldv, k, N, scal, gate, mask, walker_ws());
}

// ===========================================================================
// small dense FP64 steps (one block)
// ===========================================================================
__global__ void lanczos_coeffs_kernel(const double* A, int b, int j, double* T, int ldT, double* C3, DevState* st, size_t ws) {
  A = wofs(A, ws);
  T = wofs(T, ws);
  C3 = wofs(C3, ws);
  st = wofs(st, ws);
  if (st->gate & (kGateKrylov | kGateDone)) return;
  // one thread per (r, c) of a b x b block
  const int r = threadIdx.x >> 3, c = threadIdx.x & 7;
  if (r >= b || c >= b) return;
  // T(j, j) = sym(A)
  const double a = 0.5 * (A[r * b + c] + A[c * b + r]);
  T[(size_t)(j * b + r) * ldT + j * b + c] = a;
  // C3 rows: [R_j^T (for Q_{j-1}); T(j, j) (for Q_j)],   R_j = T(j, j-1)
  const int row0 = j > 0 ? b : 0;
  if (j > 0) C3[r * b + c] = T[(size_t)(j * b + c) * ldT + (j - 1) * b + r];
  C3[(row0 + r) * b + c] = a;
}

void launch_lanczos_coeffs(const double* A, int b, int j, double* T, int ldT, double* C3, DevState* st,
                           cudaStream_t s) {
  lanczos_coeffs_kernel<<<wgrid(1), 64, 0, s>>>(A, b, j, T, ldT, C3, st, walker_ws());
}

__global__ void arnoldi_diag_kernel(const double* G1, int b, int jr, int j, double* T, int ldT, DevState* st) {
  if (st->gate & (kGateKrylov | kGateDone)) return;
  const int r = threadIdx.x / b, c = threadIdx.x % b;
  if (r >= b) return;
  const double a = G1[(size_t)(jr * b + r) * b + c], at = G1[(size_t)(jr * b + c) * b + r];
  T[(size_t)(j * b + r) * ldT + j * b + c] = 0.5 * (a + at);
}

void launch_arnoldi_diag(const double* G1, int b, int jr, int j, double* T, int ldT, DevState* st, cudaStream_t s) {
  arnoldi_diag_kernel<<<1, 64, 0, s>>>(G1, b, jr, j, T, ldT, st);
}

// Cholesky QR factor of the b x b Gram G.  Pass 1 (second == 0) also updates
// the |T| estimate with block row j (sum of |A| and |R_j| row entries plus the
// largest new diagonal) and tests for breakdown (smallest diagonal of the
// factor <= rel_tol * |T|).  Pass 2 composes R and stores it in T.
// 64 threads, thread t = (r, c) = (t / 8, t % 8).  A dependent FP64 operation
// costs GB300 on the order of a hundred cycles, so the kernel is built around
// short chains: every global operand is read in one round trip (before the
// gate test), the right-looking factorisation has one reciprocal square root
// per pivot, the triangular inverse (one column per thread, fully unrolled)
// adds the newest term of each sum last, and the minima, maxima and the final
// product are trees or split sums.
__global__ void __launch_bounds__(64) cholqr_kernel(const double* G, int b, int second, int j, double* Rinv,
                                                    double* Racc, double* T, int ldT, DevState* st, double rel_tol,
                                                    int skip, size_t ws) {
  G = wofs(G, ws);
  Rinv = wofs(Rinv, ws);
  Racc = wofs(Racc, ws);
  T = wofs(T, ws);
  st = wofs(st, ws);
  // j >= 0: block Lanczos step j; j == -1: start block; j == -2: LOBPCG block
  __shared__ double Ls[MOTO_MAX_K][MOTO_MAX_K], Gs[MOTO_MAX_K][MOTO_MAX_K], Us[MOTO_MAX_K][MOTO_MAX_K];
  __shared__ double Ra[MOTO_MAX_K][MOTO_MAX_K];
  __shared__ double dinv[MOTO_MAX_K], rsum[MOTO_MAX_K], gdiag[MOTO_MAX_K];
  __shared__ int bad, verdict;  // verdict: 0 go on, 1 stop (gate set), 2 LOBPCG column scaling
  const int t = threadIdx.x, r = t >> 3, c = t & 7;
  const bool in = r < b && c < b;
  const bool rows_t = !second && j >= 0;
  // all loads in flight together (the buffers are valid whatever the gate says)
  double g_rc = 0.0, g_cr = 0.0, ta = 0.0, ra = 0.0;
  if (in) {
    g_rc = G[r * b + c];
    g_cr = G[c * b + r];
    if (rows_t)  // |T| row sums of block row j: T(j, j) and R_j = T(j, j - 1)
      ta = fabs(T[(size_t)(j * b + r) * ldT + j * b + c]) +
           (j > 0 ? fabs(T[(size_t)(j * b + r) * ldT + (j - 1) * b + c]) : 0.0);
    if (second) ra = Racc[r * b + c];
  }
  const double tnorm0 = st->tnorm;
  if (st->gate & (kGateKrylov | kGateDone | skip)) return;
  if (t == 0) bad = 0;
  if (in) {
    Gs[r][c] = 0.5 * (g_rc + g_cr);
    Ls[r][c] = 0.0;
    if (r == c) gdiag[r] = g_rc;
    Ra[r][c] = ra;
  }
  // row sums of |T| by shuffles within the row's eight lanes (c order fixed)
  {
    double a = ta;
    a += __shfl_down_sync(0xffffffffu, a, 4, 8);
    a += __shfl_down_sync(0xffffffffu, a, 2, 8);
    a += __shfl_down_sync(0xffffffffu, a, 1, 8);
    if (c == 0 && r < b) rsum[r] = a;
  }
  __syncthreads();
  for (int k = 0; k < b; ++k) {
    if (t == 0) {
      double d = Gs[k][k];
      if (!(d > 0.0)) {
        bad = 1;
        d = 1.0;
      }
      // one reciprocal square root on the dependent chain instead of a
      // square root and a division
      const double di = rsqrt(d);
      Ls[k][k] = d * di;
      dinv[k] = di;
    }
    __syncthreads();
    if (c == k && r > k && r < b) Ls[r][k] = Gs[r][k] * dinv[k];
    __syncthreads();
    if (r < b && c > k && c <= r) Gs[r][c] -= Ls[r][k] * Ls[c][k];
    __syncthreads();
  }
  if (t < 32) {
    // warp 0: smallest and largest diagonal, largest |T| row sum and the
    // near-dependent columns (L_kk^2 <= 1e-12 G_kk), trees over lanes 0..7
    const bool on = t < b;
    const double lkk = on ? Ls[t][t] : 0.0;
    double dmin = on ? lkk : 1e300, dmax = on ? lkk : 0.0, rs = (on && rows_t) ? rsum[t] : 0.0;
    int dep = (on && lkk * lkk <= 1e-12 * fmax(gdiag[t], 0.0)) ? 1 : 0;
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) {
      dmin = fmin(dmin, __shfl_xor_sync(0xffffffffu, dmin, o));
      dmax = fmax(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
      rs = fmax(rs, __shfl_xor_sync(0xffffffffu, rs, o));
      dep |= __shfl_xor_sync(0xffffffffu, dep, o);
    }
    if (t == 0) {
      int v = 0;
      if (rows_t) {
        const double tn = fmax(tnorm0, rs + dmax);
        st->tnorm = tn;
        if (bad || dmin <= rel_tol * tn) {
          st->gate |= kGateKrylov;
          v = 1;
        }
      } else if (bad || dep) {
        if (j == -2) {
          v = 2;
        } else {
          st->gate |= kGateKrylov;
          if (j < 0) st->status |= kStatusBreakdown;
          v = 1;
        }
      }
      verdict = v;
    }
  }
  __syncthreads();
  if (verdict == 1) return;
  if (verdict == 2) {
    // LOBPCG residual block: fall back to column scaling; the SVQB step of
    // the Rayleigh-Ritz drops what stays dependent
    if (in) Rinv[r * b + c] = (r == c) ? (gdiag[r] > 0.0 ? 1.0 / sqrt(gdiag[r]) : 1.0) : 0.0;
    return;
  }
  // Rinv = (L^T)^{-1}, upper triangular: column cc solves L^T x = e_cc by
  // back substitution, each sum taken oldest term first so that only its last
  // term waits on the entry just computed
  if (t < b) {
    const int cc = t;
    double u[MOTO_MAX_K];
#pragma unroll
    for (int rr = MOTO_MAX_K - 1; rr >= 0; --rr) {
      double a = (rr == cc) ? 1.0 : 0.0;
#pragma unroll
      for (int q = MOTO_MAX_K - 1; q > rr; --q)
        if (q <= cc) a -= Ls[q][rr] * u[q];
      u[rr] = (rr <= cc && rr < b) ? a * dinv[rr] : 0.0;
    }
#pragma unroll
    for (int rr = 0; rr < MOTO_MAX_K; ++rr)
      if (rr < b) Us[rr][cc] = u[rr];
  }
  __syncthreads();
  if (in) Rinv[r * b + c] = Us[r][c];
  if (!second) {
    if (in) Racc[r * b + c] = Ls[c][r];  // R1 = L^T
    return;
  }
  // R = L2^T R1 (two interleaved partial sums; R1 was read before it is
  // overwritten)
  double R0 = 0.0, R1 = 0.0;
  if (in) {
#pragma unroll
    for (int q = 0; q < MOTO_MAX_K; q += 2) {
      if (q < b) R0 += Ls[q][r] * Ra[q][c];
      if (q + 1 < b) R1 += Ls[q + 1][r] * Ra[q + 1][c];
    }
  }
  const double Rv = R0 + R1;
  if (in) {
    Racc[r * b + c] = Rv;
    if (j >= 0) {
      T[(size_t)((j + 1) * b + r) * ldT + j * b + c] = Rv;
      T[(size_t)(j * b + c) * ldT + (j + 1) * b + r] = Rv;
    }
  }
  if (t == 0 && j >= -1) {
    st->steps += 1;
    st->nT = st->steps * b;
  }
}

void launch_cholqr(const double* G, int b, int second, int j, double* Rinv, double* Racc, double* T, int ldT,
                   DevState* st, double rel_tol, cudaStream_t s, int skip) {
  cholqr_kernel<<<wgrid(1), 64, 0, s>>>(G, b, second, j, Rinv, Racc, T, ldT, st, rel_tol, skip, walker_ws());
}

// Cyclic Jacobi with round-robin (parallel) ordering on an n x n symmetric
// matrix A (row stride ld >= n + (n & 1)) held in shared memory; V receives the
// eigenvectors (columns), diag(A) the eigenvalues.  Whole block participates.
// scratch: cs, sn (n/2 + 1 doubles each), pp, qq (n/2 + 1 ints), red (>= 16 doubles).
__device__ void block_jacobi(double* A, double* V, int n, int ld, double* cs, double* sn, int* pp, int* qq,
                             double* red) {
  const int n2 = n + (n & 1);
  for (int idx = threadIdx.x; idx < n2 * n2; idx += blockDim.x) {
    const int r = idx / n2, c = idx - r * n2;
    if (r >= n || c >= n) A[r * ld + c] = 0.0;
    V[r * ld + c] = (r == c) ? 1.0 : 0.0;
  }
  __syncthreads();
  const int half = n2 / 2;
  __shared__ bool stop;
  for (int sweep = 0; sweep < 40; ++sweep) {
    double off = 0.0, dia = 0.0;
    for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
      const int r = idx / n, c = idx - r * n;
      const double a = A[r * ld + c];
      if (r == c)
        dia += a * a;
      else
        off += a * a;
    }
    double v2[2] = {off, dia};
    block_sum<2>(v2, red);
    if (threadIdx.x == 0) stop = !(v2[0] > 1e-30 * v2[1]) || n <= 1;
    __syncthreads();
    if (stop) break;
    for (int round = 0; round < n2 - 1; ++round) {
      for (int t = threadIdx.x; t < half; t += blockDim.x) {
        const int a0 = t, b0 = n2 - 1 - t;
        int p = a0 == 0 ? 0 : ((a0 - 1 + round) % (n2 - 1)) + 1;
        int q = b0 == 0 ? 0 : ((b0 - 1 + round) % (n2 - 1)) + 1;
        if (p > q) {
          const int x = p;
          p = q;
          q = x;
        }
        pp[t] = p;
        qq[t] = q;
        double c = 1.0, s = 0.0;
        const double apq = A[p * ld + q];
        if (q < n && fabs(apq) > 1e-300) {
          const double tau = (A[q * ld + q] - A[p * ld + p]) / (2.0 * apq);
          const double tt = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
          c = 1.0 / sqrt(1.0 + tt * tt);
          s = tt * c;
        }
        cs[t] = c;
        sn[t] = s;
      }
      __syncthreads();
      for (int idx = threadIdx.x; idx < half * n2; idx += blockDim.x) {
        const int t = idx / n2, col = idx - t * n2;
        const int p = pp[t], q = qq[t];
        const double c = cs[t], s = sn[t];
        const double ap = A[p * ld + col], aq = A[q * ld + col];
        A[p * ld + col] = c * ap - s * aq;
        A[q * ld + col] = s * ap + c * aq;
      }
      __syncthreads();
      for (int idx = threadIdx.x; idx < half * n2; idx += blockDim.x) {
        const int t = idx / n2, row = idx - t * n2;
        const int p = pp[t], q = qq[t];
        const double c = cs[t], s = sn[t];
        const double ap = A[row * ld + p], aq = A[row * ld + q];
        A[row * ld + p] = c * ap - s * aq;
        A[row * ld + q] = s * ap + c * aq;
        const double vp = V[row * ld + p], vq = V[row * ld + q];
        V[row * ld + p] = c * vp - s * vq;
        V[row * ld + q] = s * vp + c * vq;
      }
      __syncthreads();
    }
  }
}

// rank of diag entry i among the first n (ascending, ties by index)
__device__ __forceinline__ int diag_rank(const double* A, int ld, int n, int i) {
  const double li = A[i * ld + i];
  int rank = 0;
  for (int j = 0; j < n; ++j) {
    const double lj = A[j * ld + j];
    rank += (lj < li) || (lj == li && j < i);
  }
  return rank;
}

constexpr int kEigMax = MOTO_MAX_BASIS;

__global__ void __launch_bounds__(256) small_eig_kernel(const double* Tm, int ldT, double* theta, double* Y, int k,
                                                        DevState* st) {
  if (st->gate & kGateDone) return;
  extern __shared__ double sm[];
  const int n = st->nT;
  const int n2 = n + (n & 1);
  const int ld = n2 + 1;
  double* A = sm;
  double* V = A + (size_t)n2 * ld;
  double* cs = V + (size_t)n2 * ld;
  double* sn = cs + n2 / 2 + 1;
  double* red = sn + n2 / 2 + 1;
  int* pp = reinterpret_cast<int*>(red + 32);
  int* qq = pp + n2 / 2 + 1;
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    const int r = idx / n, c = idx - r * n;
    A[r * ld + c] = 0.5 * (Tm[(size_t)r * ldT + c] + Tm[(size_t)c * ldT + r]);
  }
  __syncthreads();
  block_jacobi(A, V, n, ld, cs, sn, pp, qq, red);
  for (int i = threadIdx.x; i < MOTO_MAX_BASIS; i += blockDim.x) theta[i] = 1.0 / 0.0;
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const int rank = diag_rank(A, ld, n, i);
    theta[rank] = A[i * ld + i];
    if (rank < k)
      for (int r = 0; r < n; ++r) Y[(size_t)r * k + rank] = V[r * ld + i];
  }
}

void launch_small_eig(const double* T, int ldT, double* theta, double* Y, int k, DevState* st, cudaStream_t s) {
  const int n2 = kEigMax;
  const size_t smem = (size_t)2 * n2 * (n2 + 1) * sizeof(double) + (n2 + 2) * sizeof(double) +
                      32 * sizeof(double) + (n2 + 2) * sizeof(int);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(small_eig_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    attr = true;
  }
  small_eig_kernel<<<1, 256, smem, s>>>(T, ldT, theta, Y, k, st);
}

// LOBPCG Rayleigh-Ritz on the trial subspace S = [X, W, P] (nS = nb*k columns):
// G = S^T S and M = S^T A S arrive as nb column blocks (nS x k each).  SVQB:
// D = diag(G)^-1/2, eig(D G D) = U w U^T, keep w > drop*max(w),
// Z = D U_keep w_keep^-1/2; eig(Z^T M Z) = U2 w2 U2^T ascending;
// Cx = Z U2[:, :k]; Cp = Cx with the X rows zeroed; theta = w2[:k];
// hnorm = max(hnorm, max |w2|).
__global__ void __launch_bounds__(256) lob_rr_kernel(const double* Gb, const double* Mb, int k, int nb,
                                                     double drop, double* Cx, double* Cp, double* theta,
                                                     DevState* st) {
  if (st->gate & (kGateKrylov | kGateDone)) return;
  constexpr int NM = 3 * MOTO_MAX_K;
  constexpr int LD = NM + 1;
  __shared__ double A[NM * LD], V[NM * LD], G[NM * NM], Mm[NM * NM], Z[NM * NM];
  __shared__ double cs[NM / 2 + 1], sn[NM / 2 + 1], red[32], dinv[NM], w[NM];
  __shared__ int pp[NM / 2 + 1], qq[NM / 2 + 1], keep_idx[NM];
  __shared__ int nkeep;
  const int n = nb * k;
  // assemble G and M (symmetrised)
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    const int r = idx / n, c = idx - r * n;
    const int cb = c / k, cc = c - cb * k;
    const int rb = r / k, rr = r - rb * k;
    const double g1 = Gb[(size_t)cb * n * k + r * k + cc], g2 = Gb[(size_t)rb * n * k + c * k + rr];
    const double m1 = Mb[(size_t)cb * n * k + r * k + cc], m2 = Mb[(size_t)rb * n * k + c * k + rr];
    G[r * NM + c] = 0.5 * (g1 + g2);
    Mm[r * NM + c] = 0.5 * (m1 + m2);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double d = G[i * NM + i];
    dinv[i] = d > 0.0 ? 1.0 / sqrt(d) : 0.0;
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    const int r = idx / n, c = idx - r * n;
    A[r * LD + c] = dinv[r] * G[r * NM + c] * dinv[c];
  }
  __syncthreads();
  block_jacobi(A, V, n, LD, cs, sn, pp, qq, red);
  if (threadIdx.x == 0) {
    double wmax = 0.0;
    for (int i = 0; i < n; ++i) wmax = fmax(wmax, A[i * LD + i]);
    // kept directions in ascending eigenvalue order of the scaled Gram
    int cnt = 0;
    for (int rank = 0; rank < n; ++rank)
      for (int i = 0; i < n; ++i)
        if (diag_rank(A, LD, n, i) == rank && A[i * LD + i] > drop * wmax) {
          keep_idx[cnt] = i;
          w[cnt] = A[i * LD + i];
          ++cnt;
        }
    nkeep = cnt;
  }
  __syncthreads();
  const int nk = nkeep;
  // Z = D U_keep w^-1/2  (n x nk)
  for (int idx = threadIdx.x; idx < n * nk; idx += blockDim.x) {
    const int r = idx / nk, c = idx - r * nk;
    Z[r * NM + c] = dinv[r] * V[r * LD + keep_idx[c]] / sqrt(w[c]);
  }
  __syncthreads();
  // A = Z^T M Z (nk x nk)
  for (int idx = threadIdx.x; idx < n * nk; idx += blockDim.x) {
    const int r = idx / nk, c = idx - r * nk;  // tmp = M Z  stored in V (n x nk)
    double a = 0.0;
    for (int t = 0; t < n; ++t) a += Mm[r * NM + t] * Z[t * NM + c];
    V[r * LD + c] = a;
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < nk * nk; idx += blockDim.x) {
    const int r = idx / nk, c = idx - r * nk;
    double a = 0.0;
    for (int t = 0; t < n; ++t) a += Z[t * NM + r] * V[t * LD + c];
    A[r * LD + c] = a;
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < nk * nk; idx += blockDim.x) {
    const int r = idx / nk, c = idx - r * nk;
    G[r * NM + c] = 0.5 * (A[r * LD + c] + A[c * LD + r]);
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < nk * nk; idx += blockDim.x) {
    const int r = idx / nk, c = idx - r * nk;
    A[r * LD + c] = G[r * NM + c];
  }
  __syncthreads();
  block_jacobi(A, V, nk, LD, cs, sn, pp, qq, red);
  // ascending order; Cx = Z U2[:, :k]
  for (int i = threadIdx.x; i < nk; i += blockDim.x) {
    const int rank = diag_rank(A, LD, nk, i);
    if (rank < k) {
      theta[rank] = A[i * LD + i];
      for (int r = 0; r < n; ++r) {
        double a = 0.0;
        for (int t = 0; t < nk; ++t) a += Z[r * NM + t] * V[t * LD + i];
        Cx[r * k + rank] = a;
        Cp[r * k + rank] = r < k ? 0.0 : a;
      }
    }
  }
  if (threadIdx.x == 0) {
    double h = st->hnorm;
    for (int i = 0; i < nk; ++i) h = fmax(h, fabs(A[i * LD + i]));
    st->hnorm = h;
  }
}

void launch_lob_rr(const double* Gb, const double* Mb, int k, int nb, double drop, double* Cx, double* Cp,
                   double* theta, DevState* st, cudaStream_t s) {
  lob_rr_kernel<<<1, 256, 0, s>>>(Gb, Mb, k, nb, drop, Cx, Cp, theta, st);
}

// LOBPCG convergence test on the residual Gram diagonal; also builds the
// coefficient matrix diag(theta) used to form R = AX - X theta, and sets the
// solver gate when max_j |r_j| <= tol * hnorm.
__global__ void lob_check_kernel(const double* Gw, int k, double tol, const double* theta, DevState* st) {
  if (threadIdx.x != 0) return;
  if (st->gate & (kGateKrylov | kGateDone)) return;
  double r = 0.0;
  for (int j = 0; j < k; ++j) r = fmax(r, sqrt(fmax(Gw[j * k + j], 0.0)));
  if (r <= tol * st->hnorm)
    st->gate |= kGateKrylov;
  else
    st->iters += 1;
  (void)theta;
}

void launch_lob_check(const double* Gw, int k, double tol, const double* theta, DevState* st, cudaStream_t s) {
  lob_check_kernel<<<1, 32, 0, s>>>(Gw, k, tol, theta, st);
}

// diag(theta) (k x k) and diag(1/sqrt(G_jj)) helpers for combine launches
__global__ void diag_kernel(const double* src, int k, int mode, double* out, const DevState* st, int mask) {
  if (st && (st->gate & mask)) return;
  for (int idx = threadIdx.x; idx < k * k; idx += blockDim.x) {
    const int r = idx / k, c = idx - r * k;
    double v = 0.0;
    if (r == c) {
      if (mode == 0)
        v = src[r];
      else {
        const double g = src[r * k + r];
        v = g > 0.0 ? 1.0 / sqrt(g) : 1.0;
      }
    }
    out[idx] = v;
  }
}

void launch_diag(const double* src, int k, int mode, double* out, const DevState* st, int mask, cudaStream_t s) {
  diag_kernel<<<1, 64, 0, s>>>(src, k, mode, out, st, mask);
}

// ===========================================================================
// MMF / L-BFGS
// ===========================================================================
// G = g - 2 reflect (g . v1) v1  (= -F_mmf for reflect = 1, F = -g);  max_i |G_i|.
template <typename T>
__global__ void __launch_bounds__(kThreads) mmf_force_kernel(const T* __restrict__ g, const T* __restrict__ V,
                                                             size_t ldv, int nv, const double* dots, T* G, int N,
                                                             double* part, unsigned* counter, double* fmax_out,
                                                             const int* gate, int mask, size_t ws) {
  g = wofs(g, ws);
  V = wofs(V, ws);
  dots = wofs(dots, ws);
  G = wofs(G, ws);
  part = wofs(part, ws);
  counter = wofs(counter, ws);
  fmax_out = wofs(fmax_out, ws);
  gate = wofs(gate, ws);
  if (gate && (*gate & mask)) return;
  __shared__ T a[MOTO_MAX_K];
  if (threadIdx.x < MOTO_MAX_K) a[threadIdx.x] = (int)threadIdx.x < nv ? (T)(2.0 * dots[threadIdx.x]) : (T)0;
  __syncthreads();
  T mxt = (T)0;  // the largest |G_i|^2 in the field precision (a max is exact)
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    T r[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const size_t e = (size_t)c * N + i;
      T v = g[e];
      for (int q = 0; q < nv; ++q) v -= a[q] * V[(size_t)q * ldv + e];
      r[c] = v;
      G[e] = v;
    }
    mxt = fmax(mxt, r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
  }
  __shared__ double red[8];
  double mx = block_max((double)mxt, red);
  if (threadIdx.x == 0) part[blockIdx.x] = mx;
  if (!grid_last_block(counter)) return;
  double b = 0.0;
  for (int k = threadIdx.x; k < (int)gridDim.x; k += blockDim.x) b = fmax(b, __ldcg(part + k));
  b = block_max(b, red);
  if (threadIdx.x == 0) {
    fmax_out[0] = sqrt(b);
    *counter = 0u;
  }
}

template <typename T>
void launch_mmf_force(const T* g, const T* V, size_t ldv, int nv, const double* dots, T* G, int N, double* part,
                      unsigned* counter, double* fmax_out, const int* gate, int mask, cudaStream_t st) {
  mmf_force_kernel<T><<<wgrid(stream_grid<T>(N)), kThreads, 0, st>>>(g, nv > 0 ? V : nullptr, ldv, nv, dots, G, N, part,
                                                           counter, fmax_out, gate, mask, walker_ws());
}

// ---- nonlinear CG (Polak-Ribiere+, spectral step; see internal.h) ----
__global__ void cg_coeffs_kernel(double* cg, double gamma0, DevState* dst) {
  if (threadIdx.x != 0 || (dst->gate & kGateDone)) return;
  double beta = 0.0, alpha = gamma0;
  if (dst->lb_have_prev) {
    beta = cg[9] > 0.0 ? fmax(0.0, cg[6] / cg[9]) : 0.0;  // G.(G - P G_prev) = G.y
    const double ss = cg[4], sy = cg[5], yy = cg[8];
    if (sy > 1e-12 * sqrt(ss * yy)) alpha = sy / yy;
  }
  cg[10] = beta;
  cg[11] = alpha;
  cg[9] = cg[0];  // |G|^2 becomes |G_prev|^2 of the next step
  dst->lb_have_prev = 1;
}

void launch_cg_coeffs(double* cg, double gamma0, DevState* dst, cudaStream_t st) {
  cg_coeffs_kernel<<<1, 32, 0, st>>>(cg, gamma0, dst);
}

template <typename T>
__global__ void __launch_bounds__(kThreads) cg_direction_kernel(const T* __restrict__ m, const T* __restrict__ G,
                                                                T* p, int N, const double* cg, double theta_max,
                                                                double* part, unsigned* counter, DevState* dst,
                                                                const int* gate, int mask) {
  if (gate && (*gate & mask)) return;
  const double beta_d = cg[10];
  const T beta = (T)beta_d;
  double v[3] = {0.0, 0.0, 0.0};  // p.G, max |p_i|^2, max |G_i|^2
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    T gv[3], pv[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) gv[c] = G[(size_t)c * N + i];
    if (beta_d != 0.0) {
      const T m0 = m[i], m1 = m[N + i], m2 = m[2 * (size_t)N + i];
      T q[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) q[c] = p[(size_t)c * N + i];
      const T pm = m0 * q[0] + m1 * q[1] + m2 * q[2];
      const T mm[3] = {m0, m1, m2};
#pragma unroll
      for (int c = 0; c < 3; ++c) pv[c] = -gv[c] + beta * (q[c] - pm * mm[c]);
    } else {
#pragma unroll
      for (int c = 0; c < 3; ++c) pv[c] = -gv[c];
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) p[(size_t)c * N + i] = pv[c];
    v[0] += (double)(pv[0] * gv[0] + pv[1] * gv[1] + pv[2] * gv[2]);
    v[1] = fmax(v[1], (double)(pv[0] * pv[0] + pv[1] * pv[1] + pv[2] * pv[2]));
    v[2] = fmax(v[2], (double)(gv[0] * gv[0] + gv[1] * gv[1] + gv[2] * gv[2]));
  }
  __shared__ double red[3 * (kThreads / 32)];
  double s1[1] = {v[0]};
  block_sum<1>(s1, red);
  const double m1 = block_max(v[1], red);
  const double m2 = block_max(v[2], red);
  if (threadIdx.x == 0) {
    part[(size_t)blockIdx.x * 3 + 0] = s1[0];
    part[(size_t)blockIdx.x * 3 + 1] = m1;
    part[(size_t)blockIdx.x * 3 + 2] = m2;
  }
  if (!grid_last_block(counter)) return;
  __shared__ double tot[1];
  grid_sum_entries(part, gridDim.x, 3, red);  // red[0] is the p.G total (maxima below)
  __syncthreads();
  if (threadIdx.x == 0) tot[0] = red[0];
  __syncthreads();
  double a1 = 0.0, a2 = 0.0;
  for (int k = threadIdx.x; k < (int)gridDim.x; k += blockDim.x) {
    a1 = fmax(a1, __ldcg(part + (size_t)k * 3 + 1));
    a2 = fmax(a2, __ldcg(part + (size_t)k * 3 + 2));
  }
  a1 = block_max(a1, red);
  a2 = block_max(a2, red);
  if (threadIdx.x == 0) {
    const bool restart = !(tot[0] < 0.0);  // p is not a descent direction for G
    const double alpha = cg[11];
    const double t = sqrt(restart ? a2 : a1);
    dst->pad[2] = restart ? 1 : 0;
    dst->scale = (alpha * t > theta_max) ? theta_max / t : alpha;
    *counter = 0u;
  }
}

template <typename T>
void launch_cg_direction(const T* m, const T* G, T* p, int N, const double* cg, double theta_max, double* part,
                         unsigned* counter, DevState* dst, const int* gate, int mask, cudaStream_t st) {
  cg_direction_kernel<T><<<stream_grid<T>(N), kThreads, 0, st>>>(m, G, p, N, cg, theta_max, part, counter, dst, gate,
                                                              mask);
}

// New pair at the current point: s = P d_prev, y = G - P G_prev, written into
// ring slot lb_head (interleaved storage: s at 2*head, y at 2*head+1) and into
// the two staging fields (contiguous, for the Gram launch).
template <typename T>
__global__ void lbfgs_pair_kernel(const T* __restrict__ m, const T* __restrict__ d_prev,
                                  const T* __restrict__ G_prev, const T* __restrict__ G, T* ring, size_t ld,
                                  T* stage, const DevState* dst, int N, const int* gate, int mask, size_t ws) {
  m = wofs(m, ws);
  d_prev = wofs(d_prev, ws);
  G_prev = wofs(G_prev, ws);
  G = wofs(G, ws);
  ring = wofs(ring, ws);
  stage = wofs(stage, ws);
  dst = wofs(dst, ws);
  gate = wofs(gate, ws);
  if (gate && (*gate & mask)) return;
  if (!dst->lb_have_prev) return;
  T* s_out = ring + (size_t)(2 * dst->lb_head) * ld;
  T* y_out = s_out + ld;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    const T m0 = m[i], m1 = m[N + i], m2 = m[2 * (size_t)N + i];
    T d[3], gp[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      d[c] = d_prev[(size_t)c * N + i];
      gp[c] = G_prev[(size_t)c * N + i];
    }
    const T pd = m0 * d[0] + m1 * d[1] + m2 * d[2];
    const T pg = m0 * gp[0] + m1 * gp[1] + m2 * gp[2];
    const T mm[3] = {m0, m1, m2};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const size_t e = (size_t)c * N + i;
      const T sv = d[c] - pd * mm[c];
      const T yv = G[e] - (gp[c] - pg * mm[c]);
      s_out[e] = sv;
      y_out[e] = yv;
      stage[e] = sv;
      stage[ld + e] = yv;
    }
  }
}

template <typename T>
void launch_lbfgs_pair(const T* m, const T* d_prev, const T* G_prev, const T* G, T* ring, size_t ld, T* stage,
                       const DevState* dst, int N, const int* gate, int mask, cudaStream_t st) {
  lbfgs_pair_kernel<T><<<wgrid(stream_grid<T>(N)), kThreads, 0, st>>>(m, d_prev, G_prev, G, ring, ld, stage, dst, N, gate,
                                                            mask, walker_ws());
}

// Two-loop recursion in coefficient space over the basis
//   b_{2j} = s_j, b_{2j+1} = y_j (j < R = mem + 1 ring slots), b_{2R} = G.
// The ring keeps `lb_count` <= mem accepted pairs in the slots preceding
// `lb_head`; slot lb_head is free and receives the next candidate pair, so a
// rejected candidate never evicts a kept pair.  M is the persistent
// (2R+1)^2 Gram matrix of the basis.  newdots holds, for every basis vector
// t, its dots with G, the candidate s and the candidate y at 3 t, 3 t + 1 and
// 3 t + 2.
__global__ void lbfgs_solve_kernel(double* Mg, int mem, const double* newdots, double gamma0, double* coef,
                                   DevState* dst, size_t ws) {
  Mg = wofs(Mg, ws);
  newdots = wofs(newdots, ws);
  coef = wofs(coef, ws);
  dst = wofs(dst, ws);
  if (dst->gate & kGateDone) return;
  const int R = mem + 1;
  const int nb = 2 * R + 1, gi = 2 * R;
  // the recursion is one thread's chain of dependent steps: M and the new
  // dots are staged in shared memory by the warp first (one round trip)
  constexpr int kNbMax = 2 * MOTO_MAX_MEM + 3;
  __shared__ double M[kNbMax * kNbMax], nd[3 * kNbMax];
  for (int i = threadIdx.x; i < nb * nb; i += blockDim.x) M[i] = Mg[i];
  for (int i = threadIdx.x; i < 3 * nb; i += blockDim.x) nd[i] = newdots[i];
  __syncthreads();
  if (threadIdx.x == 0) {
  if (dst->lb_have_prev) {
    const int h = dst->lb_head;
    const int si = 2 * h, yi = 2 * h + 1;
    for (int t = 0; t < nb; ++t) {
      M[si * nb + t] = M[t * nb + si] = nd[t * 3 + 1];
      M[yi * nb + t] = M[t * nb + yi] = nd[t * 3 + 2];
    }
    const double sy = M[si * nb + yi], ss = M[si * nb + si], yy = M[yi * nb + yi];
    if (sy > 1e-12 * sqrt(ss * yy)) {
      dst->lb_head = (h + 1) % R;
      dst->lb_count = min(dst->lb_count + 1, mem);
    }
  }
  for (int t = 0; t < nb; ++t) M[gi * nb + t] = M[t * nb + gi] = nd[t * 3];
  // coefficient-space dot products: u^T M w
  auto dotc = [&](const double* u, const double* w) {
    double a = 0.0;
    for (int r = 0; r < nb; ++r) {
      if (u[r] == 0.0) continue;
      double b = 0.0;
      for (int c = 0; c < nb; ++c) b += M[r * nb + c] * w[c];
      a += u[r] * b;
    }
    return a;
  };
  double q[2 * MOTO_MAX_MEM + 3], e[2 * MOTO_MAX_MEM + 3], alpha[MOTO_MAX_MEM], rho[MOTO_MAX_MEM];
  for (int t = 0; t < nb; ++t) q[t] = 0.0;
  q[gi] = 1.0;
  const int cnt = dst->lb_count;
  // newest .. oldest
  for (int k = 0; k < cnt; ++k) {
    const int slot = ((dst->lb_head - 1 - k) % R + R) % R;
    const int si = 2 * slot, yi = si + 1;
    rho[k] = 1.0 / M[yi * nb + si];
    for (int t = 0; t < nb; ++t) e[t] = 0.0;
    e[si] = 1.0;
    alpha[k] = rho[k] * dotc(e, q);
    q[yi] -= alpha[k];
  }
  double gamma = gamma0;
  if (cnt > 0) {
    const int slot = ((dst->lb_head - 1) % R + R) % R;
    const int si = 2 * slot, yi = si + 1;
    gamma = M[si * nb + yi] / M[yi * nb + yi];
  }
  for (int t = 0; t < nb; ++t) q[t] *= gamma;  // r
  // oldest .. newest
  for (int k = cnt - 1; k >= 0; --k) {
    const int slot = ((dst->lb_head - 1 - k) % R + R) % R;
    const int si = 2 * slot, yi = si + 1;
    for (int t = 0; t < nb; ++t) e[t] = 0.0;
    e[yi] = 1.0;
    const double beta = rho[k] * dotc(e, q);
    q[si] += alpha[k] - beta;
  }
  for (int t = 0; t < nb; ++t) q[t] = -q[t];  // d = -r
  for (int t = 0; t < nb; ++t) e[t] = 0.0;
  e[gi] = 1.0;
  if (dotc(q, e) >= 0.0) {
    dst->lb_count = 0;
    for (int t = 0; t < nb; ++t) q[t] = 0.0;
    q[gi] = -gamma0;
  }
  for (int t = 0; t < nb; ++t) coef[t] = q[t];
  dst->lb_have_prev = 1;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < nb * nb; i += blockDim.x) Mg[i] = M[i];
}

void launch_lbfgs_solve(double* M, int mem, const double* newdots, double gamma0, double* coef, DevState* dst,
                        cudaStream_t st) {
  lbfgs_solve_kernel<<<wgrid(1), 32, 0, st>>>(M, mem, newdots, gamma0, coef, dst, walker_ws());
}

// d = P(sum_t coef_t b_t); max_i |d_i| -> step scale min(1, theta_max / max).
template <typename T>
__global__ void __launch_bounds__(kThreads) lbfgs_direction_kernel(const T* __restrict__ basis, size_t ld, int nb,
                                                                   const double* coef, const T* __restrict__ m,
                                                                   T* d, int N, double theta_max, double* part,
                                                                   unsigned* counter, DevState* dst,
                                                                   const int* gate, int mask, size_t ws) {
  basis = wofs(basis, ws);
  coef = wofs(coef, ws);
  m = wofs(m, ws);
  d = wofs(d, ws);
  part = wofs(part, ws);
  counter = wofs(counter, ws);
  dst = wofs(dst, ws);
  gate = wofs(gate, ws);
  if (gate && (*gate & mask)) return;
  __shared__ T cf[2 * MOTO_MAX_MEM + 3];
  if (threadIdx.x < nb) cf[threadIdx.x] = (T)coef[threadIdx.x];
  __syncthreads();
  T mxt = (T)0;  // the largest |d_i|^2 in the field precision (a max is exact)
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    T a[3] = {0, 0, 0};
    for (int t = 0; t < nb; ++t) {
      const T w = cf[t];
      if (w == (T)0) continue;
      const T* b = basis + (size_t)t * ld;
      a[0] += w * b[i];
      a[1] += w * b[N + i];
      a[2] += w * b[2 * (size_t)N + i];
    }
    const T m0 = m[i], m1 = m[N + i], m2 = m[2 * (size_t)N + i];
    const T p = m0 * a[0] + m1 * a[1] + m2 * a[2];
    a[0] -= p * m0;
    a[1] -= p * m1;
    a[2] -= p * m2;
    d[i] = a[0];
    d[N + i] = a[1];
    d[2 * (size_t)N + i] = a[2];
    mxt = fmax(mxt, a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
  }
  __shared__ double red[8];
  double mx = block_max((double)mxt, red);
  if (threadIdx.x == 0) part[blockIdx.x] = mx;
  if (!grid_last_block(counter)) return;
  double b = 0.0;
  for (int k = threadIdx.x; k < (int)gridDim.x; k += blockDim.x) b = fmax(b, __ldcg(part + k));
  b = block_max(b, red);
  if (threadIdx.x == 0) {
    const double t = sqrt(b);
    dst->scale = (t > theta_max) ? theta_max / t : 1.0;
    *counter = 0u;
  }
}

template <typename T>
void launch_lbfgs_direction(const T* basis, size_t ld, int nb, const double* coef, const T* m, T* d, int N,
                            double theta_max, double* part, unsigned* counter, DevState* dst, const int* gate,
                            int mask, cudaStream_t st) {
  lbfgs_direction_kernel<T><<<wgrid(stream_grid<T>(N)), kThreads, 0, st>>>(basis, ld, nb, coef, m, d, N, theta_max, part,
                                                                 counter, dst, gate, mask, walker_ws());
}

// d <- scale d;  m_i <- m_i cos|d_i| + d_i/|d_i| sin|d_i|, renormalised.
template <typename T>
__device__ __forceinline__ void rodrigues(T& m0, T& m1, T& m2, T d0, T d1, T d2) {
  const T th = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
  if (th > (T)0) {
    T sn, cs;
    if (sizeof(T) == 4) {
      float sf, cf;
      sincosf((float)th, &sf, &cf);
      sn = (T)sf;
      cs = (T)cf;
    } else {
      double sd, cd;
      sincos((double)th, &sd, &cd);
      sn = (T)sd;
      cs = (T)cd;
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

template <typename T>
__global__ void retract_kernel(T* m, T* d, const DevState* dst, int N, const int* gate, int mask, size_t ws) {
  m = wofs(m, ws);
  d = wofs(d, ws);
  dst = wofs(dst, ws);
  gate = wofs(gate, ws);
  if (gate && (*gate & mask)) return;
  const T sc = (T)dst->scale;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    T d0 = d[i] * sc, d1 = d[N + i] * sc, d2 = d[2 * (size_t)N + i] * sc;
    d[i] = d0;
    d[N + i] = d1;
    d[2 * (size_t)N + i] = d2;
    T m0 = m[i], m1 = m[N + i], m2 = m[2 * (size_t)N + i];
    rodrigues(m0, m1, m2, d0, d1, d2);
    m[i] = m0;
    m[N + i] = m1;
    m[2 * (size_t)N + i] = m2;
  }
}

template <typename T>
void launch_retract(T* m, T* d, const DevState* dst, int N, const int* gate, int mask, cudaStream_t st) {
  retract_kernel<T><<<wgrid(stream_grid<T>(N)), kThreads, 0, st>>>(m, d, dst, N, gate, mask, walker_ws());
}

template <typename T>
__global__ void cg_retract_kernel(T* m, const T* __restrict__ G, T* p, T* d, const DevState* dst, int N,
                                  const int* gate, int mask) {
  if (gate && (*gate & mask)) return;
  const bool restart = dst->pad[2] != 0;
  const T sc = (T)dst->scale;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    T dv[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const size_t e = (size_t)c * N + i;
      T dir = p[e];
      if (restart) {
        dir = -G[e];
        p[e] = dir;
      }
      dv[c] = dir * sc;
      d[e] = dv[c];
    }
    T m0 = m[i], m1 = m[N + i], m2 = m[2 * (size_t)N + i];
    rodrigues(m0, m1, m2, dv[0], dv[1], dv[2]);
    m[i] = m0;
    m[N + i] = m1;
    m[2 * (size_t)N + i] = m2;
  }
}

template <typename T>
void launch_cg_retract(T* m, const T* G, T* p, T* d, const DevState* dst, int N, const int* gate, int mask,
                       cudaStream_t st) {
  cg_retract_kernel<T><<<stream_grid<T>(N), kThreads, 0, st>>>(m, G, p, d, dst, N, gate, mask);
}

// ---- damped spin dynamics (Landau-Lifshitz-Gilbert, Heun; see internal.h) ----
template <typename T>
__device__ __forceinline__ void llg_rate(const T (&m)[3], const T (&g)[3], T c1, T c2, T (&f)[3]) {
  // f = (m x g - alpha g) / (1 + alpha^2) = c1 (m x g) - c2 g
  f[0] = c1 * (m[1] * g[2] - m[2] * g[1]) - c2 * g[0];
  f[1] = c1 * (m[2] * g[0] - m[0] * g[2]) - c2 * g[1];
  f[2] = c1 * (m[0] * g[1] - m[1] * g[0]) - c2 * g[2];
}
template <typename T>
__device__ __forceinline__ void unit3(T (&x)[3]) {
  const T inv = (T)1 / sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
  x[0] *= inv;
  x[1] *= inv;
  x[2] *= inv;
}

template <typename T>
__global__ void llg_predict_kernel(const T* __restrict__ m, const T* __restrict__ g, T* mp, T c1, T c2, T dt, int N,
                                   const int* gate, int mask) {
  if (gate && (*gate & mask)) return;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    T mm[3], gg[3], f[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      mm[c] = m[(size_t)c * N + i];
      gg[c] = g[(size_t)c * N + i];
    }
    llg_rate(mm, gg, c1, c2, f);
    T x[3] = {mm[0] + dt * f[0], mm[1] + dt * f[1], mm[2] + dt * f[2]};
    unit3(x);
#pragma unroll
    for (int c = 0; c < 3; ++c) mp[(size_t)c * N + i] = x[c];
  }
}

template <typename T>
__global__ void llg_correct_kernel(T* m, const T* __restrict__ g0, const T* __restrict__ mp,
                                   const T* __restrict__ g1, T c1, T c2, T hdt, int N, const int* gate, int mask) {
  if (gate && (*gate & mask)) return;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    T mm[3], ga[3], mq[3], gb[3], f1[3], f2[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const size_t e = (size_t)c * N + i;
      mm[c] = m[e];
      ga[c] = g0[e];
      mq[c] = mp[e];
      gb[c] = g1[e];
    }
    llg_rate(mm, ga, c1, c2, f1);
    llg_rate(mq, gb, c1, c2, f2);
    T x[3] = {mm[0] + hdt * (f1[0] + f2[0]), mm[1] + hdt * (f1[1] + f2[1]), mm[2] + hdt * (f1[2] + f2[2])};
    unit3(x);
#pragma unroll
    for (int c = 0; c < 3; ++c) m[(size_t)c * N + i] = x[c];
  }
}

template <typename T>
void launch_llg_predict(const T* m, const T* g, T* mp, double alpha, double dt, int N, const int* gate, int mask,
                        cudaStream_t st) {
  const double d = 1.0 + alpha * alpha;
  llg_predict_kernel<T><<<stream_grid<T>(N), kThreads, 0, st>>>(m, g, mp, (T)(1.0 / d), (T)(alpha / d), (T)dt, N, gate,
                                                             mask);
}
template <typename T>
void launch_llg_correct(T* m, const T* g0, const T* mp, const T* g1, double alpha, double dt, int N,
                        const int* gate, int mask, cudaStream_t st) {
  const double d = 1.0 + alpha * alpha;
  llg_correct_kernel<T><<<stream_grid<T>(N), kThreads, 0, st>>>(m, g0, mp, g1, (T)(1.0 / d), (T)(alpha / d),
                                                             (T)(0.5 * dt), N, gate, mask);
}

// Descent seed: out = Rodrigues(m, sign * eta * v1), eta = eta_theta / max|v1_i|.
template <typename T>
__global__ void __launch_bounds__(kThreads) vmax_kernel(const T* v, int N, double* part, unsigned* counter,
                                                        double* out, size_t ws) {
  v = wofs(v, ws);
  part = wofs(part, ws);
  counter = wofs(counter, ws);
  out = wofs(out, ws);
  double mx = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    const double a = v[i], b = v[N + i], c = v[2 * (size_t)N + i];
    mx = fmax(mx, a * a + b * b + c * c);
  }
  __shared__ double red[8];
  mx = block_max(mx, red);
  if (threadIdx.x == 0) part[blockIdx.x] = mx;
  if (!grid_last_block(counter)) return;
  double b = 0.0;
  for (int k = threadIdx.x; k < (int)gridDim.x; k += blockDim.x) b = fmax(b, __ldcg(part + k));
  b = block_max(b, red);
  if (threadIdx.x == 0) {
    out[0] = sqrt(b);
    *counter = 0u;
  }
}

template <typename T>
__global__ void seed_kernel(const T* m, const T* v1, const double* vmax, double eta_theta, double sign, T* out,
                            int N, size_t ws) {
  m = wofs(m, ws);
  v1 = wofs(v1, ws);
  vmax = wofs(vmax, ws);
  out = wofs(out, ws);
  const T f = (T)(sign * eta_theta / vmax[0]);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    T m0 = m[i], m1 = m[N + i], m2 = m[2 * (size_t)N + i];
    rodrigues(m0, m1, m2, f * v1[i], f * v1[N + i], f * v1[2 * (size_t)N + i]);
    out[i] = m0;
    out[N + i] = m1;
    out[2 * (size_t)N + i] = m2;
  }
}

template <typename T>
void launch_descent_seed(const T* m, const T* v1, double eta_theta, double sign, T* out, int N, double* part,
                         unsigned* counter, double* scal, cudaStream_t st) {
  vmax_kernel<T><<<wgrid(stream_grid<T>(N)), kThreads, 0, st>>>(v1, N, part, counter, scal, walker_ws());
  seed_kernel<T><<<wgrid(stream_grid<T>(N)), kThreads, 0, st>>>(m, v1, scal, eta_theta, sign, out, N, walker_ws());
}

// Saddle / minimum test and the per-step output vector.
// last: the final test of a run (no step follows it, so none is counted)
// indexed: out6 is the first row of a trace; the record goes to the row of
// the outer steps taken so far (dst->pad[1], at most rows - 1), so a captured
// step writes each replay's record to its own row.
__global__ void saddle_test_kernel(const double* eg_out, const double* fmax, const double* lam, const double* gdot,
                                   double tau_F, double tau_lambda, double* out6, int* status_out, DevState* dst,
                                   int ascent, int last, int indexed, size_t ws) {
  eg_out = wofs(eg_out, ws);
  fmax = wofs(fmax, ws);
  lam = wofs(lam, ws);
  gdot = wofs(gdot, ws);
  out6 = wofs(out6, ws);
  status_out = wofs(status_out, ws);
  dst = wofs(dst, ws);
  if (threadIdx.x != 0) return;
  if (dst->gate & kGateDone) {
    if (status_out) *status_out = 1;
    return;
  }
  const double E = eg_out[0], gmax = eg_out[1];
  if (out6 && indexed > 0) out6 += 6 * (size_t)min(max(dst->pad[1], 0), indexed - 1);
  bool conv;
  if (ascent) {
    // lambda_1 < 0 < lambda_2 with the curvature threshold tau_lambda:
    // lambda_1 clearly negative, lambda_2 not below -tau_lambda
    conv = fmax[0] <= tau_F && lam[0] < -tau_lambda && -tau_lambda < lam[1];
    if (out6) {
      out6[0] = E;
      out6[1] = fmax[0];
      out6[2] = lam[0];
      out6[3] = lam[1];
      out6[4] = gmax;
      out6[5] = -gdot[0];  // F . v1 = -g . v1
    }
  } else {
    conv = gmax <= tau_F;
    if (out6) {
      out6[0] = E;
      out6[1] = gmax;
    }
  }
  if (!isfinite(E) || !isfinite(gmax)) dst->status |= kStatusNonfinite;
  if (conv) {
    dst->gate |= kGateDone;
    dst->converged = 1;
  } else if (!last) {
    dst->pad[1] += 1;  // outer steps taken
  }
  if (status_out) *status_out = conv ? 1 : 0;
}

void launch_saddle_test(const double* eg_out, const double* fmax, const double* lam, const double* gdot,
                        double tau_F, double tau_lambda, double* out6, int* status_out, DevState* dst, int ascent,
                        int last, int indexed, cudaStream_t st) {
  saddle_test_kernel<<<wgrid(1), 32, 0, st>>>(eg_out, fmax, lam, gdot, tau_F, tau_lambda, out6, status_out, dst, ascent,
                                       last, indexed, walker_ws());
}

#define INST(T)                                                                                                   \
  template void launch_gram<T>(const T*, size_t, int, const T*, size_t, int, size_t, double*, double*, unsigned*, \
                               const int*, int, cudaStream_t);                                                    \
  template bool launch_chol2<T>(const T*, size_t, int, const double*, const double*, T*, size_t, const T*, int,  \
                                double*, double*, unsigned*, const int*, int, bool, cudaStream_t);             \
  template void launch_combine<T>(const T*, size_t, int, const int*, const double*, int, const T*, size_t,        \
                                  double, double, T*, size_t, const T*, int, const int*, int, cudaStream_t);      \
  template void launch_project<T>(const T*, const T*, size_t, T*, size_t, int, int, const int*, int,              \
                                  cudaStream_t);                                                                  \
  template void launch_finish<T>(const T*, T*, size_t, int, int, double*, unsigned*, double*, const int*, int,    \
                                 cudaStream_t);                                                                   \
  template void launch_mmf_force<T>(const T*, const T*, size_t, int, const double*, T*, int, double*, unsigned*,  \
                                    double*, const int*, int, cudaStream_t);                                      \
  template void launch_cg_direction<T>(const T*, const T*, T*, int, const double*, double, double*, unsigned*,   \
                                       DevState*, const int*, int, cudaStream_t);                                 \
  template void launch_cg_retract<T>(T*, const T*, T*, T*, const DevState*, int, const int*, int, cudaStream_t);  \
  template void launch_llg_predict<T>(const T*, const T*, T*, double, double, int, const int*, int, cudaStream_t); \
  template void launch_llg_correct<T>(T*, const T*, const T*, const T*, double, double, int, const int*, int,     \
                                      cudaStream_t);                                                             \
  template void launch_lbfgs_pair<T>(const T*, const T*, const T*, const T*, T*, size_t, T*, const DevState*,     \
                                     int, const int*, int, cudaStream_t);                                         \
  template void launch_lbfgs_direction<T>(const T*, size_t, int, const double*, const T*, T*, int, double,        \
                                          double*, unsigned*, DevState*, const int*, int, cudaStream_t);          \
  template void launch_retract<T>(T*, T*, const DevState*, int, const int*, int, cudaStream_t);                   \
  template void launch_descent_seed<T>(const T*, const T*, double, double, T*, int, double*, unsigned*, double*,  \
                                       cudaStream_t);
INST(float)
INST(double)
#undef INST

}  // namespace moto
