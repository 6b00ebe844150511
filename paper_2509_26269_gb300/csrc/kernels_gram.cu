// Skinny Gram product out[r][c] = X_r . Y_c  (nx <= 96 rows, ny <= 8 columns,
// n elements), the reorthogonalisation and Rayleigh-Ritz workhorse of the
// Krylov solvers.  HBM-bound: every element of the nx + ny fields is read once.
//
// Pipeline: one persistent block per SM walks a contiguous range of 1 KB
// element tiles.  Per tile, one thread issues nx + ny bulk copies
// (cp.async.bulk, the TMA engine) of 1 KB rows into a two-stage shared-memory
// ring completed on an mbarrier (transaction bytes).  Warp w owns rows
// [R w, R w + R), lane l owns elements l, l + 32, ...; each lane keeps an
// R x NY block of FP32 partial sums in registers, flushed every kFlush tiles
// by a warp reduction into FP64 accumulators in shared memory.  Block results
// go to FP64 partials reduced in block order by the last block.
#include "internal.h"

namespace moto {

namespace {

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_async_shared() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait: gives up after ~2^22 polls (each poll may itself suspend for a
// while) and reports a timeout instead of hanging.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity) {
  for (int i = 0; i < (1 << 22); ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

constexpr int kStages = 2;
constexpr int kFlush = 4;  // tiles between FP32 -> FP64 flushes

}  // namespace

template <typename T, int R, int NY>
__global__ void __launch_bounds__(256, 1) gram_tma_kernel(const T* __restrict__ X, size_t ldx, int nx,
                                                          const T* __restrict__ Y, size_t ldy, int ny, size_t n,
                                                          double* out, double* part, unsigned* counter,
                                                          const int* gate, int mask, int* status) {
  if (gate && (*gate & mask)) return;
  constexpr int KT = 1024 / (int)sizeof(T);  // elements per 1 KB row chunk
  constexpr int VEC = 16 / (int)sizeof(T);   // elements per 16 B
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) uint64_t full[kStages];
  __shared__ double facc[MOTO_MAX_BASIS * 8];
  __shared__ int timed_out;
  const int rows = nx + ny;
  T* stage_buf = reinterpret_cast<T*>(smem);
  const size_t stage_elems = (size_t)rows * KT;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int r0 = w * R;

  const size_t ntiles = (n + KT - 1) / KT;
  const size_t t_begin = ntiles * blockIdx.x / gridDim.x;
  const size_t t_end = ntiles * (blockIdx.x + 1) / gridDim.x;

  for (int i = threadIdx.x; i < nx * ny; i += blockDim.x) facc[i] = 0.0;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) mbar_init(&full[s], 1);
    timed_out = 0;
    fence_async_shared();
  }
  __syncthreads();

  // issue tile t into stage s: bulk copies for the 16 B-aligned prefix, plain
  // loads for the ragged remainder and zeros past the end
  auto issue = [&](size_t t, int s) {
    const size_t e0 = t * KT;
    const int len = (int)min((size_t)KT, n - e0);
    const int pre = (len / VEC) * VEC;
    T* buf = stage_buf + (size_t)s * stage_elems;
    if (threadIdx.x == 0) {
      fence_async_shared();
      mbar_expect_tx(&full[s], (unsigned)(pre * sizeof(T)) * rows);
      if (pre > 0) {
        for (int r = 0; r < nx; ++r) bulk_g2s(buf + (size_t)r * KT, X + (size_t)r * ldx + e0, pre * sizeof(T), &full[s]);
        for (int c = 0; c < ny; ++c)
          bulk_g2s(buf + (size_t)(nx + c) * KT, Y + (size_t)c * ldy + e0, pre * sizeof(T), &full[s]);
      }
    }
    if (pre < KT) {
      const int tail = KT - pre;
      for (int idx = threadIdx.x; idx < rows * tail; idx += blockDim.x) {
        const int r = idx / tail, k = pre + (idx - r * tail);
        T v = (T)0;
        if (k < len) v = r < nx ? X[(size_t)r * ldx + e0 + k] : Y[(size_t)(r - nx) * ldy + e0 + k];
        buf[(size_t)r * KT + k] = v;
      }
    }
  };

  for (int s = 0; s < kStages; ++s)
    if (t_begin + s < t_end) issue(t_begin + s, s);
  __syncthreads();

  T acc[R][NY];
#pragma unroll
  for (int j = 0; j < R; ++j)
#pragma unroll
    for (int c = 0; c < NY; ++c) acc[j][c] = (T)0;

  auto flush = [&]() {
#pragma unroll
    for (int j = 0; j < R; ++j) {
#pragma unroll
      for (int c = 0; c < NY; ++c) {
        T v = acc[j][c];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0 && r0 + j < nx && c < ny) facc[(r0 + j) * ny + c] += (double)v;
        acc[j][c] = (T)0;
      }
    }
  };

  int since = 0;
  for (size_t t = t_begin; t < t_end; ++t) {
    const int it = (int)(t - t_begin);
    const int s = it % kStages;
    const unsigned parity = (unsigned)((it / kStages) & 1);
    const bool ok = mbar_wait(&full[s], parity);
    if (__syncthreads_or(!ok)) {  // every thread leaves the loop together
      if (threadIdx.x == 0) {
        timed_out = 1;
        if (status) atomicOr(status, kStatusTimeout);
      }
      break;
    }
    const T* buf = stage_buf + (size_t)s * stage_elems;
    const T* Ys = buf + (size_t)nx * KT;
    if (r0 < nx) {
#pragma unroll 2
      for (int k = lane; k < KT; k += 32) {
        T y[NY];
#pragma unroll
        for (int c = 0; c < NY; ++c) y[c] = c < ny ? Ys[(size_t)c * KT + k] : (T)0;
#pragma unroll
        for (int j = 0; j < R; ++j) {
          if (r0 + j < nx) {
            const T x = buf[(size_t)(r0 + j) * KT + k];
#pragma unroll
            for (int c = 0; c < NY; ++c) acc[j][c] += x * y[c];
          }
        }
      }
    }
    if (++since == kFlush) {
      since = 0;
      if (r0 < nx) flush();
    }
    __syncthreads();  // every warp is done with stage s
    if (t + kStages < t_end) issue(t + kStages, s);
    __syncthreads();  // tail fill of the new tile visible before its compute
  }
  if (r0 < nx) flush();
  __syncthreads();
  if (timed_out) {
    // bounded drain: let bulk copies still in flight land before the block
    // exits (a phase that already completed returns at once)
    if (threadIdx.x == 0)
      for (int s = 0; s < kStages; ++s) {
        mbar_wait(&full[s], 0);
        mbar_wait(&full[s], 1);
      }
    __syncthreads();
  }
  const int nout = nx * ny;
  for (int o = threadIdx.x; o < nout; o += blockDim.x) part[(size_t)blockIdx.x * nout + o] = facc[o];
  if (!grid_last_block(counter)) return;
  grid_sum_entries(part, gridDim.x, nout, out);
  if (threadIdx.x == 0) *counter = 0u;
}

namespace {

template <typename T, int R, int NY>
void gram_tma_launch(const T* X, size_t ldx, int nx, const T* Y, size_t ldy, int ny, size_t n, double* out,
                     double* part, unsigned* counter, const int* gate, int mask, int* status, cudaStream_t st) {
  constexpr int KT = 1024 / (int)sizeof(T);
  const size_t smem = (size_t)kStages * (nx + ny) * KT * sizeof(T);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(gram_tma_kernel<T, R, NY>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
    attr = true;
  }
  const size_t ntiles = (n + KT - 1) / KT;
  const int grid = (int)(ntiles < (size_t)kSMs ? (ntiles > 0 ? ntiles : 1) : kSMs);
  gram_tma_kernel<T, R, NY><<<grid, 256, smem, st>>>(X, ldx, nx, Y, ldy, ny, n, out, part, counter, gate, mask,
                                                     status);
}

template <typename T, int NY>
void gram_tma_rows(const T* X, size_t ldx, int nx, const T* Y, size_t ldy, int ny, size_t n, double* out,
                   double* part, unsigned* counter, const int* gate, int mask, int* status, cudaStream_t st) {
  const int r = (nx + 7) / 8;
  if (r <= 1)
    gram_tma_launch<T, 1, NY>(X, ldx, nx, Y, ldy, ny, n, out, part, counter, gate, mask, status, st);
  else if (r <= 2)
    gram_tma_launch<T, 2, NY>(X, ldx, nx, Y, ldy, ny, n, out, part, counter, gate, mask, status, st);
  else if (r <= 4)
    gram_tma_launch<T, 4, NY>(X, ldx, nx, Y, ldy, ny, n, out, part, counter, gate, mask, status, st);
  else if (r <= 8)
    gram_tma_launch<T, 8, NY>(X, ldx, nx, Y, ldy, ny, n, out, part, counter, gate, mask, status, st);
  else
    gram_tma_launch<T, 12, NY>(X, ldx, nx, Y, ldy, ny, n, out, part, counter, gate, mask, status, st);
}

}  // namespace

template <typename T>
bool launch_gram_tma(const T* X, size_t ldx, int nx, const T* Y, size_t ldy, int ny, size_t n, double* out,
                     double* part, unsigned* counter, const int* gate, int mask, int* status, cudaStream_t st) {
  constexpr int VEC = 16 / (int)sizeof(T);
  const bool aligned = ((uintptr_t)X % 16 == 0) && ((uintptr_t)Y % 16 == 0) && (ldx % VEC == 0) && (ldy % VEC == 0);
  if (!aligned || nx < 1 || nx > MOTO_MAX_BASIS || ny < 1 || ny > 8) return false;
  if (ny <= 1)
    gram_tma_rows<T, 1>(X, ldx, nx, Y, ldy, ny, n, out, part, counter, gate, mask, status, st);
  else if (ny <= 2)
    gram_tma_rows<T, 2>(X, ldx, nx, Y, ldy, ny, n, out, part, counter, gate, mask, status, st);
  else if (ny <= 4)
    gram_tma_rows<T, 4>(X, ldx, nx, Y, ldy, ny, n, out, part, counter, gate, mask, status, st);
  else
    gram_tma_rows<T, 8>(X, ldx, nx, Y, ldy, ny, n, out, part, counter, gate, mask, status, st);
  return true;
}

template bool launch_gram_tma<float>(const float*, size_t, int, const float*, size_t, int, size_t, double*, double*,
                                     unsigned*, const int*, int, int*, cudaStream_t);
template bool launch_gram_tma<double>(const double*, size_t, int, const double*, size_t, int, size_t, double*,
                                      double*, unsigned*, const int*, int, int*, cudaStream_t);

}  // namespace moto
