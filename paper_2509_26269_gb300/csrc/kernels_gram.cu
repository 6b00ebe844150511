// Skinny Gram product out[r][c] = X_r . Y_c  (nx <= 96 rows, ny <= 8 columns,
// n elements), the reorthogonalisation and Rayleigh-Ritz workhorse of the
// Krylov solvers.  HBM-bound: every element of the nx + ny fields is read once.
//
// Pipeline: one persistent block per SM walks a contiguous range of element
// tiles.  The fields of X (and of Y) are equally strided, so each operand is a
// 2D tensor (elements x fields) and one TMA instruction
// (cp.async.bulk.tensor.2d) moves a whole [fields][KT] tile into shared
// memory, completed on an mbarrier by transaction bytes; elements past n are
// zero-filled by the TMA unit.  A 4-stage ring keeps ~150 KB in flight per SM.
// Warp w owns rows [R w, R w + R), lane l owns elements l, l + 32, ...; each
// lane keeps an R x NY block of FP32 partial sums in registers, flushed every
// kFlush tiles by a warp reduction into FP64 accumulators in shared memory.
// Block results go to FP64 partials reduced in block order by the last block.
#include <cuda.h>
#include <cudaTypedefs.h>

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

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
      "[%4];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
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

constexpr int kStages = 4;
constexpr int kTileBytes = 512;  // bytes of one field row in a tile
constexpr int kFlush = 8;        // tiles between FP32 -> FP64 flushes

}  // namespace

template <typename T, int R, int NY>
__global__ void __launch_bounds__(256) gram_tma_kernel(const __grid_constant__ CUtensorMap tmX,
                                                          const __grid_constant__ CUtensorMap tmY, int nx, int ny,
                                                          size_t n, double* out, double* part, unsigned* counter,
                                                          const int* gate, int mask, int* status) {
  if (gate && (*gate & mask)) return;
  constexpr int KT = kTileBytes / (int)sizeof(T);
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t full[kStages];
  __shared__ double facc[MOTO_MAX_BASIS * 8];
  __shared__ int timed_out;
  const int rows = nx + ny;
  // stage s: X tile [nx][KT] then Y tile [ny][KT]; stage stride rounded up to 1 KB
  const size_t stage_bytes = ((size_t)rows * kTileBytes + 1023) / 1024 * 1024;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int r0 = w * R;

  const size_t ntiles = (n + KT - 1) / KT;
  const size_t t_begin = ntiles * blockIdx.x / gridDim.x;
  const size_t t_end = ntiles * (blockIdx.x + 1) / gridDim.x;
  const unsigned tx_bytes = (unsigned)rows * kTileBytes;

  for (int i = threadIdx.x; i < nx * ny; i += blockDim.x) facc[i] = 0.0;
  if (threadIdx.x == 0) {
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmX)) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmY)) : "memory");
    for (int s = 0; s < kStages; ++s) mbar_init(&full[s], 1);
    timed_out = 0;
    fence_async_shared();
  }
  __syncthreads();

  auto issue = [&](size_t t, int s) {  // thread 0 only
    unsigned char* buf = smem + (size_t)s * stage_bytes;
    fence_async_shared();
    mbar_expect_tx(&full[s], tx_bytes);
    const int x = (int)(t * KT);
    tma_load_2d(buf, &tmX, x, 0, &full[s]);
    tma_load_2d(buf + (size_t)nx * kTileBytes, &tmY, x, 0, &full[s]);
  };

  if (threadIdx.x == 0)
    for (int s = 0; s < kStages; ++s)
      if (t_begin + s < t_end) issue(t_begin + s, s);

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
    const T* buf = reinterpret_cast<const T*>(smem + (size_t)s * stage_bytes);
    const T* Ys = buf + (size_t)nx * KT;
    if (r0 < nx) {
#pragma unroll
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
      if (++since == kFlush) {
        since = 0;
        flush();
      }
    }
    __syncthreads();  // every warp is done with stage s
    if (threadIdx.x == 0 && t + kStages < t_end) issue(t + kStages, s);
  }
  if (r0 < nx) flush();
  __syncthreads();
  if (timed_out) {
    // bounded drain: let tensor copies still in flight land before the block
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

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

// 2D map over `rows` fields of n elements, field stride ld elements; box
// [rows][KT].
template <typename T>
bool make_map(CUtensorMap* map, const T* base, size_t n, int rows, size_t ld) {
  auto fn = encode_fn();
  if (!fn) return false;
  constexpr int KT = kTileBytes / (int)sizeof(T);
  cuuint64_t dims[2] = {(cuuint64_t)n, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)(ld * sizeof(T))};
  cuuint32_t box[2] = {(cuuint32_t)KT, (cuuint32_t)rows};
  cuuint32_t estr[2] = {1, 1};
  const CUtensorMapDataType dt = sizeof(T) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64;
  return fn(map, dt, 2, const_cast<T*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
         CUDA_SUCCESS;
}

template <typename T, int R, int NY>
void gram_tma_launch(const CUtensorMap& mx, const CUtensorMap& my, int nx, int ny, size_t n, double* out,
                     double* part, unsigned* counter, const int* gate, int mask, int* status, cudaStream_t st) {
  constexpr int KT = kTileBytes / (int)sizeof(T);
  const size_t stage_bytes = ((size_t)(nx + ny) * kTileBytes + 1023) / 1024 * 1024;
  const size_t smem = kStages * stage_bytes;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(gram_tma_kernel<T, R, NY>, cudaFuncAttributeMaxDynamicSharedMemorySize, 216 * 1024);
    attr = true;
  }
  // as many resident blocks per SM as registers and shared memory allow: the
  // small-row shapes are latency-bound with a single block of 8 warps
  static int per_sm[MOTO_MAX_BASIS + 9] = {0};
  const int key = nx + ny;
  if (!per_sm[key]) {
    int b = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, gram_tma_kernel<T, R, NY>, 256, smem) != cudaSuccess ||
        b < 1)
      b = 1;
    per_sm[key] = b < 8 ? b : 8;
  }
  const size_t ntiles = (n + KT - 1) / KT;
  size_t want = (size_t)kSMs * per_sm[key];
  // every context holds at least kStreamBlocks * MOTO_MAX_BASIS * MOTO_MAX_K
  // partial sums; keep grid * nx * ny within that
  const size_t cap = (size_t)kStreamBlocks * MOTO_MAX_BASIS * MOTO_MAX_K / ((size_t)nx * ny);
  if (want > cap) want = cap;
  const int grid = (int)(ntiles < want ? (ntiles > 0 ? ntiles : 1) : want);
  gram_tma_kernel<T, R, NY><<<grid, 256, smem, st>>>(mx, my, nx, ny, n, out, part, counter, gate, mask, status);
}

template <typename T, int NY>
void gram_tma_rows(const CUtensorMap& mx, const CUtensorMap& my, int nx, int ny, size_t n, double* out,
                   double* part, unsigned* counter, const int* gate, int mask, int* status, cudaStream_t st) {
  const int r = (nx + 7) / 8;
  if (r <= 1)
    gram_tma_launch<T, 1, NY>(mx, my, nx, ny, n, out, part, counter, gate, mask, status, st);
  else if (r <= 2)
    gram_tma_launch<T, 2, NY>(mx, my, nx, ny, n, out, part, counter, gate, mask, status, st);
  else if (r <= 4)
    gram_tma_launch<T, 4, NY>(mx, my, nx, ny, n, out, part, counter, gate, mask, status, st);
  else if (r <= 8)
    gram_tma_launch<T, 8, NY>(mx, my, nx, ny, n, out, part, counter, gate, mask, status, st);
  else
    gram_tma_launch<T, 12, NY>(mx, my, nx, ny, n, out, part, counter, gate, mask, status, st);
}

}  // namespace

template <typename T>
bool launch_gram_tma(const T* X, size_t ldx, int nx, const T* Y, size_t ldy, int ny, size_t n, double* out,
                     double* part, unsigned* counter, const int* gate, int mask, int* status, cudaStream_t st) {
  // TMA: 16 B-aligned bases and strides, box dims <= 256, 4 stages fit in
  // shared memory
  const bool aligned = ((uintptr_t)X % 16 == 0) && ((uintptr_t)Y % 16 == 0) && ((ldx * sizeof(T)) % 16 == 0) &&
                       ((ldy * sizeof(T)) % 16 == 0);
  if (!aligned || nx < 1 || nx > MOTO_MAX_BASIS || ny < 1 || ny > 8 || n >= (1ull << 31)) return false;
  CUtensorMap mx, my;
  if (!make_map<T>(&mx, X, n, nx, ldx) || !make_map<T>(&my, Y, n, ny, ldy)) return false;
  if (ny <= 1)
    gram_tma_rows<T, 1>(mx, my, nx, ny, n, out, part, counter, gate, mask, status, st);
  else if (ny <= 2)
    gram_tma_rows<T, 2>(mx, my, nx, ny, n, out, part, counter, gate, mask, status, st);
  else if (ny <= 4)
    gram_tma_rows<T, 4>(mx, my, nx, ny, n, out, part, counter, gate, mask, status, st);
  else
    gram_tma_rows<T, 8>(mx, my, nx, ny, n, out, part, counter, gate, mask, status, st);
  return true;
}

template bool launch_gram_tma<float>(const float*, size_t, int, const float*, size_t, int, size_t, double*, double*,
                                     unsigned*, const int*, int, int*, cudaStream_t);
template bool launch_gram_tma<double>(const double*, size_t, int, const double*, size_t, int, size_t, double*,
                                      double*, unsigned*, const int*, int, int*, cudaStream_t);

}  // namespace moto
