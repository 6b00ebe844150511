// Streaming kernels of the block-Krylov reorthogonalisation over element
// tiles.  The fields of X (nx <= 96) and of Y (ny <= 8) are equally strided, so
// each operand is a 2D tensor [fields][n]; one TMA instruction
// (cp.async.bulk.tensor.2d) moves a [fields][KT] tile of 512-byte rows into
// shared memory, completed on an mbarrier by transaction bytes; the TMA unit
// zero-fills elements past n.  Modes:
//
//   0 (kGram)    : out = X^T Y
//   1 (kUpdGram) : Y <- Y - X C, then out = X^T Y      (CGS pass + next Gram)
//   2 (kUpdSelf) : Y <- Y - X C, then out = Y^T Y      (CGS pass + Cholesky Gram)
//   3 (kMulSelf) : Z <- X C,     then out = Z^T Z      (Cholesky QR step)
//
// C is nx x ny (FP64 in global memory, FP32/FP64 in shared memory).  Updated
// fields are written back with coalesced stores and reused from shared memory
// by the Gram phase: every field crosses HBM once per launch.
//
// 512 threads (16 warps).  Update phase: thread -> (element e, 4 columns),
// loop over the nx rows with one shared load of X and one broadcast 16-byte
// load of C per row.  Gram phase: warp w owns R rows of A (X, or Y itself for
// modes 2/3), lane l owns 16 contiguous bytes of every row (one 16-byte shared
// load per row and column field), R x NY FP32 partial sums per lane flushed
// every kFlush tiles by a warp reduction into FP64 (all FP64 for double).
// Block partials in FP64 are reduced in block order by the last block.  A
// 3-stage TMA ring with bounded waits (timeouts are reported, never hung).
#include <cuda.h>
#include <cudaTypedefs.h>

#include "internal.h"
#include "tma.cuh"

namespace moto {

using namespace tma;

namespace {
constexpr int kStagesT = 3;
constexpr int kRowB = 512;  // bytes of one field row of a tile
constexpr int kFlushT = 8;
constexpr int kPrefetch = 6;  // tiles prefetched into L2 ahead of the shared-memory ring
constexpr int kWarps = 12;  // consumer warps; with the producer warp at most 4 warps share a scheduler, so 128 registers each
constexpr int kThr = 32 * kWarps;

// OR-vote of `pred` over the kThr consumer threads (named barrier 2); a set
// abort flag counts as a vote.
__device__ __forceinline__ int __syncthreads_or_consumers(int pred, int abort_flag) {
  int r;
  pred = (pred || abort_flag) ? 1 : 0;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.s32 p, %1, 0;\n bar.red.or.pred q, 2, %2, p;\n selp.s32 %0, 1, 0, q;\n}\n"
      : "=r"(r)
      : "r"(pred), "r"(kThr)
      : "memory");
  return r;
}

template <typename T>
struct V16;
template <>
struct V16<float> {
  typedef float4 type;
  static constexpr int n = 4;
};
template <>
struct V16<double> {
  typedef double2 type;
  static constexpr int n = 2;
};

template <typename T>
__device__ __forceinline__ T vget(const typename V16<T>::type& v, int i);
template <>
__device__ __forceinline__ float vget<float>(const float4& v, int i) {
  return i == 0 ? v.x : i == 1 ? v.y : i == 2 ? v.z : v.w;
}
template <>
__device__ __forceinline__ double vget<double>(const double2& v, int i) {
  return i == 0 ? v.x : v.y;
}
}  // namespace

template <typename T, int MODE, int R, int NY>
__global__ void __launch_bounds__(kThr + 32, 1) tile2d_kernel(const __grid_constant__ CUtensorMap tmX,
                                                              const __grid_constant__ CUtensorMap tmY, int nx, int ny,
                                                              size_t n, const double* __restrict__ C,
                                                              T* __restrict__ Yout, size_t ldo, double* out,
                                                              double* part, unsigned* counter, const int* gate,
                                                              int mask, int* status) {
  if (gate && (*gate & mask)) return;
  typedef typename V16<T>::type VT;
  constexpr int VN = V16<T>::n;
  constexpr int KT = kRowB / (int)sizeof(T);  // elements per row of a tile
  static_assert(KT == 32 * VN, "one 16-byte chunk per lane per row");
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t full[kStagesT];
  __shared__ __align__(8) uint64_t empty[kStagesT];
  __shared__ double facc[MOTO_MAX_BASIS * 8];
  __shared__ __align__(16) T Cs[MOTO_MAX_BASIS * 8];
  __shared__ int abort_flag;

  const int rows = nx + ny;
  const size_t stage_bytes = ((size_t)rows * kRowB + 1023) / 1024 * 1024;
  const unsigned tx_bytes = (unsigned)((MODE == 3 ? nx : rows) * kRowB);
  const int na = (MODE <= 1) ? nx : ny;  // Gram rows
  const int a_off = (MODE <= 1) ? 0 : nx;
  const int nout = na * ny;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const bool producer = (w == kWarps);
  const int r0 = w * R;

  const size_t ntiles = (n + KT - 1) / KT;
  const size_t t_begin = ntiles * blockIdx.x / gridDim.x;
  const size_t t_end = ntiles * (blockIdx.x + 1) / gridDim.x;

  for (int i = threadIdx.x; i < nout; i += blockDim.x) facc[i] = 0.0;
  if (MODE != 0)
    for (int i = threadIdx.x; i < nx * 8; i += blockDim.x) {
      const int r = i >> 3, c = i & 7;
      const double cf = c < ny ? C[r * ny + c] : 0.0;
      Cs[i] = (T)(MODE == 3 ? cf : -cf);
    }
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStagesT; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], kWarps);
    }
    abort_flag = 0;
    fence_async_shared();
  }
  __syncthreads();

  if (producer) {
    // ---- TMA producer warp: refill a stage once every consumer warp freed it
    if (lane == 0) {
      // warm L2 with the first tiles beyond the ring
      for (int p = 0; p < kPrefetch; ++p) {
        const size_t tp = t_begin + kStagesT + p;
        if (tp < t_end) {
          tma_prefetch_2d(&tmX, (int)(tp * KT), 0);
          if (MODE != 3) tma_prefetch_2d(&tmY, (int)(tp * KT), 0);
        }
      }
      for (size_t t = t_begin; t < t_end; ++t) {
        const int it = (int)(t - t_begin);
        const int s = it % kStagesT;
        if (it >= kStagesT && !mbar_wait(&empty[s], (unsigned)(((it / kStagesT) - 1) & 1))) {
          atomicExch(&abort_flag, 1);
          if (status) atomicOr(status, kStatusTimeout);
          break;
        }
        if (*(volatile int*)&abort_flag) break;
        unsigned char* buf = smem + (size_t)s * stage_bytes;
        fence_async_shared();
        mbar_expect_tx(&full[s], tx_bytes);
        const int x = (int)(t * KT);
        tma_load_2d(buf, &tmX, x, 0, &full[s]);
        if (MODE != 3) tma_load_2d(buf + (size_t)nx * kRowB, &tmY, x, 0, &full[s]);
        const size_t tp = t + kStagesT + kPrefetch;
        if (tp < t_end) {
          tma_prefetch_2d(&tmX, (int)(tp * KT), 0);
          if (MODE != 3) tma_prefetch_2d(&tmY, (int)(tp * KT), 0);
        }
      }
    }
  } else {
    // ---- consumer warps
    T acc[R][NY];
#pragma unroll
    for (int j = 0; j < R; ++j)
#pragma unroll
      for (int c = 0; c < NY; ++c) acc[j][c] = (T)0;
    auto flush = [&]() {
#pragma unroll
      for (int j = 0; j < R; ++j)
#pragma unroll
        for (int c = 0; c < NY; ++c) {
          T v = acc[j][c];
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
          if (lane == 0 && r0 + j < na && c < ny) facc[(r0 + j) * ny + c] += (double)v;
          acc[j][c] = (T)0;
        }
    };
    int since = 0;
    for (size_t t = t_begin; t < t_end; ++t) {
      const int it = (int)(t - t_begin);
      const int s = it % kStagesT;
      bool ok = mbar_wait(&full[s], (unsigned)((it / kStagesT) & 1));
      if (MODE != 0) {
        // consumers agree before the update phase (it is followed by a
        // consumer-wide barrier)
        ok = __syncthreads_or_consumers(!ok, abort_flag) == 0;
      } else if (!ok) {
        atomicExch(&abort_flag, 1);
        if (status) atomicOr(status, kStatusTimeout);
      }
      if (!ok || *(volatile int*)&abort_flag) break;
      T* buf = reinterpret_cast<T*>(smem + (size_t)s * stage_bytes);
      T* Ys = buf + (size_t)nx * KT;
      if (MODE != 0) {
        // update phase: thread -> element e, columns 4q .. 4q+3
        const int e = threadIdx.x % KT, q = threadIdx.x / KT;
        if (4 * q < ny && q < 2) {
          T v[4];
#pragma unroll
          for (int j = 0; j < 4; ++j)
            v[j] = (MODE == 3 || 4 * q + j >= ny) ? (T)0 : Ys[(size_t)(4 * q + j) * KT + e];
          const T* xc = buf + e;
          const T* cc = Cs + 4 * q;
#pragma unroll 4
          for (int r = 0; r < nx; ++r) {
            const T x = xc[(size_t)r * KT];
            v[0] += x * cc[r * 8];
            v[1] += x * cc[r * 8 + 1];
            v[2] += x * cc[r * 8 + 2];
            v[3] += x * cc[r * 8 + 3];
          }
          const size_t el = t * KT + e;
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const int c = 4 * q + j;
            if (c < ny) {
              Ys[(size_t)c * KT + e] = el < n ? v[j] : (T)0;
              if (el < n) Yout[(size_t)c * ldo + el] = v[j];
            }
          }
        }
        asm volatile("bar.sync 1, %0;" ::"r"(kThr) : "memory");  // consumers only
      }
      // Gram phase
      if (r0 < na) {
        const T* As = buf + (size_t)a_off * KT;
        VT y[NY];
#pragma unroll
        for (int c = 0; c < NY; ++c) {
          if (c < ny)
            y[c] = reinterpret_cast<const VT*>(Ys + (size_t)c * KT)[lane];
          else
            y[c] = VT();
        }
#pragma unroll
        for (int j = 0; j < R; ++j) {
          if (r0 + j < na) {
            const VT x = reinterpret_cast<const VT*>(As + (size_t)(r0 + j) * KT)[lane];
#pragma unroll
            for (int c = 0; c < NY; ++c) {
              T a = acc[j][c];
#pragma unroll
              for (int i = 0; i < VN; ++i) a += vget<T>(x, i) * vget<T>(y[c], i);
              acc[j][c] = a;
            }
          }
        }
        if (++since == kFlushT) {
          since = 0;
          flush();
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[s]);
    }
    if (r0 < na) flush();
  }
  __syncthreads();
  if (abort_flag) {
    // bounded drain: let tensor copies still in flight land before the block
    // exits (a phase that already completed returns at once)
    if (threadIdx.x == 0)
      for (int s = 0; s < kStagesT; ++s) {
        mbar_wait(&full[s], 0);
        mbar_wait(&full[s], 1);
      }
    __syncthreads();
  }
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

// 2D map over `rows` fields of n elements, field stride ld; box [rows][KT]
template <typename T>
bool make_map(CUtensorMap* map, const T* base, size_t n, int rows, size_t ld) {
  auto fn = encode_fn();
  if (!fn) return false;
  constexpr int KT = kRowB / (int)sizeof(T);
  cuuint64_t dims[2] = {(cuuint64_t)n, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)(ld * sizeof(T))};
  cuuint32_t box[2] = {(cuuint32_t)KT, (cuuint32_t)rows};
  cuuint32_t estr[2] = {1, 1};
  const CUtensorMapDataType dt = sizeof(T) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64;
  return fn(map, dt, 2, const_cast<T*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
         CUDA_SUCCESS;
}

template <typename T, int MODE, int R, int NY>
void tile_launch(const CUtensorMap& mx, const CUtensorMap& my, int nx, int ny, size_t n, const double* C, T* Yout,
                 size_t ldo, double* out, double* part, unsigned* counter, const int* gate, int mask, int* status,
                 cudaStream_t st) {
  constexpr int KT = kRowB / (int)sizeof(T);
  const size_t stage_bytes = ((size_t)(nx + ny) * kRowB + 1023) / 1024 * 1024;
  const size_t smem = kStagesT * stage_bytes;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(tile2d_kernel<T, MODE, R, NY>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr = true;
  }
  static int per_sm[MOTO_MAX_BASIS + 10] = {0};
  const int key = nx + ny;
  if (!per_sm[key]) {
    int b = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, tile2d_kernel<T, MODE, R, NY>, kThr + 32, smem) != cudaSuccess ||
        b < 1)
      b = 1;
    per_sm[key] = b < 4 ? b : 4;
  }
  const int na = MODE <= 1 ? nx : ny;
  size_t want = (size_t)kSMs * per_sm[key];
  const size_t cap = (size_t)kStreamBlocks * MOTO_MAX_BASIS * MOTO_MAX_K / ((size_t)na * ny);
  if (want > cap) want = cap;
  const size_t ntiles = (n + KT - 1) / KT;
  const int grid = (int)(ntiles < want ? (ntiles > 0 ? ntiles : 1) : want);
  tile2d_kernel<T, MODE, R, NY><<<grid, kThr + 32, smem, st>>>(mx, my, nx, ny, n, C, Yout, ldo, out, part, counter, gate,
                                                          mask, status);
}

template <typename T, int MODE>
void tile_dispatch(const CUtensorMap& mx, const CUtensorMap& my, int nx, int ny, size_t n, const double* C, T* Yout,
                   size_t ldo, double* out, double* part, unsigned* counter, const int* gate, int mask, int* status,
                   cudaStream_t st) {
  const int na = MODE <= 1 ? nx : ny;
  const int r = (na + kWarps - 1) / kWarps;
#define TL(RR, YY) tile_launch<T, MODE, RR, YY>(mx, my, nx, ny, n, C, Yout, ldo, out, part, counter, gate, mask, status, st)
#define TROWS(YY)      \
  if (r <= 1)          \
    TL(1, YY);         \
  else if (r <= 2)     \
    TL(2, YY);         \
  else if (r <= 4)     \
    TL(4, YY);         \
  else if (r <= 6)     \
    TL(6, YY);         \
  else                 \
    TL(8, YY);
  if (ny <= 1) {
    TROWS(1)
  } else if (ny <= 2) {
    TROWS(2)
  } else if (ny <= 4) {
    TROWS(4)
  } else {
    TROWS(8)
  }
#undef TROWS
#undef TL
}

}  // namespace

template <typename T>
bool launch_tile(int mode, const T* X, size_t ldx, int nx, const T* Y, size_t ldy, int ny, size_t n, const double* C,
                 T* Yout, size_t ldo, double* out, double* part, unsigned* counter, const int* gate, int mask,
                 int* status, cudaStream_t st) {
  auto al = [](const void* p) { return ((uintptr_t)p % 16) == 0; };
  if ((ldx * sizeof(T)) % 16 || (ldy * sizeof(T)) % 16 || !al(X) || (mode != 3 && !al(Y))) return false;
  if (mode != 0 && ((ldo * sizeof(T)) % 16 || !al(Yout))) return false;
  if (nx < 1 || nx > MOTO_MAX_BASIS || ny < 1 || ny > 8 || n >= (1ull << 31)) return false;
  CUtensorMap mx, my;
  if (!make_map<T>(&mx, X, n, nx, ldx)) return false;
  if (mode != 3) {
    if (!make_map<T>(&my, Y, n, ny, ldy)) return false;
  } else {
    my = mx;
  }
  switch (mode) {
    case 0: tile_dispatch<T, 0>(mx, my, nx, ny, n, C, Yout, ldo, out, part, counter, gate, mask, status, st); break;
    case 1: tile_dispatch<T, 1>(mx, my, nx, ny, n, C, Yout, ldo, out, part, counter, gate, mask, status, st); break;
    case 2: tile_dispatch<T, 2>(mx, my, nx, ny, n, C, Yout, ldo, out, part, counter, gate, mask, status, st); break;
    default: tile_dispatch<T, 3>(mx, my, nx, ny, n, C, Yout, ldo, out, part, counter, gate, mask, status, st); break;
  }
  return true;
}

template bool launch_tile<float>(int, const float*, size_t, int, const float*, size_t, int, size_t, const double*,
                                 float*, size_t, double*, double*, unsigned*, const int*, int, int*, cudaStream_t);
template bool launch_tile<double>(int, const double*, size_t, int, const double*, size_t, int, size_t, const double*,
                                  double*, size_t, double*, double*, unsigned*, const int*, int, int*, cudaStream_t);

}  // namespace moto
