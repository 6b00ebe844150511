// Streaming kernels of the block-Krylov reorthogonalisation over element
// tiles.  The fields of X (nx <= 96) and of Y (ny <= 8) are equally strided, so
// each operand is a 2D tensor [fields][n].  A tile is TB bytes (256 to 1024) of
// every field, moved by one TMA load per operand (cp.async.bulk.tensor.2d,
// box [fields][TB]) into a dense [fields][TB] shared-memory stage; the TMA
// unit zero-fills elements past n.  Rows of at least 256 contiguous bytes keep
// the tensor copies at full HBM rate (128-byte rows, as a swizzled layout
// would need, stream at about two thirds of it), so bank conflicts are avoided
// in the reads instead: in the Gram phase lane l starts its walk over the
// 16-byte chunks of a row at chunk (l & 7), so the eight lanes of a quarter
// warp always touch eight different bank groups.  Modes:
//
//   0 (kGram)    : out = X^T Y
//   1 (kUpdGram) : Y <- Y - X[u0, u0 + nu) C, then out = X^T Y (the updated
//                  Y may stay unstored: the Gram reads it from the stage)
//   2 (kUpdSelf) : Y <- Y - X C, then out = Y^T Y (C may be the sum of two
//                  coefficient blocks, a local one added to some of its rows)
//   3 (kMulSelf) : Z <- X C,     then out = Z^T Z (Z may stay unstored)
//
// C is nu x ny (FP64 in global memory, T in shared memory).  Updated fields are
// written back with coalesced vector stores; in mode 1 they also replace Y in
// the staged tile, from where the Gram phase reads them, so every field crosses
// HBM once per launch.
//
// Warp pairs per tile: one producer warp keeps a ring of up to 32 stages
// full; each of the kPairs consumer warp pairs takes every kPairs-th tile of
// the block's contiguous range, and warp g of the pair works alone on half g
// of every row (update and Gram need only the elements they own, so the two
// warps never wait for each other; a stage is freed by their two mbarrier
// arrivals).  Two consumer warps share each scheduler and hide each other's
// latencies.  Gram layout (modes 0, 1): lane (rl, cl, ks) owns the outputs of
// rows rl + NRL i (i < R) and columns cl CW + j (j < CW) over every KS-th
// chunk of a tile (the KS lanes of an output are summed once, at the end);
// per 16-byte chunk it loads its R rows of X and CW rows of Y and multiplies
// them with packed FP32 FMAs (fma.rn.f32x2).  Update layout (modes
// 1-3): a lane owns TB / 64 bytes of the tile of all 8 columns and loops over
// the rows of X with one load of X and broadcast loads of the C row.  FP32
// partial sums are flushed every 512 elements of a lane's share into a second
// FP32 total (a lane sees a few thousand elements, so a few tens of flushes);
// lane, warp, block and grid totals are summed in a fixed order in two-float
// arithmetic (FP64 for FP64 fields), the block partials by the last block.
// All waits are bounded (timeouts are reported, never hung).
#include <algorithm>
#include <cuda.h>
#include <type_traits>
#include <cudaTypedefs.h>

#include "internal.h"
#include "tma.cuh"

namespace moto {

using namespace tma;

namespace {
// consumer warp pairs per block: with the producer 11 warps, at most three on
// one scheduler, so 168 registers a thread still fit its quarter of the
// register file (six pairs would put four warps on one scheduler and cap the
// threads at 128 registers)
constexpr int kPairs = 5;
constexpr int kConsumers = 2 * kPairs;
constexpr int kThrT = 32 * (kConsumers + 1);
#define MOTO_TILE_MAXREG 168
constexpr int kMaxStages = 32;
constexpr int kFlushE = 512;  // elements between flushes of the FP32 partial sums
constexpr int kSelf = 36;  // upper-triangle entries of an 8 x 8 Gram
constexpr size_t kDynBudget = 219 * 1024;  // dynamic shared memory of the ring (1 KB of it alignment slack)

__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) {
  unsigned long long d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;"
      : "=l"(d)
      : "l"(*reinterpret_cast<unsigned long long*>(&a)), "l"(*reinterpret_cast<unsigned long long*>(&b)),
        "l"(*reinterpret_cast<unsigned long long*>(&c)));
  return *reinterpret_cast<float2*>(&d);
}

__device__ __forceinline__ float4 lds128f(uint32_t a) {
  float4 v;
  asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(a));
  return v;
}
__device__ __forceinline__ double2 lds128d(uint32_t a) {
  double2 v;
  asm volatile("ld.shared.v2.f64 {%0, %1}, [%2];" : "=d"(v.x), "=d"(v.y) : "r"(a));
  return v;
}
__device__ __forceinline__ float2 lds64f(uint32_t a) {
  float2 v;
  asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(a));
  return v;
}
__device__ __forceinline__ double lds64d(uint32_t a) {
  double v;
  asm volatile("ld.shared.f64 %0, [%1];" : "=d"(v) : "r"(a));
  return v;
}

// The lane's EL elements of one row of a stage (EL x sizeof(T) = 4, 8 or 16
// bytes), as loads and stores.
template <typename T, int EL>
struct Lane {
  static __device__ __forceinline__ void load(uint32_t a, T (&v)[EL]) {
    if constexpr (sizeof(T) == 4 && EL == 1) {
      asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v[0]) : "r"(a));
    } else if constexpr (sizeof(T) == 4 && EL == 2) {
      const float2 x = lds64f(a);
      v[0] = x.x;
      v[EL - 1] = x.y;
    } else if constexpr (sizeof(T) == 4) {
      const float4 x = lds128f(a);
      v[0] = x.x;
      v[1 % EL] = x.y;
      v[2 % EL] = x.z;
      v[3 % EL] = x.w;
    } else if constexpr (EL == 1) {
      v[0] = lds64d(a);
    } else {
      const double2 x = lds128d(a);
      v[0] = x.x;
      v[EL - 1] = x.y;
    }
  }
  static __device__ __forceinline__ void store_smem(uint32_t a, const T (&v)[EL]) {
    if constexpr (sizeof(T) == 4 && EL == 1) {
      asm volatile("st.shared.f32 [%0], %1;" ::"r"(a), "f"((float)v[0]) : "memory");
    } else if constexpr (sizeof(T) == 4 && EL == 2) {
      asm volatile("st.shared.v2.f32 [%0], {%1, %2};" ::"r"(a), "f"((float)v[0]), "f"((float)v[EL - 1]) : "memory");
    } else if constexpr (sizeof(T) == 4) {
      asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(a), "f"((float)v[0]), "f"((float)v[1 % EL]),
                   "f"((float)v[2 % EL]), "f"((float)v[3 % EL])
                   : "memory");
    } else if constexpr (EL == 1) {
      asm volatile("st.shared.f64 [%0], %1;" ::"r"(a), "d"((double)v[0]) : "memory");
    } else {
      asm volatile("st.shared.v2.f64 [%0], {%1, %2};" ::"r"(a), "d"((double)v[0]), "d"((double)v[EL - 1]) : "memory");
    }
  }
  // global store of elements el .. el + EL - 1 (those below n)
  static __device__ __forceinline__ void store_global(T* dst, size_t el, size_t n, const T (&v)[EL]) {
    if (el + EL <= n) {
      if constexpr (EL == 1) {
        *dst = v[0];
      } else if constexpr (sizeof(T) == 4 && EL == 2) {
        *reinterpret_cast<float2*>(dst) = make_float2((float)v[0], (float)v[EL - 1]);
      } else if constexpr (sizeof(T) == 4) {
        *reinterpret_cast<float4*>(dst) = make_float4((float)v[0], (float)v[1 % EL], (float)v[2 % EL], (float)v[3 % EL]);
      } else if constexpr (EL == 1) {
        *dst = v[0];
      } else {
        *reinterpret_cast<double2*>(dst) = make_double2((double)v[0], (double)v[EL - 1]);
      }
    } else {
#pragma unroll
      for (int e = 0; e < EL; ++e)
        if (el + e < n) dst[e] = v[e];
    }
  }
};

// Gram accumulation of one 16-byte chunk: acc[s][i][j] += <x_i, y_j>.  Each
// FP32 chunk is two packed FMAs; with few outputs per lane the two halves go
// to separate accumulator sets (NS = 2) to keep more independent chains.
template <int NS, int NR, int NC>
__device__ __forceinline__ void gram_chunk(float2 (&acc)[NS][NR][NC], const float4 (&x)[NR], const float4 (&y)[NC]) {
#pragma unroll
  for (int i = 0; i < NR; ++i)
#pragma unroll
    for (int j = 0; j < NC; ++j)
      acc[0][i][j] = ffma2(make_float2(x[i].x, x[i].y), make_float2(y[j].x, y[j].y), acc[0][i][j]);
#pragma unroll
  for (int i = 0; i < NR; ++i)
#pragma unroll
    for (int j = 0; j < NC; ++j)
      acc[NS - 1][i][j] = ffma2(make_float2(x[i].z, x[i].w), make_float2(y[j].z, y[j].w), acc[NS - 1][i][j]);
}
template <int NS, int NR, int NC>
__device__ __forceinline__ void gram_chunk(double (&acc)[NS][NR][NC], const double2 (&x)[NR], const double2 (&y)[NC]) {
#pragma unroll
  for (int i = 0; i < NR; ++i)
#pragma unroll
    for (int j = 0; j < NC; ++j) acc[0][i][j] = fma(x[i].x, y[j].x, acc[0][i][j]);
#pragma unroll
  for (int i = 0; i < NR; ++i)
#pragma unroll
    for (int j = 0; j < NC; ++j) acc[NS - 1][i][j] = fma(x[i].y, y[j].y, acc[NS - 1][i][j]);
}

template <typename T>
struct TileT;
template <>
struct TileT<float> {
  typedef float2 Acc;
  typedef float4 V16;
  static __device__ __forceinline__ Acc zero() { return make_float2(0.f, 0.f); }
  static __device__ __forceinline__ double to_d(const Acc& a) { return (double)a.x + (double)a.y; }
  static __device__ __forceinline__ float4 lds128(uint32_t a) { return lds128f(a); }
};
template <>
struct TileT<double> {
  typedef double Acc;
  typedef double2 V16;
  static __device__ __forceinline__ Acc zero() { return 0.0; }
  static __device__ __forceinline__ double to_d(const Acc& a) { return a; }
  static __device__ __forceinline__ double2 lds128(uint32_t a) { return lds128d(a); }
};

// Update of the lane's EL elements of the 8 columns: y += X[u0 .. u0 + nu) Cs
// (Cs rows of 8, padded with zeros past ny).  FP32 keeps column pairs,
// p[q][e] = (column 2q, column 2q + 1) of element e, for packed FMAs.
template <int EL, int TB>
__device__ __forceinline__ void update_rows(float2 (&p)[4][EL], uint32_t xa, int u0, int nu, const float* Cs) {
#pragma unroll 4
  for (int r = 0; r < nu; ++r) {
    float xe[EL];
    Lane<float, EL>::load(xa + (uint32_t)(u0 + r) * TB, xe);
    const float4 c0 = *reinterpret_cast<const float4*>(Cs + r * 8);
    const float4 c1 = *reinterpret_cast<const float4*>(Cs + r * 8 + 4);
#pragma unroll
    for (int e = 0; e < EL; ++e) {
      const float2 xx = make_float2(xe[e], xe[e]);
      p[0][e] = ffma2(xx, make_float2(c0.x, c0.y), p[0][e]);
      p[1][e] = ffma2(xx, make_float2(c0.z, c0.w), p[1][e]);
      p[2][e] = ffma2(xx, make_float2(c1.x, c1.y), p[2][e]);
      p[3][e] = ffma2(xx, make_float2(c1.z, c1.w), p[3][e]);
    }
  }
}

template <int EL, int TB>
__device__ __forceinline__ void update_rows_d(double (&y)[8][EL], uint32_t xa, int u0, int nu, const double* Cs) {
#pragma unroll 2
  for (int r = 0; r < nu; ++r) {
    double xe[EL];
    Lane<double, EL>::load(xa + (uint32_t)(u0 + r) * TB, xe);
    const double2* cr = reinterpret_cast<const double2*>(Cs + r * 8);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const double2 c = cr[q];
#pragma unroll
      for (int e = 0; e < EL; ++e) {
        y[2 * q][e] = fma(xe[e], c.x, y[2 * q][e]);
        y[2 * q + 1][e] = fma(xe[e], c.y, y[2 * q + 1][e]);
      }
    }
  }
}

}  // namespace

template <typename T, int MODE, int R, int CW, int NRL, int TB>
__global__ void __maxnreg__(MOTO_TILE_MAXREG)
    tile2d_kernel(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmY, int nx, int ny,
                  int u0, int nu, size_t n, const double* __restrict__ C, const double* __restrict__ Cadd, int uadd,
                  int nadd, T* __restrict__ Yout, size_t ldo, double* out, double* part, unsigned* counter, int nst,
                  int tps, const int* gate, int mask, int* status, int polls, size_t ws) {
  // walker batches: tensor coordinate z = walker, the other pointers offset
  C = wofs(C, ws);
  Cadd = wofs(Cadd, ws);
  Yout = wofs(Yout, ws);
  out = wofs(out, ws);
  part = wofs(part, ws);
  counter = wofs(counter, ws);
  gate = wofs(gate, ws);
  status = wofs(status, ws);
  const int wz = ws ? (int)blockIdx.z : -1;
  if (gate && (*gate & mask)) return;
  typedef TileT<T> TT;
  typedef typename TT::Acc Acc;
  typedef typename TT::V16 VT;
  constexpr int TE = TB / (int)sizeof(T);  // elements of a tile
  constexpr int HB = TB / 2;  // bytes of a row a warp of the pair owns
  constexpr int EL = TE / 64;  // elements of a lane in the update layout
  constexpr int NCH = HB / 16;  // 16-byte chunks of a half row
  static_assert(EL == 1 || EL == 2 || (EL == 4 && MODE <= 2), "a lane owns 4 to 16 bytes of a row");
  static_assert(EL * (int)sizeof(T) >= 4 && EL * (int)sizeof(T) <= 16, "lane share");
  constexpr bool kGramMode = (MODE <= 1);
  constexpr bool kF32 = sizeof(T) == 4;
  constexpr int NR = kGramMode ? R : 1, NC = kGramMode ? CW : 1;
  // Gram layout: NRL row lanes x NCG column groups, the remaining lanes split
  // the chunks of a tile (KS lanes per output, summed at the end)
  constexpr int NCG = 8 / CW, KS = 32 / (NRL * NCG);
  static_assert(KS >= 1 && NRL * NCG * KS == 32, "Gram lane layout");
  static_assert(NRL * NCG >= 8, "the KS lanes of an output share their chunk skew (lane & 7)");
  constexpr int NS = (kF32 && NR * NC <= 8) ? 2 : 1;  // accumulator sets
  constexpr int ND = kGramMode ? (kF32 ? NR * NC : 1) : kSelf;  // FP64 totals
  constexpr int kFlushT = kFlushE / (TE / 2);
  extern __shared__ unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t full[kMaxStages];
  __shared__ __align__(8) uint64_t empty[kMaxStages];
  __shared__ int tile_of[kMaxStages];  // tile of the stage's latest fill
  __shared__ __align__(16) T Cs[MOTO_MAX_BASIS * 8];
  __shared__ int abort_flag;

  // ring base, 1024-byte aligned
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t ring = (raw + 1023u) & ~1023u;
  unsigned char* ring_ptr = smem_raw + (ring - raw);
  const int nxp = (nx + 7) & ~7;
  const uint32_t yoff = (uint32_t)nxp * TB;
  const uint32_t tile_b = yoff + (MODE == 3 ? 0u : 8u * TB);  // one tile of a stage
  const uint32_t stage_bytes = (uint32_t)tps * tile_b;
  const unsigned tx_bytes = (unsigned)(tps * (nx + (MODE == 3 ? 0 : ny)) * TB);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int na = kGramMode ? nx : ny;

  // stage groups (tps tiles each) interleaved over the blocks: group g goes
  // to block g mod gridDim.x, so the blocks stream neighbouring tiles of each
  // field at the same time (DRAM pages are shared between SMs rather than
  // opened for one 256-byte row each); tiles past the end of the fields read
  // zeros and store nothing
  const size_t ngroups = ((n + TE - 1) / TE + tps - 1) / tps;
  const int ntile = (int)(ngroups > blockIdx.x ? (ngroups - blockIdx.x + gridDim.x - 1) / gridDim.x : 0);

  if (MODE != 0)
    for (int i = threadIdx.x; i < nu * 8; i += blockDim.x) {
      const int r = i >> 3, c = i & 7;
      double cf = c < ny ? C[r * ny + c] : 0.0;
      if (Cadd && c < ny && r >= uadd && r < uadd + nadd) cf += Cadd[(r - uadd) * ny + c];
      Cs[i] = (T)(MODE == 3 ? cf : -cf);
    }
  if (threadIdx.x == 0) {
    for (int s = 0; s < nst; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 2);
      tile_of[s] = -1;
    }
    abort_flag = 0;
    fence_async_shared();
  }
  __syncthreads();

  // FP64 totals of the lane's outputs (Gram layout, FP32) or of the self-Gram
  // entries (update layout)
  // FP32 fields: a second FP32 level collects the flushed partial sums (a
  // lane sees at most a few tens of flushes); FP64 fields accumulate here
  typedef typename std::conditional<kF32, float, double>::type DT;
  DT dacc[ND];
#pragma unroll
  for (int i = 0; i < ND; ++i) dacc[i] = (DT)0;
  Acc acc[NS][NR][NC];
#pragma unroll
  for (int s2 = 0; s2 < NS; ++s2)
#pragma unroll
    for (int i = 0; i < NR; ++i)
#pragma unroll
      for (int j = 0; j < NC; ++j) acc[s2][i][j] = TT::zero();

  if (w == kConsumers) {
    // ---- TMA producer: lane 0 refills a stage once its consumer freed it
    if (lane == 0) {
      for (int it = 0; it < ntile; ++it) {
        const int s = it % nst;
        if (it >= nst && !mbar_wait_or_abort(&empty[s], (unsigned)(((it / nst) - 1) & 1), &abort_flag)) {
          atomicExch(&abort_flag, 1);
          if (status) atomicOr(status, kStatusTimeout);
          break;
        }
        if (*(volatile int*)&abort_flag) break;
        unsigned char* buf = ring_ptr + (size_t)s * stage_bytes;
        *(volatile int*)&tile_of[s] = it;
        mbar_expect_tx(&full[s], tx_bytes);
        for (int q = 0; q < tps; ++q) {
          const int x = (int)(((blockIdx.x + (size_t)it * gridDim.x) * tps + q) * TE);
          if (wz < 0) {
            tma_load_2d(buf + (size_t)q * tile_b, &tmX, x, 0, &full[s]);
            if (MODE != 3) tma_load_2d(buf + (size_t)q * tile_b + yoff, &tmY, x, 0, &full[s]);
          } else {
            tma_load_3d(buf + (size_t)q * tile_b, &tmX, x, 0, wz, &full[s]);
            if (MODE != 3) tma_load_3d(buf + (size_t)q * tile_b + yoff, &tmY, x, 0, wz, &full[s]);
          }
        }
      }
    }
  } else {
    // ---- consumer warp w: pair pw, half g of the rows; tiles it = pw, pw + kPairs, ...
    // Gram layout: byte offsets of the lane's rows, chunk skew
    uint32_t xrow[NR], yrow[NC];
    {
      const int rl = lane % NRL, cl = (lane / NRL) % NCG;
#pragma unroll
      for (int i = 0; i < NR; ++i) xrow[i] = (uint32_t)min(rl + NRL * i, na - 1) * TB;
#pragma unroll
      for (int j = 0; j < NC; ++j) yrow[j] = yoff + (uint32_t)min(cl * CW + j, ny - 1) * TB;
    }
    const int skew = lane & 7;
    const int ks = lane / (NRL * NCG);  // the lane's share of the chunks
    float sacc[(MODE >= 2 && kF32) ? kSelf : 1];
#pragma unroll
    for (int i = 0; i < ((MODE >= 2 && kF32) ? kSelf : 1); ++i) sacc[i] = 0.f;
    const int pw = w >> 1, g = w & 1;
    const uint32_t hoff = (uint32_t)g * HB;
    const uint32_t lane_b = hoff + (uint32_t)lane * EL * sizeof(T);  // update layout: the lane's bytes of a row
    int since = 0;
    // When the ring has a multiple of kPairs stages a stage always goes to the
    // same pair, whose previous fill of it the pair itself consumed, so the
    // parity wait cannot confuse fills.  Otherwise a pair may reach a stage two
    // fills ahead of the producer: it first waits until the producer has
    // started the fill of its own tile (which happens only after the previous
    // fill was consumed), which makes the parity wait unambiguous.
    const bool shared_stages = (nst % kPairs) != 0;
    for (int it = pw; it < ntile; it += kPairs) {
      const int s = it % nst;
      if (shared_stages) {
        int spins = 0;
        while (*(volatile int*)&tile_of[s] != it && !*(volatile int*)&abort_flag && ++spins < (1 << 22))
          __nanosleep(32);
        if (spins >= (1 << 22)) {
          atomicExch(&abort_flag, 1);
          if (status) atomicOr(status, kStatusTimeout);
        }
      }
      if (*(volatile int*)&abort_flag) break;
      if (!(polls > 0 ? mbar_test_n(&full[s], (unsigned)((it / nst) & 1), polls)
                      : mbar_wait(&full[s], (unsigned)((it / nst) & 1)))) {
        atomicExch(&abort_flag, 1);
        if (status) atomicOr(status, kStatusTimeout);
      }
      if (*(volatile int*)&abort_flag) break;
      for (int qt = 0; qt < tps; ++qt) {
      const uint32_t sb = ring + (uint32_t)s * stage_bytes + (uint32_t)qt * tile_b;
      if (MODE != 0) {
        const uint32_t xa = sb + lane_b, ya = sb + yoff + lane_b;
        const size_t el =
            ((blockIdx.x + (size_t)it * gridDim.x) * tps + qt) * TE + (size_t)g * (TE / 2) + (size_t)lane * EL;
        T yv[8][EL];
        if constexpr (kF32) {
          float2 p[4][EL];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            float a[EL], b[EL];
#pragma unroll
            for (int e = 0; e < EL; ++e) a[e] = b[e] = 0.f;
            if (MODE != 3) {
              if (2 * q < ny) Lane<float, EL>::load(ya + (uint32_t)(2 * q) * TB, a);
              if (2 * q + 1 < ny) Lane<float, EL>::load(ya + (uint32_t)(2 * q + 1) * TB, b);
            }
#pragma unroll
            for (int e = 0; e < EL; ++e) p[q][e] = make_float2(a[e], b[e]);
          }
          update_rows<EL, TB>(p, xa, MODE == 1 ? u0 : 0, nu, reinterpret_cast<const float*>(Cs));
#pragma unroll
          for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int e = 0; e < EL; ++e) {
              yv[2 * q][e] = p[q][e].x;
              yv[2 * q + 1][e] = p[q][e].y;
            }
        } else {
          double y[8][EL];
#pragma unroll
          for (int c = 0; c < 8; ++c) {
#pragma unroll
            for (int e = 0; e < EL; ++e) y[c][e] = 0.0;
            if (MODE != 3 && c < ny) Lane<double, EL>::load(ya + (uint32_t)c * TB, y[c]);
          }
          update_rows_d<EL, TB>(y, xa, MODE == 1 ? u0 : 0, nu, reinterpret_cast<const double*>(Cs));
#pragma unroll
          for (int c = 0; c < 8; ++c)
#pragma unroll
            for (int e = 0; e < EL; ++e) yv[c][e] = y[c][e];
        }
        // write back (and, in mode 1, into the staged tile for the Gram phase)
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          if (c < ny) {
            if (MODE == 2 || Yout) Lane<T, EL>::store_global(Yout + (size_t)c * ldo + el, el, n, yv[c]);
            if (MODE == 1) Lane<T, EL>::store_smem(ya + (uint32_t)c * TB, yv[c]);
          }
        }
        if constexpr (MODE >= 2) {
          // self Gram of the updated columns (elements past n are zero)
          int q = 0;
#pragma unroll
          for (int c1 = 0; c1 < 8; ++c1)
#pragma unroll
            for (int c2 = c1; c2 < 8; ++c2, ++q) {
              if constexpr (kF32) {
                float a = sacc[q];
#pragma unroll
                for (int e = 0; e < EL; ++e) a = fmaf((float)yv[c1][e], (float)yv[c2][e], a);
                sacc[q] = a;
              } else {
#pragma unroll
                for (int e = 0; e < EL; ++e) dacc[q] = fma((double)yv[c1][e], (double)yv[c2][e], dacc[q]);
              }
            }
        }
        if (MODE == 1) __syncwarp();
      }
      if constexpr (kGramMode) {
        // Gram phase: acc[.][i][j] += <X row i, Y row j> over the lane's
        // chunks of the tile (every KS-th), its walk starting at chunk `skew`
        // (the KS lanes of an output share the skew, so together they cover
        // every chunk once)
#pragma unroll 8
        for (int k = ks; k < NCH; k += KS) {
          const uint32_t co = sb + hoff + (uint32_t)(((k + skew) & (NCH - 1)) << 4);
          VT xv[NR], yw[NC];
#pragma unroll
          for (int i = 0; i < NR; ++i) xv[i] = TT::lds128(co + xrow[i]);
#pragma unroll
          for (int j = 0; j < NC; ++j) yw[j] = TT::lds128(co + yrow[j]);
          gram_chunk<NS, NR, NC>(acc, xv, yw);
        }
      }
      if (kF32 && ++since == kFlushT) {
        since = 0;
        if constexpr (kGramMode && kF32) {
#pragma unroll
          for (int i = 0; i < NR; ++i)
#pragma unroll
            for (int j = 0; j < NC; ++j) {
              DT a = (DT)acc[0][i][j].x + (DT)acc[0][i][j].y;
              if (NS == 2) a += (DT)acc[NS - 1][i][j].x + (DT)acc[NS - 1][i][j].y;
              dacc[i * NC + j] += a;
              acc[0][i][j] = TT::zero();
              acc[NS - 1][i][j] = TT::zero();
            }
        } else if constexpr (MODE >= 2 && kF32) {
#pragma unroll
          for (int q = 0; q < kSelf; ++q) {
            dacc[q] += (DT)sacc[q];
            sacc[q] = 0.f;
          }
        }
      }
      }  // tiles of the stage
      // free the stage; the generic-proxy writes of mode 1 are ordered before
      // the next tensor copy into it
      if (MODE == 1) fence_async_shared();
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[s]);
    }
    if constexpr (MODE >= 2 && kF32) {
#pragma unroll
      for (int q = 0; q < kSelf; ++q) dacc[q] += (DT)sacc[q];
    }
  }
  __syncthreads();
  if (abort_flag) {
    // bounded drain (full bound): the last fill issued into a stage (tile
    // tile_of[s], the stage's fill number tile_of[s] / nst) must land before
    // the ring is reused; earlier fills of the stage were consumed, so they
    // landed, and a fill that already landed returns at once
    if (threadIdx.x == 0)
      for (int s = 0; s < nst; ++s) {
        const int t = *(volatile int*)&tile_of[s];
        if (t >= 0) mbar_wait(&full[s], (unsigned)((t / nst) & 1));
      }
    __syncthreads();
  }
  // Sums in a fixed order: lane totals -> warp -> block partial -> grid
  // total.  FP32 fields sum in two-float arithmetic (RT = F2), FP64 fields in
  // FP64; block partials go to `part` as 8-byte RT values.
  typedef typename std::conditional<kF32, F2, double>::type RT;
  const int nout = na * ny;
  RT* red = reinterpret_cast<RT*>(ring_ptr);  // the ring is idle now
  RT* rpart = reinterpret_cast<RT*>(part) + (size_t)blockIdx.x * nout;
  if constexpr (kGramMode) {
    // per-warp partials, then the block partial over the warps in order
    if (w < kConsumers) {
      RT* rw = red + (size_t)w * nout;
      const int rl = lane % NRL, cl = (lane / NRL) % NCG, ks = lane / (NRL * NCG);
#pragma unroll
      for (int i = 0; i < NR; ++i)
#pragma unroll
        for (int j = 0; j < NC; ++j) {
          const int r = rl + NRL * i, c = cl * CW + j;
          RT v;
          if constexpr (kF32) {
            v = f2_of(dacc[i * NC + j]);
#pragma unroll
            for (int s2 = 0; s2 < NS; ++s2) {
              v = radd(v, f2_of(acc[s2][i][j].x));
              v = radd(v, f2_of(acc[s2][i][j].y));
            }
          } else {
            v = acc[0][i][j];
            if (NS == 2) v += acc[NS - 1][i][j];
          }
          // the KS lanes of an output, in a fixed order
#pragma unroll
          for (int o = NRL * NCG; o < 32; o <<= 1) v = radd(v, rshfl(v, o));
          if (ks == 0 && r < na && c < ny) rw[r * ny + c] = v;
        }
    }
    __syncthreads();
    for (int o = threadIdx.x; o < nout; o += blockDim.x) {
      RT a = red[o];
      for (int ww = 1; ww < kConsumers; ++ww) a = radd(a, red[(size_t)ww * nout + o]);
      rpart[o] = a;
    }
  } else {
    // update layout: every lane holds all kSelf entries.  Lane values go to
    // shared memory; thread (entry, chunk) adds a chunk of kChunkLanes lanes,
    // then one thread per entry adds the chunks (no cross-lane shuffles)
    constexpr int kLanes = kConsumers * 32, kChunkLanes = 40, kChunks = kLanes / kChunkLanes;
    static_assert(kChunks * kChunkLanes == kLanes && kChunks * kSelf <= kThrT, "self-Gram block sum layout");
    RT* lv = red;                       // [kLanes][kSelf]
    RT* cs = red + (size_t)kLanes * kSelf;  // [kChunks][kSelf]
    if (w < kConsumers)
#pragma unroll
      for (int q = 0; q < kSelf; ++q) {
        if constexpr (kF32)
          lv[(size_t)(w * 32 + lane) * kSelf + q] = f2_of(dacc[q]);
        else
          lv[(size_t)(w * 32 + lane) * kSelf + q] = dacc[q];
      }
    __syncthreads();
    if (threadIdx.x < kChunks * kSelf) {
      const int q = threadIdx.x % kSelf, ch = threadIdx.x / kSelf;
      const RT* src = lv + (size_t)ch * kChunkLanes * kSelf + q;
      RT a = src[0];
      for (int l = 1; l < kChunkLanes; ++l) a = radd(a, src[(size_t)l * kSelf]);
      cs[ch * kSelf + q] = a;
    }
    __syncthreads();
    if (threadIdx.x < kSelf) {
      const int q = threadIdx.x;
      RT a = cs[q];
      for (int ch = 1; ch < kChunks; ++ch) a = radd(a, cs[ch * kSelf + q]);
      int c1 = 0, rem = q;
      while (rem >= 8 - c1) {
        rem -= 8 - c1;
        ++c1;
      }
      const int c2 = c1 + rem;
      if (c2 < ny) {
        rpart[c1 * ny + c2] = a;
        rpart[c2 * ny + c1] = a;
      }
    }
  }
  if (!grid_last_block(counter)) return;
  if constexpr (kF32)
    grid_sum_f2(reinterpret_cast<const F2*>(part), gridDim.x, nout, out, red);
  else
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

// 2D map over `rows` fields of n elements, field stride ld; box [rows][TB
// bytes], no swizzle.  For a walker batch (nw > 1) a 3D map whose third
// dimension steps from walker to walker by ws bytes (box depth 1).
template <typename T>
bool make_map(CUtensorMap* map, const T* base, size_t n, int rows, size_t ld, int tb, int nw = 1, size_t ws = 0) {
  auto fn = encode_fn();
  if (!fn) return false;
  const CUtensorMapDataType dt = sizeof(T) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64;
  cuuint64_t dims[3] = {(cuuint64_t)n, (cuuint64_t)rows, (cuuint64_t)nw};
  cuuint64_t strides[2] = {(cuuint64_t)(ld * sizeof(T)), (cuuint64_t)ws};
  cuuint32_t box[3] = {(cuuint32_t)(tb / sizeof(T)), (cuuint32_t)rows, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  const cuuint32_t rank = nw > 1 ? 3 : 2;
  if (nw > 1 && (ws % 16 != 0 || ws < (size_t)rows * ld * sizeof(T))) return false;
  return fn(map, dt, rank, const_cast<T*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
         CUDA_SUCCESS;
}

// Row bytes of a tile.  FP64: 512 (a lane's share is one element).  FP32: the
// largest of 1024, 512 and 256 at which every consumer pair can still hold a
// stage of its own (fewer, larger stages stream faster), 1024 only for Grams
// (modes 0, 1) and for the update of 9 to 16 fields (mode 2), where it was
// measured faster (larger updates stream as fast at 512).
template <typename T>
int tile_bytes(int mode, int nx, int ny) {
  if (sizeof(T) == 8) return 512;
  const int rows = (nx + 7) / 8 * 8 + (mode == 3 ? 0 : 8);
  auto fits = [&](int tb) { return (size_t)rows * tb * kPairs <= kDynBudget - 1024; };
  if ((mode <= 1 || (mode == 2 && nx > 8 && nx <= 16)) && ny <= 8 && fits(1024)) return 1024;
  return fits(512) ? 512 : 256;
}

template <typename T, int MODE, int R, int CW, int NRL, int TB>
void tile_launch(const CUtensorMap& mx, const CUtensorMap& my, int nx, int ny, int u0, int nu, size_t n,
                 const double* C, const double* Cadd, int uadd, int nadd, T* Yout, size_t ldo, double* out, double* part, unsigned* counter, const int* gate,
                 int mask, int* status, int polls, cudaStream_t st) {
  constexpr int TE = TB / (int)sizeof(T);
  const int nxp = (nx + 7) & ~7;
  const size_t tile_b = (size_t)(nxp + (MODE == 3 ? 0 : 8)) * TB;
  const size_t loaded = (size_t)(nx + (MODE == 3 ? 0 : ny)) * TB;
  // tiles per stage: a stage costs one CTA a roughly fixed handshake, so it
  // should move 16 KB or more (32 KB for at most 8 + 8 fields, where that was
  // measured faster), while every consumer pair can still hold a stage
  const size_t stage_min = nx <= 8 ? 32768 : 16384;
  int tps = 1;
  while (tps < 4 && loaded * tps < stage_min && (size_t)2 * tps * tile_b * kPairs <= kDynBudget - 1024) tps *= 2;
  const size_t stage_bytes = tps * tile_b;
  int nst = (int)((kDynBudget - 1024) / stage_bytes);
  if (nst > kMaxStages) nst = kMaxStages;
  // the epilogue reuses the ring for its partial sums (8 bytes an entry)
  const size_t epi = MODE >= 2 ? (size_t)(kConsumers * 32 + 8) * kSelf * 8
                               : (size_t)kConsumers * (MODE <= 1 ? nx : ny) * ny * 8;
  const size_t smem = std::max((size_t)nst * stage_bytes, epi) + 1024;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(tile2d_kernel<T, MODE, R, CW, NRL, TB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)kDynBudget);
    attr = true;
  }
  const int na = MODE <= 1 ? nx : ny;
  size_t want = kSMs;
  const size_t cap = (size_t)kStreamBlocks * MOTO_MAX_BASIS * MOTO_MAX_K / ((size_t)na * ny);
  if (want > cap) want = cap;
  const size_t ngroups = ((n + TE - 1) / TE + tps - 1) / tps;
  // a CTA (one an SM) pays a few microseconds of set-up and reduction, so it
  // streams at least ~256 KB: small fields (the walkers of a batch, the local
  // passes on small lattices) get fewer CTAs, large ones still one an SM.
  // The rule depends on the field size only, so a walker of a batch and the
  // same walker alone sum in the same order.
  // (FP64 fields: 32 KB, the FP64 arithmetic of a CTA being the slower part)
  const size_t target = sizeof(T) == 4 ? 262144 : 32768;
  const size_t per_cta = std::max<size_t>(1, (target + tps * loaded - 1) / (tps * loaded));
  const size_t need = (ngroups + per_cta - 1) / per_cta;
  if (want > need) want = need;
  const int grid = (int)(ngroups < want ? (ngroups > 0 ? ngroups : 1) : want);
  tile2d_kernel<T, MODE, R, CW, NRL, TB><<<wgrid(grid), kThrT, smem, st>>>(
      mx, my, nx, ny, u0, nu, n, C, Cadd, uadd, nadd, Yout, ldo, out, part, counter, nst, tps, gate, mask, status,
      polls, walker_ws());
}

// Gram lane layouts (R rows x CW columns a lane, NRL row lanes): FP32 fits
// the rows exactly where registers allow (NRL x R = the fields rounded up to
// 8; padded rows cost their loads and FMAs like real ones), and only the
// layouts that a row size can meet are instantiated for it.
template <typename T, int MODE, int TB>
void tile_dispatch(const CUtensorMap& mx, const CUtensorMap& my, int nx, int ny, int u0, int nu, size_t n,
                   const double* C, const double* Cadd, int uadd, int nadd, T* Yout, size_t ldo, double* out,
                   double* part, unsigned* counter, const int* gate, int mask, int* status, int polls,
                   cudaStream_t st) {
#define TL(RR, CC, NN)                                                                                           \
  tile_launch<T, MODE, RR, CC, NN, TB>(mx, my, nx, ny, u0, nu, n, C, Cadd, uadd, nadd, Yout, ldo, out, part,    \
                                       counter, gate, mask, status, polls, st)
  const int nxp = (nx + 7) & ~7;
  if constexpr (MODE >= 2) {
    TL(1, 4, 16);
  } else if constexpr (sizeof(T) == 8) {
    if (nxp <= 8) {
      TL(1, 2, 8);
    } else if (nxp <= 16) {
      TL(4, 4, 4);
    } else if (nxp <= 32) {
      TL(4, 4, 8);
    } else if (nxp <= 64) {
      TL(4, 4, 16);
    } else {
      TL(6, 4, 16);
    }
  } else if constexpr (TB == 1024) {  // at most 32 fields
    if (nxp <= 8) {
      TL(2, 4, 4);
    } else if (nxp <= 16) {
      TL(4, 4, 4);
    } else if (nxp <= 24) {
      TL(3, 4, 8);
    } else {
      TL(4, 4, 8);
    }
  } else if constexpr (TB == 512) {  // up to 72 fields
    switch (nxp) {
      case 8: case 16: case 24: case 32: TL(4, 4, 8); break;
      case 40: TL(5, 4, 8); break;
      case 48: TL(6, 4, 8); break;
      case 56: TL(7, 4, 8); break;
      case 64: TL(4, 4, 16); break;
      case 72: case 80: TL(5, 4, 16); break;
      default: TL(6, 4, 16); break;
    }
  } else {
    if (nxp <= 80) {
      TL(5, 4, 16);
    } else {
      TL(6, 4, 16);
    }
  }
#undef TL
}

}  // namespace

template <typename T>
bool launch_tile(int mode, const T* X, size_t ldx, int nx, int u0, int nu, const T* Y, size_t ldy, int ny, size_t n,
                 const double* C, T* Yout, size_t ldo, double* out, double* part, unsigned* counter, const int* gate,
                 int mask, int* status, cudaStream_t st, const double* Cadd, int uadd, int nadd, int polls) {
  auto al = [](const void* p) { return ((uintptr_t)p % 16) == 0; };
  if ((ldx * sizeof(T)) % 16 || (ldy * sizeof(T)) % 16 || !al(X) || (mode != 3 && !al(Y))) return false;
  if (mode == 2 && !Yout) return false;
  if (mode != 0 && Yout && ((ldo * sizeof(T)) % 16 || !al(Yout))) return false;
  if (Cadd && (mode != 2 || uadd < 0 || nadd < 0 || uadd + nadd > nx)) return false;
  if (nx < 1 || nx > MOTO_MAX_BASIS || ny < 1 || ny > 8 || n >= (1ull << 31)) return false;
  if (mode == 1 && (u0 < 0 || nu < 0 || u0 + nu > nx)) return false;
  if (mode >= 2) {
    u0 = 0;
    nu = nx;
  }
  const int tb = tile_bytes<T>(mode, nx, ny);
  CUtensorMap mx, my;
  const WalkerGrid wg = walker_grid();
  if (!make_map<T>(&mx, X, n, nx, ldx, tb, wg.nw, wg.ws)) return false;
  if (mode != 3) {
    if (!make_map<T>(&my, Y, n, ny, ldy, tb, wg.nw, wg.ws)) return false;
  } else {
    my = mx;
  }
#define TD(M, B) tile_dispatch<T, M, B>(mx, my, nx, ny, u0, nu, n, C, Cadd, uadd, nadd, Yout, ldo, out, part, counter, gate, mask, status, polls, st)
  if constexpr (sizeof(T) == 8) {
    switch (mode) {
      case 0: TD(0, 512); break;
      case 1: TD(1, 512); break;
      case 2: TD(2, 512); break;
      default: TD(3, 512); break;
    }
  } else {
    if (tb == 1024) {
      if (mode == 0)
        TD(0, 1024);
      else if (mode == 1)
        TD(1, 1024);
      else
        TD(2, 1024);
      return true;
    }
    switch (mode * 2 + (tb == 512 ? 1 : 0)) {
      case 0: TD(0, 256); break;
      case 1: TD(0, 512); break;
      case 2: TD(1, 256); break;
      case 3: TD(1, 512); break;
      case 4: TD(2, 256); break;
      case 5: TD(2, 512); break;
      case 6: TD(3, 256); break;
      default: TD(3, 512); break;
    }
  }
#undef TD
  return true;
}

template bool launch_tile<float>(int, const float*, size_t, int, int, int, const float*, size_t, int, size_t,
                                 const double*, float*, size_t, double*, double*, unsigned*, const int*, int, int*,
                                 cudaStream_t, const double*, int, int, int);
template bool launch_tile<double>(int, const double*, size_t, int, int, int, const double*, size_t, int, size_t,
                                  const double*, double*, size_t, double*, double*, unsigned*, const int*, int, int*,
                                  cudaStream_t, const double*, int, int, int);

}  // namespace moto
