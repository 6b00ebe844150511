// Register-blocked tangent HVP, the eigensolvers' operator (Methods, "HVP
// operator mode"):
//   (H v)_i = P_i [ h_i(v) - 2 K v_iz z - s_i v_i ]
// with h the linear stencil of the exchange shells and the Neel DMI
// (strip.cuh gives the formula and its reading of Eq. param-hamiltonian).
//
// A block stages a TY x 64-site tile of v with asynchronous copies,
// double-buffered over the vectors of the call, and m, s of its sites once.
// Threads own column pairs of SW-row strips (strip.cuh); the -s_i v_i and
// -2 K v_iz terms are added when the walk reaches the site's own row, so the
// result does not depend on the variant (SW, warps per block, m held in
// registers or re-read from shared memory), which the launcher picks per
// lattice, precision and vector count by timing (see hvp_variant).
#include <cuda_runtime.h>

#include <mutex>
#include <vector>

#include "internal.h"
#include "strip.cuh"

namespace moto {

using namespace strip;

namespace {

// on-site hook of the HVP walk: (hx, hy, hz) += -s v - 2 K v_z z at the
// site's own row
template <typename T, int SW, class P>
struct HvpOnSite {
  typename PK<T>::V nsi[SW];  // -s_i of the strip's site pairs
  typename PK<T>::V twoK;
  template <int S>
  __device__ __forceinline__ void center(const RowP<T>& r, typename PK<T>::V& hx, typename PK<T>::V& hy,
                                         typename PK<T>::V& hz) {
    hx = P::fma(nsi[S], r.x[2], hx);
    hy = P::fma(nsi[S], r.y[2], hy);
    hz = P::fma(P::sub(nsi[S], twoK), r.z[2], hz);
  }
};

}  // namespace

// m and s of the block's sites are staged once; with MREG the thread moves
// its sites' m into registers for all vectors, otherwise it re-reads them from
// shared memory per vector.  AR: FP32 pair arithmetic as packed f32x2
// instructions (1) or scalar pairs (0) (PA; the same sums bit for bit).
// `aligned`: L1 and the field strides are multiples of 16 bytes / sizeof(T)
// and the fields start on 16-byte boundaries (interior blocks then stage
// with 16-byte copies).
template <typename T, int SW, int WY, bool MREG, int AR>
__global__ void __launch_bounds__(32 * WY) hvp_strip_kernel(ModelDev md, Weights<T> hw, const T* __restrict__ m,
                                                            const T* __restrict__ s, const T* __restrict__ V,
                                                            size_t ldv, T* __restrict__ HV, size_t ldhv, int nvec,
                                                            int aligned, const int* gate, int mask, size_t ws) {
  m = wofs(m, ws);
  s = wofs(s, ws);
  V = wofs(V, ws);
  HV = wofs(HV, ws);
  gate = wofs(gate, ws);
  if (gate && (*gate & mask)) return;
  constexpr int TY = SW * WY;
  typedef Dims<TY> DM;
  typedef typename PA<T, AR>::P P;
  typedef typename PK<T>::V VP;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* tiles = reinterpret_cast<T*>(smem_raw);  // [2][3][SY][kSX]
  T* ms = tiles + 2 * DM::kTile;               // [4][TY][kTX]: m_x, m_y, m_z, s
  const int lane = threadIdx.x & 31, wy = threadIdx.x >> 5;
  const int x0 = blockIdx.x * kTX, y0 = blockIdx.y * TY;
  const int L1 = md.L1, L2 = md.L2;
  const size_t N = md.N;
  const WP<T> w(hw);
  const bool vec16 = aligned && tile_inside<TY>(x0, y0, L1, L2);
  // m, s of the tile (sites outside the lattice are never read back)
  if (vec16) {
    constexpr int kE = 16 / (int)sizeof(T), kCh = kTX / kE;
    for (int idx = threadIdx.x; idx < 4 * TY * kCh; idx += blockDim.x) {
      const int comp = idx / (TY * kCh), rem = idx - comp * (TY * kCh);
      const int ly = rem / kCh, ch = rem - ly * kCh;
      const size_t g = (size_t)(y0 + ly) * L1 + x0 + ch * kE;
      const T* src = comp < 3 ? m + (size_t)comp * N + g : s + g;
      cp_async16(ms + (size_t)comp * TY * kTX + ly * kTX + ch * kE, src);
    }
  } else {
    for (int idx = threadIdx.x; idx < 4 * TY * kTX; idx += blockDim.x) {
      const int comp = idx / (TY * kTX), rem = idx - comp * (TY * kTX);
      const int ly = rem / kTX, lx = rem - ly * kTX;
      const int gx = x0 + lx, gy = y0 + ly;
      if (gx < L1 && gy < L2) {
        const size_t g = (size_t)gy * L1 + gx;
        cp_elem(ms + idx, comp < 3 ? m + (size_t)comp * N + g : s + g);
      }
    }
  }
  // interior tiles: the copies' source offsets once for all vectors
  TileCopies<T, DM::SY, 32 * WY> tc;
  if (vec16) {
    tc.init(N, L1, x0, y0);
    tc.stage(tiles, V);
  } else {
    stage_tile<T, DM::SY>(tiles, V, N, L1, L2, x0, y0, false);
  }
  const int x = x0 + 2 * lane;  // the thread's columns x, x + 1
  const bool pair_store = aligned && x + 1 < L1;
  HvpOnSite<T, SW, P> os;
  os.twoK = P::bc(hw.twoK);
  VP mr[MREG ? SW : 1][3];
  for (int j = 0; j < nvec; ++j) {
    T* tile = tiles + (size_t)(j & 1) * DM::kTile;
    T* hv = HV + (size_t)j * ldhv;
    if (j + 1 < nvec) {
      T* nt = tiles + (size_t)((j + 1) & 1) * DM::kTile;
      if (vec16)
        tc.stage(nt, V + (size_t)(j + 1) * ldv);
      else
        stage_tile<T, DM::SY>(nt, V + (size_t)(j + 1) * ldv, N, L1, L2, x0, y0, false);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    if (j == 0) {
#pragma unroll
      for (int k = 0; k < SW; ++k) {
        const int mi = (wy * SW + k) * kTX + 2 * lane;
        os.nsi[k] = P::mul(*reinterpret_cast<const VP*>(ms + 3 * TY * kTX + mi), P::bc((T)-1));
        if constexpr (MREG) {
#pragma unroll
          for (int c = 0; c < 3; ++c) mr[k][c] = *reinterpret_cast<const VP*>(ms + c * TY * kTX + mi);
        }
      }
    }
    VP ax[SW], ay[SW], az[SW];
    walk<T, SW, DM::SY, P>(tile, wy * SW, lane, ax, ay, az, w, os);
    if (x < L1) {
#pragma unroll
      for (int k = 0; k < SW; ++k) {
        const int ly = wy * SW + k;
        const int y = y0 + ly;
        if (y >= L2) break;
        const size_t i = (size_t)y * L1 + x;
        VP m0, m1, m2;
        if constexpr (MREG) {
          m0 = mr[k][0];
          m1 = mr[k][1];
          m2 = mr[k][2];
        } else {
          const int mi = ly * kTX + 2 * lane;
          m0 = *reinterpret_cast<const VP*>(ms + mi);
          m1 = *reinterpret_cast<const VP*>(ms + TY * kTX + mi);
          m2 = *reinterpret_cast<const VP*>(ms + 2 * TY * kTX + mi);
        }
        const VP p = P::fma(m2, az[k], P::fma(m1, ay[k], P::mul(m0, ax[k])));
        const VP np = P::mul(p, P::bc((T)-1));
        const VP ox = P::fma(np, m0, ax[k]);
        const VP oy = P::fma(np, m1, ay[k]);
        const VP oz = P::fma(np, m2, az[k]);
        if (pair_store) {
          *reinterpret_cast<VP*>(hv + i) = ox;
          *reinterpret_cast<VP*>(hv + N + i) = oy;
          *reinterpret_cast<VP*>(hv + 2 * N + i) = oz;
        } else {
          hv[i] = ox.x;
          hv[N + i] = oy.x;
          hv[2 * N + i] = oz.x;
          if (x + 1 < L1) {
            hv[i + 1] = ox.y;
            hv[N + i + 1] = oy.y;
            hv[2 * N + i + 1] = oz.y;
          }
        }
      }
    }
    // every warp is done with this buffer before the copy issued in the next
    // iteration (for vector j + 2) overwrites it
    __syncthreads();
  }
}

namespace {

// The variants the launcher chooses from (all give bit-identical results).
struct HvpVariant {
  int sw, wy, mreg, ar;
};
constexpr HvpVariant kHvpVariants[] = {{4, 4, 1, 0}, {4, 4, 0, 0}, {8, 2, 0, 0}, {2, 8, 1, 0},
                                       {2, 8, 1, 1}, {4, 4, 1, 1}, {4, 4, 0, 1}, {8, 2, 0, 1}};
constexpr int kNumHvpVariants = sizeof(kHvpVariants) / sizeof(kHvpVariants[0]);

template <typename T, int SW, int WY, bool MREG, int AR0>
void hvp_launch_v(const ModelDev& md, const Weights<T>& hw, const T* m, const T* s, const T* V, size_t ldv, T* HV,
                  size_t ldhv, int nvec, int aligned, const int* gate, int mask, cudaStream_t st) {
  constexpr int AR = sizeof(T) == 4 ? AR0 : 1;  // FP64 pairs are scalar in every form
  constexpr int TY = SW * WY;
  const dim3 grid((md.L1 + kTX - 1) / kTX, (md.L2 + TY - 1) / TY);
  const size_t smem = (2 * Dims<TY>::kTile + 4 * (size_t)TY * kTX) * sizeof(T);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(hvp_strip_kernel<T, SW, WY, MREG, AR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    attr = true;
  }
  hvp_strip_kernel<T, SW, WY, MREG, AR><<<wgrid(grid), 32 * WY, smem, st>>>(md, hw, m, s, V, ldv, HV, ldhv, nvec, aligned, gate,
                                                                 mask, walker_ws());
}

template <typename T>
void hvp_launch_index(int v, const ModelDev& md, const Weights<T>& hw, const T* m, const T* s, const T* V, size_t ldv,
                      T* HV, size_t ldhv, int nvec, int aligned, const int* gate, int mask, cudaStream_t st) {
  switch (v) {
    case 1: hvp_launch_v<T, 4, 4, false, 0>(md, hw, m, s, V, ldv, HV, ldhv, nvec, aligned, gate, mask, st); break;
    case 2: hvp_launch_v<T, 8, 2, false, 0>(md, hw, m, s, V, ldv, HV, ldhv, nvec, aligned, gate, mask, st); break;
    case 3: hvp_launch_v<T, 2, 8, true, 0>(md, hw, m, s, V, ldv, HV, ldhv, nvec, aligned, gate, mask, st); break;
    case 4: hvp_launch_v<T, 2, 8, true, 1>(md, hw, m, s, V, ldv, HV, ldhv, nvec, aligned, gate, mask, st); break;
    case 5: hvp_launch_v<T, 4, 4, true, 1>(md, hw, m, s, V, ldv, HV, ldhv, nvec, aligned, gate, mask, st); break;
    case 6: hvp_launch_v<T, 4, 4, false, 1>(md, hw, m, s, V, ldv, HV, ldhv, nvec, aligned, gate, mask, st); break;
    case 7: hvp_launch_v<T, 8, 2, false, 1>(md, hw, m, s, V, ldv, HV, ldhv, nvec, aligned, gate, mask, st); break;
    default: hvp_launch_v<T, 4, 4, true, 0>(md, hw, m, s, V, ldv, HV, ldhv, nvec, aligned, gate, mask, st); break;
  }
}

// Process-wide choices of the autotuner: (L1, L2, element size, nvec) ->
// variant.  Lattices without an entry use variant 0.
struct HvpChoice {
  int L1, L2, esize, nvec, variant;
};
std::mutex g_hvp_mutex;
std::vector<HvpChoice> g_hvp_choices;

int hvp_choice(int L1, int L2, int esize, int nvec) {
  std::lock_guard<std::mutex> lock(g_hvp_mutex);
  for (const HvpChoice& c : g_hvp_choices)
    if (c.L1 == L1 && c.L2 == L2 && c.esize == esize && c.nvec == nvec) return c.variant;
  return -1;
}

}  // namespace

int hvp_variant_count() { return kNumHvpVariants; }

template <typename T>
void launch_hvp_strip_variant(int variant, const ModelDev& md, const T* m, const T* s, const T* V, size_t ldv, T* HV,
                              size_t ldhv, int nvec, const int* gate, int mask, cudaStream_t st) {
  constexpr size_t kE = 16 / sizeof(T);
  auto al16 = [](const void* p) { return ((uintptr_t)p % 16) == 0; };
  const int aligned = (md.L1 % (int)kE == 0) && (nvec < 2 || (ldv % kE == 0 && ldhv % kE == 0)) && al16(m) &&
                      al16(s) && al16(V) && al16(HV);
  const Weights<T> hw = make_weights<T>(md);
  hvp_launch_index<T>(variant, md, hw, m, s, V, ldv, HV, ldhv, nvec, aligned, gate, mask, st);
}

template <typename T>
void launch_hvp_strip(const ModelDev& md, const T* m, const T* s, const T* V, size_t ldv, T* HV, size_t ldhv,
                      int nvec, const int* gate, int mask, cudaStream_t st) {
  int v = hvp_choice(md.L1, md.L2, (int)sizeof(T), nvec);
  launch_hvp_strip_variant<T>(v < 0 ? 0 : v, md, m, s, V, ldv, HV, ldhv, nvec, gate, mask, st);
}

int hvp_tuned_variant(int L1, int L2, int esize, int nvec) { return hvp_choice(L1, L2, esize, nvec); }

void hvp_record_variant(int L1, int L2, int esize, int nvec, int variant) {
  std::lock_guard<std::mutex> lock(g_hvp_mutex);
  for (HvpChoice& c : g_hvp_choices)
    if (c.L1 == L1 && c.L2 == L2 && c.esize == esize && c.nvec == nvec) {
      c.variant = variant;
      return;
    }
  g_hvp_choices.push_back(HvpChoice{L1, L2, esize, nvec, variant});
}

template void launch_hvp_strip<float>(const ModelDev&, const float*, const float*, const float*, size_t, float*,
                                      size_t, int, const int*, int, cudaStream_t);
template void launch_hvp_strip<double>(const ModelDev&, const double*, const double*, const double*, size_t, double*,
                                       size_t, int, const int*, int, cudaStream_t);
template void launch_hvp_strip_variant<float>(int, const ModelDev&, const float*, const float*, const float*, size_t,
                                              float*, size_t, int, const int*, int, cudaStream_t);
template void launch_hvp_strip_variant<double>(int, const ModelDev&, const double*, const double*, const double*,
                                               size_t, double*, size_t, int, const int*, int, cudaStream_t);

}  // namespace moto
