// Register-blocked tangent HVP, the eigensolvers' operator:
//   (H v)_i = P_i [ h_i(v) - 2 K v_iz z - s_i v_i ]
// with h the linear stencil of the exchange shells and the Neel DMI (see
// stencil.cuh for the formula and its reading of Eq. param-hamiltonian).
//
// A block stages a 32 x 64-site tile of v (plus a 2-site periodic halo) in
// shared memory with asynchronous copies, double-buffered over the vectors,
// and m, s of its sites once.  A thread then owns a column strip of
// kStrip sites along a2: it walks the kStrip + 4 tile rows the strip needs,
// reading each row once (five columns x - 2 .. x + 2 of the three components)
// and scattering it into the accumulators of the (up to five) strip sites it is
// a neighbour of, so a site costs ~22 shared loads instead of the 54 of a
// per-site gather.  m and s are read once per site.  Multi-vector calls loop
// over the vectors inside the kernel.
#include "internal.h"

namespace moto {

namespace {
constexpr int kStrip = 8;  // sites per thread along a2
constexpr int kWarpsY = 8;  // warps per block, stacked along a2

template <typename T>
struct Row {
  T x[5], y[5], z[5];  // columns x-2 .. x+2
};

// Adds to h the contribution of a row at offset d2 (= row - site) from the
// site; w holds -2 J_s per shell and 2 D.
template <typename T, int D2>
__device__ __forceinline__ void add_row(const Row<T>& r, T& hx, T& hy, T& hz, T j0, T j1, T j2, T twoD) {
  // column c of the row is offset d1 = c - 2
  const T s3 = (T)0.86602540378443864676, h = (T)0.5;
#define XC(c) r.x[(c) + 2]
#define YC(c) r.y[(c) + 2]
#define ZC(c) r.z[(c) + 2]
  if (D2 == -2) {  // (1,-2) s2; (0,-2), (2,-2) s3
    hx += j1 * XC(1) + j2 * (XC(0) + XC(2));
    hy += j1 * YC(1) + j2 * (YC(0) + YC(2));
    hz += j1 * ZC(1) + j2 * (ZC(0) + ZC(2));
  } else if (D2 == -1) {  // (0,-1), (1,-1) s1; (-1,-1), (2,-1) s2
    hx += j0 * (XC(0) + XC(1)) + j1 * (XC(-1) + XC(2));
    hy += j0 * (YC(0) + YC(1)) + j1 * (YC(-1) + YC(2));
    hz += j0 * (ZC(0) + ZC(1)) + j1 * (ZC(-1) + ZC(2));
    // DMI: (0,-1) d_hat = (-1/2, -s3); (1,-1) d_hat = (1/2, -s3)
    hx += twoD * (-h * ZC(0) + h * ZC(1));
    hy += twoD * (-s3 * (ZC(0) + ZC(1)));
    hz -= twoD * (-h * XC(0) - s3 * YC(0) + h * XC(1) - s3 * YC(1));
  } else if (D2 == 0) {  // (1,0), (-1,0) s1; (2,0), (-2,0) s3
    hx += j0 * (XC(1) + XC(-1)) + j2 * (XC(2) + XC(-2));
    hy += j0 * (YC(1) + YC(-1)) + j2 * (YC(2) + YC(-2));
    hz += j0 * (ZC(1) + ZC(-1)) + j2 * (ZC(2) + ZC(-2));
    // DMI: (1,0) d_hat = (1, 0); (-1,0) d_hat = (-1, 0)
    hx += twoD * (ZC(1) - ZC(-1));
    hz -= twoD * (XC(1) - XC(-1));
  } else if (D2 == 1) {  // (0,1), (-1,1) s1; (1,1), (-2,1) s2
    hx += j0 * (XC(0) + XC(-1)) + j1 * (XC(1) + XC(-2));
    hy += j0 * (YC(0) + YC(-1)) + j1 * (YC(1) + YC(-2));
    hz += j0 * (ZC(0) + ZC(-1)) + j1 * (ZC(1) + ZC(-2));
    // DMI: (0,1) d_hat = (1/2, s3); (-1,1) d_hat = (-1/2, s3)
    hx += twoD * (h * ZC(0) - h * ZC(-1));
    hy += twoD * (s3 * (ZC(0) + ZC(-1)));
    hz -= twoD * (h * XC(0) + s3 * YC(0) - h * XC(-1) + s3 * YC(-1));
  } else {  // D2 == 2: (-1,2) s2; (0,2), (-2,2) s3
    hx += j1 * XC(-1) + j2 * (XC(0) + XC(-2));
    hy += j1 * YC(-1) + j2 * (YC(0) + YC(-2));
    hz += j1 * ZC(-1) + j2 * (ZC(0) + ZC(-2));
  }
#undef XC
#undef YC
#undef ZC
}

template <typename T, int RR, int S>
__device__ __forceinline__ void scatter(const Row<T>& r, T (&ax)[kStrip], T (&ay)[kStrip], T (&az)[kStrip], T j0,
                                        T j1, T j2, T twoD) {
  // row RR of the walk (site rows start at RR = 2) meets site S at offset d2
  constexpr int D2 = RR - 2 - S;
  if (S >= 0 && S < kStrip && D2 >= -2 && D2 <= 2) add_row<T, D2>(r, ax[S], ay[S], az[S], j0, j1, j2, twoD);
}

template <typename T, int RR>
__device__ __forceinline__ void scatter_row(const Row<T>& r, T (&ax)[kStrip], T (&ay)[kStrip], T (&az)[kStrip], T j0,
                                            T j1, T j2, T twoD) {
  scatter<T, RR, RR - 4>(r, ax, ay, az, j0, j1, j2, twoD);
  scatter<T, RR, RR - 3>(r, ax, ay, az, j0, j1, j2, twoD);
  scatter<T, RR, RR - 2>(r, ax, ay, az, j0, j1, j2, twoD);
  scatter<T, RR, RR - 1>(r, ax, ay, az, j0, j1, j2, twoD);
  scatter<T, RR, RR>(r, ax, ay, az, j0, j1, j2, twoD);
}

constexpr int kTX = 32, kTY = kWarpsY * kStrip;  // sites per block tile
constexpr int kSX = kTX + 4, kSY = kTY + 4;          // staged tile with halo

template <typename T, int RR>
struct SWalk {
  static __device__ __forceinline__ void run(const T* __restrict__ tile, int row0, int lane, T (&ax)[kStrip],
                                             T (&ay)[kStrip], T (&az)[kStrip], T j0, T j1, T j2, T twoD) {
    SWalk<T, RR - 1>::run(tile, row0, lane, ax, ay, az, j0, j1, j2, twoD);
    Row<T> r;
    const T* p = tile + (size_t)(row0 + RR) * kSX + lane;
#pragma unroll
    for (int c = 0; c < 5; ++c) {
      r.x[c] = p[c];
      r.y[c] = p[(size_t)kSX * kSY + c];
      r.z[c] = p[2 * (size_t)kSX * kSY + c];
    }
    scatter_row<T, RR>(r, ax, ay, az, j0, j1, j2, twoD);
  }
};
template <typename T>
struct SWalk<T, -1> {
  static __device__ __forceinline__ void run(const T*, int, int, T (&)[kStrip], T (&)[kStrip], T (&)[kStrip], T, T, T,
                                             T) {}
};

}  // namespace

// 4-byte asynchronous global -> shared copy (cp.async, cached in L1)
__device__ __forceinline__ void cp_async4(void* smem_dst, const void* gsrc) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((uint32_t)__cvta_generic_to_shared(smem_dst)),
               "l"(gsrc)
               : "memory");
}
__device__ __forceinline__ void cp_async8(void* smem_dst, const void* gsrc) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((uint32_t)__cvta_generic_to_shared(smem_dst)),
               "l"(gsrc)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Starts the copy of vector v's halo'd tile into `tile` (one element per copy;
// periodic wrap at the lattice edges).
template <typename T>
__device__ __forceinline__ void stage_tile(T* tile, const T* __restrict__ v, size_t N, int L1, int L2, int x0, int y0,
                                           bool interior) {
  for (int idx = threadIdx.x; idx < kSX * kSY; idx += blockDim.x) {
    const int ly = idx / kSX, lx = idx - ly * kSX;
    int gx = x0 + lx - 2, gy = y0 + ly - 2;
    if (!interior) {
      gx = wrap(gx, L1);
      gy = wrap(gy, L2);
    }
    const size_t g = (size_t)gy * L1 + gx;
    if constexpr (sizeof(T) == 4) {
      cp_async4(tile + idx, v + g);
      cp_async4(tile + (size_t)kSX * kSY + idx, v + N + g);
      cp_async4(tile + 2 * (size_t)kSX * kSY + idx, v + 2 * N + g);
    } else {
      cp_async8(tile + idx, v + g);
      cp_async8(tile + (size_t)kSX * kSY + idx, v + N + g);
      cp_async8(tile + 2 * (size_t)kSX * kSY + idx, v + 2 * N + g);
    }
  }
  cp_async_commit();
}

// Two tile buffers: the copy of vector j + 1 runs while vector j is computed.
// m and s of the block's sites are staged once (they are read for every
// vector in the output phase).
template <typename T>
__global__ void __launch_bounds__(32 * kWarpsY) hvp_strip_kernel(ModelDev md, const T* __restrict__ m,
                                                                 const T* __restrict__ s, const T* __restrict__ V,
                                                                 size_t ldv, T* __restrict__ HV, size_t ldhv, int nvec,
                                                                 const int* gate, int mask) {
  if (gate && (*gate & mask)) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* tiles = reinterpret_cast<T*>(smem_raw);  // [2][3][kSY][kSX]
  constexpr size_t kTileElems = 3 * (size_t)kSX * kSY;
  T* ms = tiles + 2 * kTileElems;  // [4][kTY][kTX]: m_x, m_y, m_z, s
  const int lane = threadIdx.x & 31, wy = threadIdx.x >> 5;
  const int x0 = blockIdx.x * kTX, y0 = blockIdx.y * kTY;
  const int L1 = md.L1, L2 = md.L2;
  const size_t N = md.N;
  const T j0 = (T)(-2.0 * md.J[0]);
  const T j1 = (T)(md.n_shells > 1 ? -2.0 * md.J[1] : 0.0);
  const T j2 = (T)(md.n_shells > 2 ? -2.0 * md.J[2] : 0.0);
  const T twoD = (T)(2.0 * md.D), twoK = (T)(2.0 * md.K);
  const bool interior = x0 >= 2 && y0 >= 2 && x0 + kTX + 2 <= L1 && y0 + kTY + 2 <= L2;
  const int x = x0 + lane;
  // m, s of the tile (sites outside the lattice are never read back)
  for (int idx = threadIdx.x; idx < 4 * kTY * kTX; idx += blockDim.x) {
    const int comp = idx / (kTY * kTX), rem = idx - comp * (kTY * kTX);
    const int ly = rem / kTX, lx = rem - ly * kTX;
    const int gx = x0 + lx, gy = y0 + ly;
    if (gx < L1 && gy < L2) {
      const size_t g = (size_t)gy * L1 + gx;
      const T* src = comp < 3 ? m + (size_t)comp * N + g : s + g;
      if constexpr (sizeof(T) == 4)
        cp_async4(ms + idx, src);
      else
        cp_async8(ms + idx, src);
    }
  }
  stage_tile(tiles, V, N, L1, L2, x0, y0, interior);
  for (int j = 0; j < nvec; ++j) {
    T* tile = tiles + (size_t)(j & 1) * kTileElems;
    T* hv = HV + (size_t)j * ldhv;
    if (j + 1 < nvec) {
      stage_tile(tiles + (size_t)((j + 1) & 1) * kTileElems, V + (size_t)(j + 1) * ldv, N, L1, L2, x0, y0, interior);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    T ax[kStrip], ay[kStrip], az[kStrip];
#pragma unroll
    for (int k = 0; k < kStrip; ++k) ax[k] = ay[k] = az[k] = (T)0;
    SWalk<T, kStrip + 3>::run(tile, wy * kStrip, lane, ax, ay, az, j0, j1, j2, twoD);
    if (x < L1) {
#pragma unroll
      for (int k = 0; k < kStrip; ++k) {
        const int ly = wy * kStrip + k;
        const int y = y0 + ly;
        if (y >= L2) break;
        const size_t i = (size_t)y * L1 + x;
        const size_t ti = (size_t)(ly + 2) * kSX + lane + 2;
        const T vx = tile[ti], vy = tile[(size_t)kSX * kSY + ti], vz = tile[2 * (size_t)kSX * kSY + ti];
        const int mi = ly * kTX + lane;
        const T m0 = ms[mi], m1 = ms[kTY * kTX + mi], m2 = ms[2 * kTY * kTX + mi], si = ms[3 * kTY * kTX + mi];
        const T hx = ax[k] - si * vx, hy = ay[k] - si * vy, hz = az[k] - twoK * vz - si * vz;
        const T p = m0 * hx + m1 * hy + m2 * hz;
        hv[i] = hx - p * m0;
        hv[N + i] = hy - p * m1;
        hv[2 * N + i] = hz - p * m2;
      }
    }
    // every warp is done with this buffer before the copy issued in the next
    // iteration (for vector j + 2) overwrites it
    __syncthreads();
  }
}

template <typename T>
void launch_hvp_strip(const ModelDev& md, const T* m, const T* s, const T* V, size_t ldv, T* HV, size_t ldhv,
                      int nvec, const int* gate, int mask, cudaStream_t st) {
  const dim3 grid((md.L1 + kTX - 1) / kTX, (md.L2 + kTY - 1) / kTY);
  const size_t smem = (2 * 3 * (size_t)kSX * kSY + 4 * (size_t)kTY * kTX) * sizeof(T);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(hvp_strip_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    attr = true;
  }
  hvp_strip_kernel<T><<<grid, 32 * kWarpsY, smem, st>>>(md, m, s, V, ldv, HV, ldhv, nvec, gate, mask);
}

template void launch_hvp_strip<float>(const ModelDev&, const float*, const float*, const float*, size_t, float*,
                                      size_t, int, const int*, int, cudaStream_t);
template void launch_hvp_strip<double>(const ModelDev&, const double*, const double*, const double*, size_t, double*,
                                       size_t, int, const int*, int, cudaStream_t);

}  // namespace moto
