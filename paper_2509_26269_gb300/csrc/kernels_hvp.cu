// Register-blocked tangent HVP, the eigensolvers' operator:
//   (H v)_i = P_i [ h_i(v) - 2 K v_iz z - s_i v_i ]
// with h the linear stencil of the exchange shells and the Neel DMI (see
// stencil.cuh for the formula and its reading of Eq. param-hamiltonian).
//
// A block stages a kTY x 64-site tile of v (plus a 2-site periodic halo,
// widened to 4 columns on each side so that every staged row starts on a
// 16-byte boundary) in shared memory with asynchronous 16-byte copies,
// double-buffered over the vectors, and m, s of its sites once.  A thread owns
// two adjacent columns (x, x + 1) of a strip of kStrip rows: it walks the
// kStrip + 4 tile rows the strip needs, reading each row once as three 8-byte
// column pairs per component, and scatters it into the accumulators of the
// (up to five) strip sites it is a neighbour of.  Every value of the walk is
// a column pair, so in FP32 each add and FMA is one packed f32x2 instruction
// for two sites (FP64 takes the same path with scalar pairs).  Multi-vector
// calls loop over the vectors inside the kernel.
#include "internal.h"

namespace moto {

namespace {
constexpr int kStrip = 4;  // rows per thread along a2
// warps per block, stacked along a2: 16 x 64-site tiles, four blocks an SM
// (measured faster than 32 x 64 tiles at two blocks an SM)
constexpr int kWarpsY = 4;
constexpr int kTX = 64, kTY = kWarpsY * kStrip;  // sites per block tile
constexpr int kPadL = 4;  // staged columns left of the tile (2 halo + 2 alignment)
constexpr int kSX = kTX + 2 * kPadL, kSY = kTY + 4;  // staged tile

// Column pairs and their arithmetic: packed f32x2 instructions for FP32,
// two scalar operations for FP64.
template <typename T>
struct PK;
template <>
struct PK<float> {
  typedef float2 V;
  static __device__ __forceinline__ unsigned long long u(const V& a) {
    return *reinterpret_cast<const unsigned long long*>(&a);
  }
  static __device__ __forceinline__ V v(unsigned long long d) { return *reinterpret_cast<V*>(&d); }
  static __device__ __forceinline__ V bc(float s) { return make_float2(s, s); }
  static __device__ __forceinline__ V mk(float a, float b) { return make_float2(a, b); }
  static __device__ __forceinline__ V add(V a, V b) {
    unsigned long long d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(u(a)), "l"(u(b)));
    return v(d);
  }
  static __device__ __forceinline__ V sub(V a, V b) {
    unsigned long long d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(u(a)), "l"(u(b)));
    return v(d);
  }
  static __device__ __forceinline__ V mul(V a, V b) {
    unsigned long long d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(u(a)), "l"(u(b)));
    return v(d);
  }
  static __device__ __forceinline__ V fma(V a, V b, V c) {
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(u(a)), "l"(u(b)), "l"(u(c)));
    return v(d);
  }
};
template <>
struct PK<double> {
  typedef double2 V;
  static __device__ __forceinline__ V bc(double s) { return make_double2(s, s); }
  static __device__ __forceinline__ V mk(double a, double b) { return make_double2(a, b); }
  static __device__ __forceinline__ V add(V a, V b) { return make_double2(a.x + b.x, a.y + b.y); }
  static __device__ __forceinline__ V sub(V a, V b) { return make_double2(a.x - b.x, a.y - b.y); }
  static __device__ __forceinline__ V mul(V a, V b) { return make_double2(a.x * b.x, a.y * b.y); }
  static __device__ __forceinline__ V fma(V a, V b, V c) {
    return make_double2(::fma(a.x, b.x, c.x), ::fma(a.y, b.y, c.y));
  }
};

// One staged row as seen from the column pair (x, x + 1): p[c + 2] holds the
// columns (x + c, x + 1 + c), c = -2 .. 2, of each component.
template <typename T>
struct RowP {
  typename PK<T>::V x[5], y[5], z[5];
};

// Stencil weights as pairs: -2 J_s per shell, D (= 2 D / 2), 2 D, and
// +-2 D sqrt(3)/2.
template <typename T>
struct WP {
  typename PK<T>::V j0, j1, j2, dh, dh2, ds, nds;
};
// The same weights in the field precision, formed on the host, and 2 K.
template <typename T>
struct HvpW {
  T j0, j1, j2, dh, dh2, ds, twoK;
};

// Adds to (hx, hy, hz) the contribution of a row at offset d2 (= row - site).
template <typename T, int D2>
__device__ __forceinline__ void add_row(const RowP<T>& r, typename PK<T>::V& hx, typename PK<T>::V& hy,
                                        typename PK<T>::V& hz, const WP<T>& w) {
  typedef PK<T> P;
#define XC(c) r.x[(c) + 2]
#define YC(c) r.y[(c) + 2]
#define ZC(c) r.z[(c) + 2]
  if (D2 == -2) {  // (1,-2) s2; (0,-2), (2,-2) s3
    hx = P::fma(w.j1, XC(1), hx);
    hy = P::fma(w.j1, YC(1), hy);
    hz = P::fma(w.j1, ZC(1), hz);
    hx = P::fma(w.j2, P::add(XC(0), XC(2)), hx);
    hy = P::fma(w.j2, P::add(YC(0), YC(2)), hy);
    hz = P::fma(w.j2, P::add(ZC(0), ZC(2)), hz);
  } else if (D2 == -1) {  // (0,-1), (1,-1) s1; (-1,-1), (2,-1) s2
    // DMI: (0,-1) d_hat = (-1/2, -s3); (1,-1) d_hat = (1/2, -s3)
    const typename P::V z01 = P::add(ZC(0), ZC(1));
    hx = P::fma(w.j0, P::add(XC(0), XC(1)), hx);
    hy = P::fma(w.j0, P::add(YC(0), YC(1)), hy);
    hz = P::fma(w.j0, z01, hz);
    hx = P::fma(w.j1, P::add(XC(-1), XC(2)), hx);
    hy = P::fma(w.j1, P::add(YC(-1), YC(2)), hy);
    hz = P::fma(w.j1, P::add(ZC(-1), ZC(2)), hz);
    hx = P::fma(w.dh, P::sub(ZC(1), ZC(0)), hx);
    hy = P::fma(w.nds, z01, hy);
    hz = P::fma(w.dh, P::sub(XC(0), XC(1)), hz);
    hz = P::fma(w.ds, P::add(YC(0), YC(1)), hz);
  } else if (D2 == 0) {  // (1,0), (-1,0) s1; (2,0), (-2,0) s3
    // DMI: (1,0) d_hat = (1, 0); (-1,0) d_hat = (-1, 0)
    hx = P::fma(w.j0, P::add(XC(1), XC(-1)), hx);
    hy = P::fma(w.j0, P::add(YC(1), YC(-1)), hy);
    hz = P::fma(w.j0, P::add(ZC(1), ZC(-1)), hz);
    hx = P::fma(w.j2, P::add(XC(2), XC(-2)), hx);
    hy = P::fma(w.j2, P::add(YC(2), YC(-2)), hy);
    hz = P::fma(w.j2, P::add(ZC(2), ZC(-2)), hz);
    hx = P::fma(w.dh2, P::sub(ZC(1), ZC(-1)), hx);
    hz = P::fma(w.dh2, P::sub(XC(-1), XC(1)), hz);
  } else if (D2 == 1) {  // (0,1), (-1,1) s1; (1,1), (-2,1) s2
    // DMI: (0,1) d_hat = (1/2, s3); (-1,1) d_hat = (-1/2, s3)
    const typename P::V z0m = P::add(ZC(0), ZC(-1));
    hx = P::fma(w.j0, P::add(XC(0), XC(-1)), hx);
    hy = P::fma(w.j0, P::add(YC(0), YC(-1)), hy);
    hz = P::fma(w.j0, z0m, hz);
    hx = P::fma(w.j1, P::add(XC(1), XC(-2)), hx);
    hy = P::fma(w.j1, P::add(YC(1), YC(-2)), hy);
    hz = P::fma(w.j1, P::add(ZC(1), ZC(-2)), hz);
    hx = P::fma(w.dh, P::sub(ZC(0), ZC(-1)), hx);
    hy = P::fma(w.ds, z0m, hy);
    hz = P::fma(w.dh, P::sub(XC(-1), XC(0)), hz);
    hz = P::fma(w.nds, P::add(YC(0), YC(-1)), hz);
  } else {  // D2 == 2: (-1,2) s2; (0,2), (-2,2) s3
    hx = P::fma(w.j1, XC(-1), hx);
    hy = P::fma(w.j1, YC(-1), hy);
    hz = P::fma(w.j1, ZC(-1), hz);
    hx = P::fma(w.j2, P::add(XC(0), XC(-2)), hx);
    hy = P::fma(w.j2, P::add(YC(0), YC(-2)), hy);
    hz = P::fma(w.j2, P::add(ZC(0), ZC(-2)), hz);
  }
#undef XC
#undef YC
#undef ZC
}

template <typename T, int RR, int S>
__device__ __forceinline__ void scatter(const RowP<T>& r, typename PK<T>::V (&ax)[kStrip],
                                        typename PK<T>::V (&ay)[kStrip], typename PK<T>::V (&az)[kStrip],
                                        const WP<T>& w) {
  // row RR of the walk (site rows start at RR = 2) meets site S at offset d2
  constexpr int D2 = RR - 2 - S;
  if (S >= 0 && S < kStrip && D2 >= -2 && D2 <= 2) add_row<T, D2>(r, ax[S], ay[S], az[S], w);
}

template <typename T, int RR>
__device__ __forceinline__ void scatter_row(const RowP<T>& r, typename PK<T>::V (&ax)[kStrip],
                                            typename PK<T>::V (&ay)[kStrip], typename PK<T>::V (&az)[kStrip],
                                            const WP<T>& w) {
  scatter<T, RR, RR - 4>(r, ax, ay, az, w);
  scatter<T, RR, RR - 3>(r, ax, ay, az, w);
  scatter<T, RR, RR - 2>(r, ax, ay, az, w);
  scatter<T, RR, RR - 1>(r, ax, ay, az, w);
  scatter<T, RR, RR>(r, ax, ay, az, w);
}

// Reads the three aligned column pairs (x - 2, x - 1), (x, x + 1),
// (x + 2, x + 3) of one component row and forms the two odd pairs.
template <typename T>
__device__ __forceinline__ void read_pairs(const T* p, typename PK<T>::V (&o)[5]) {
  typedef typename PK<T>::V V;
  const V a = *reinterpret_cast<const V*>(p);
  const V b = *reinterpret_cast<const V*>(p + 2);
  const V c = *reinterpret_cast<const V*>(p + 4);
  o[0] = a;
  o[1] = PK<T>::mk(a.y, b.x);
  o[2] = b;
  o[3] = PK<T>::mk(b.y, c.x);
  o[4] = c;
}

template <typename T, int RR>
struct SWalk {
  static __device__ __forceinline__ void run(const T* __restrict__ tile, int row0, int lane,
                                             typename PK<T>::V (&ax)[kStrip], typename PK<T>::V (&ay)[kStrip],
                                             typename PK<T>::V (&az)[kStrip], const WP<T>& w) {
    SWalk<T, RR - 1>::run(tile, row0, lane, ax, ay, az, w);
    RowP<T> r;
    // staged column of x - 2 is 2 lane + kPadL - 2
    const T* p = tile + (size_t)(row0 + RR) * kSX + 2 * lane + kPadL - 2;
    read_pairs<T>(p, r.x);
    read_pairs<T>(p + (size_t)kSX * kSY, r.y);
    read_pairs<T>(p + 2 * (size_t)kSX * kSY, r.z);
    scatter_row<T, RR>(r, ax, ay, az, w);
  }
};
template <typename T>
struct SWalk<T, -1> {
  static __device__ __forceinline__ void run(const T*, int, int, typename PK<T>::V (&)[kStrip],
                                             typename PK<T>::V (&)[kStrip], typename PK<T>::V (&)[kStrip],
                                             const WP<T>&) {}
};

}  // namespace

// asynchronous global -> shared copies (cp.async; 16-byte copies bypass L1)
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
__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gsrc) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(smem_dst)),
               "l"(gsrc)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

template <typename T>
__device__ __forceinline__ void cp_elem(T* dst, const T* src) {
  if constexpr (sizeof(T) == 4)
    cp_async4(dst, src);
  else
    cp_async8(dst, src);
}

// Starts the copy of vector v's staged tile: staged (ly, lx) holds lattice
// site (x0 - kPadL + lx, y0 - 2 + ly), periodic.  `vec16`: the block's
// staged columns lie inside the lattice and every staged row starts on a
// 16-byte boundary, so rows go as 16-byte copies.
template <typename T>
__device__ __forceinline__ void stage_tile(T* tile, const T* __restrict__ v, size_t N, int L1, int L2, int x0, int y0,
                                           bool vec16) {
  constexpr size_t kPlane = (size_t)kSX * kSY;
  if (vec16) {
    constexpr int kE = 16 / (int)sizeof(T);  // elements per copy
    constexpr int kCh = kSX / kE;            // copies per staged row
    for (int idx = threadIdx.x; idx < 3 * kSY * kCh; idx += blockDim.x) {
      const int comp = idx / (kSY * kCh), rem = idx - comp * (kSY * kCh);
      const int ly = rem / kCh, ch = rem - ly * kCh;
      const int gy = y0 - 2 + ly;
      const size_t g = (size_t)comp * N + (size_t)gy * L1 + (x0 - kPadL) + ch * kE;
      cp_async16(tile + comp * kPlane + (size_t)ly * kSX + ch * kE, v + g);
    }
  } else {
    for (int idx = threadIdx.x; idx < kSX * kSY; idx += blockDim.x) {
      const int ly = idx / kSX, lx = idx - ly * kSX;
      const int gx = wrap(x0 - kPadL + lx, L1), gy = wrap(y0 - 2 + ly, L2);
      const size_t g = (size_t)gy * L1 + gx;
      cp_elem(tile + idx, v + g);
      cp_elem(tile + kPlane + idx, v + N + g);
      cp_elem(tile + 2 * kPlane + idx, v + 2 * N + g);
    }
  }
  cp_async_commit();
}

// Two tile buffers: the copy of vector j + 1 runs while vector j is computed.
// m and s of the block's sites are staged once (they are read for every
// vector in the output phase).  `aligned`: L1 and the field strides are
// multiples of 16 bytes / sizeof(T) and the fields start on 16-byte
// boundaries (interior blocks then stage with 16-byte copies).
template <typename T>
__global__ void __launch_bounds__(32 * kWarpsY) hvp_strip_kernel(ModelDev md, HvpW<T> hw, const T* __restrict__ m,
                                                                 const T* __restrict__ s, const T* __restrict__ V,
                                                                 size_t ldv, T* __restrict__ HV, size_t ldhv, int nvec,
                                                                 int aligned, const int* gate, int mask) {
  if (gate && (*gate & mask)) return;
  typedef PK<T> P;
  typedef typename P::V VP;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* tiles = reinterpret_cast<T*>(smem_raw);  // [2][3][kSY][kSX]
  constexpr size_t kTileElems = 3 * (size_t)kSX * kSY;
  T* ms = tiles + 2 * kTileElems;  // [4][kTY][kTX]: m_x, m_y, m_z, s
  const int lane = threadIdx.x & 31, wy = threadIdx.x >> 5;
  const int x0 = blockIdx.x * kTX, y0 = blockIdx.y * kTY;
  const int L1 = md.L1, L2 = md.L2;
  const size_t N = md.N;
  WP<T> w;
  w.j0 = P::bc(hw.j0);
  w.j1 = P::bc(hw.j1);
  w.j2 = P::bc(hw.j2);
  w.dh = P::bc(hw.dh);
  w.dh2 = P::bc(hw.dh2);
  w.ds = P::bc(hw.ds);
  w.nds = P::bc(-hw.ds);
  const T twoK = hw.twoK;
  const bool inside = x0 >= kPadL && y0 >= 2 && x0 + kTX + kPadL <= L1 && y0 + kTY + 2 <= L2;
  const bool vec16 = aligned && inside;
  // m, s of the tile (sites outside the lattice are never read back)
  if (vec16) {
    constexpr int kE = 16 / (int)sizeof(T), kCh = kTX / kE;
    for (int idx = threadIdx.x; idx < 4 * kTY * kCh; idx += blockDim.x) {
      const int comp = idx / (kTY * kCh), rem = idx - comp * (kTY * kCh);
      const int ly = rem / kCh, ch = rem - ly * kCh;
      const size_t g = (size_t)(y0 + ly) * L1 + x0 + ch * kE;
      const T* src = comp < 3 ? m + (size_t)comp * N + g : s + g;
      cp_async16(ms + (size_t)comp * kTY * kTX + ly * kTX + ch * kE, src);
    }
  } else {
    for (int idx = threadIdx.x; idx < 4 * kTY * kTX; idx += blockDim.x) {
      const int comp = idx / (kTY * kTX), rem = idx - comp * (kTY * kTX);
      const int ly = rem / kTX, lx = rem - ly * kTX;
      const int gx = x0 + lx, gy = y0 + ly;
      if (gx < L1 && gy < L2) {
        const size_t g = (size_t)gy * L1 + gx;
        cp_elem(ms + idx, comp < 3 ? m + (size_t)comp * N + g : s + g);
      }
    }
  }
  stage_tile(tiles, V, N, L1, L2, x0, y0, vec16);
  const int x = x0 + 2 * lane;  // the thread's columns x, x + 1
  const bool pair_store = aligned && x + 1 < L1;
  for (int j = 0; j < nvec; ++j) {
    T* tile = tiles + (size_t)(j & 1) * kTileElems;
    T* hv = HV + (size_t)j * ldhv;
    if (j + 1 < nvec) {
      stage_tile(tiles + (size_t)((j + 1) & 1) * kTileElems, V + (size_t)(j + 1) * ldv, N, L1, L2, x0, y0, vec16);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    VP ax[kStrip], ay[kStrip], az[kStrip];
#pragma unroll
    for (int k = 0; k < kStrip; ++k) ax[k] = ay[k] = az[k] = P::bc((T)0);
    SWalk<T, kStrip + 3>::run(tile, wy * kStrip, lane, ax, ay, az, w);
    if (x < L1) {
#pragma unroll
      for (int k = 0; k < kStrip; ++k) {
        const int ly = wy * kStrip + k;
        const int y = y0 + ly;
        if (y >= L2) break;
        const size_t i = (size_t)y * L1 + x;
        const size_t ti = (size_t)(ly + 2) * kSX + 2 * lane + kPadL;
        const VP vx = *reinterpret_cast<const VP*>(tile + ti);
        const VP vy = *reinterpret_cast<const VP*>(tile + kSX * kSY + ti);
        const VP vz = *reinterpret_cast<const VP*>(tile + 2 * kSX * kSY + ti);
        const int mi = ly * kTX + 2 * lane;
        const VP m0 = *reinterpret_cast<const VP*>(ms + mi);
        const VP m1 = *reinterpret_cast<const VP*>(ms + kTY * kTX + mi);
        const VP m2 = *reinterpret_cast<const VP*>(ms + 2 * kTY * kTX + mi);
        const VP si = *reinterpret_cast<const VP*>(ms + 3 * kTY * kTX + mi);
        const VP nsi = P::mul(si, P::bc((T)-1));
        const VP hx = P::fma(nsi, vx, ax[k]);
        const VP hy = P::fma(nsi, vy, ay[k]);
        const VP hz = P::fma(P::sub(nsi, P::bc(twoK)), vz, az[k]);
        const VP p = P::fma(m2, hz, P::fma(m1, hy, P::mul(m0, hx)));
        const VP np = P::mul(p, P::bc((T)-1));
        const VP ox = P::fma(np, m0, hx);
        const VP oy = P::fma(np, m1, hy);
        const VP oz = P::fma(np, m2, hz);
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
  constexpr size_t kE = 16 / sizeof(T);
  auto al16 = [](const void* p) { return ((uintptr_t)p % 16) == 0; };
  const int aligned = (md.L1 % (int)kE == 0) && (nvec < 2 || (ldv % kE == 0 && ldhv % kE == 0)) && al16(m) &&
                      al16(s) && al16(V) && al16(HV);
  HvpW<T> hw;
  hw.j0 = (T)(-2.0 * md.J[0]);
  hw.j1 = (T)(md.n_shells > 1 ? -2.0 * md.J[1] : 0.0);
  hw.j2 = (T)(md.n_shells > 2 ? -2.0 * md.J[2] : 0.0);
  hw.dh = (T)md.D;
  hw.dh2 = (T)(2.0 * md.D);
  hw.ds = (T)(2.0 * md.D * 0.86602540378443864676);
  hw.twoK = (T)(2.0 * md.K);
  hvp_strip_kernel<T><<<grid, 32 * kWarpsY, smem, st>>>(md, hw, m, s, V, ldv, HV, ldhv, nvec, aligned, gate, mask);
}

template void launch_hvp_strip<float>(const ModelDev&, const float*, const float*, const float*, size_t, float*,
                                      size_t, int, const int*, int, cudaStream_t);
template void launch_hvp_strip<double>(const ModelDev&, const double*, const double*, const double*, size_t, double*,
                                       size_t, int, const int*, int, cudaStream_t);

}  // namespace moto
