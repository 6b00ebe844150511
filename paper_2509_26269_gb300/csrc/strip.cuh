// Register-strip evaluation of the lattice stencil, shared by the tangent HVP
// (kernels_hvp.cu) and the energy / gradient and charge kernels
// (kernels_stencil.cu).
//
// The linear field of the spin Hamiltonian (Eq. param-hamiltonian, ordered
// pairs, Neel DMI D_ij = D z x r_hat_ij on shell 1):
//   h_i(x) = -2 sum_s J_s sum_{d in shell s} x_{i+d}
//            - 2 D sum_{d in shell 1} [ z (x_{i+d} . d_hat) - d_hat x_{i+d,z} ].
//
// A block stages a TY x 64-site tile of a field (plus a 2-site periodic halo,
// widened to 4 columns on each side so that every staged row starts on a
// 16-byte boundary) in shared memory with asynchronous copies.  A thread owns
// two adjacent columns (x, x + 1) of a strip of SW rows: it walks the SW + 4
// staged rows the strip needs, reading each row once as three aligned column
// pairs per component and forming the two odd pairs, and adds the row into
// the accumulators of the (up to five) strip sites it is a neighbour of.  In
// FP32 every add and FMA of the walk is either one packed f32x2 instruction
// for two sites or two scalar ones with the same per-lane rounding (PA; the
// launchers time both); FP64 takes the same path with scalar pairs.  The row of a site
// itself is handed to an on-site hook (the -s v and -2K v_z terms of the HVP,
// the spins of the energy kernel) before its own stencil terms, so every
// site's sum runs in the same order whatever the strip length or the number
// of warps of a block.
#pragma once

#include "common.cuh"

namespace moto {
namespace strip {

constexpr int kTX = 64;               // sites of a tile along a1
constexpr int kPadL = 4;              // staged columns left of the tile (2 halo + 2 alignment)
constexpr int kSX = kTX + 2 * kPadL;  // staged columns

// staged rows and plane size of a tile TY sites high
template <int TY>
struct Dims {
  static constexpr int SY = TY + 4;
  static constexpr size_t kPlane = (size_t)kSX * SY;
  static constexpr size_t kTile = 3 * kPlane;
};

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

// Scalar arithmetic on FP32 column pairs: per lane the same round-to-nearest
// add, sub, mul and fused multiply-add as PK<float> (the intrinsics are never
// contracted or reassociated), issued as two scalar instructions, so a walk
// gives bit-identical sums with either form.
struct PKs {
  typedef float2 V;
  static __device__ __forceinline__ V bc(float s) { return make_float2(s, s); }
  static __device__ __forceinline__ V mk(float a, float b) { return make_float2(a, b); }
  static __device__ __forceinline__ V add(V a, V b) { return make_float2(__fadd_rn(a.x, b.x), __fadd_rn(a.y, b.y)); }
  static __device__ __forceinline__ V sub(V a, V b) { return make_float2(__fsub_rn(a.x, b.x), __fsub_rn(a.y, b.y)); }
  static __device__ __forceinline__ V mul(V a, V b) { return make_float2(__fmul_rn(a.x, b.x), __fmul_rn(a.y, b.y)); }
  static __device__ __forceinline__ V fma(V a, V b, V c) {
    return make_float2(__fmaf_rn(a.x, b.x, c.x), __fmaf_rn(a.y, b.y, c.y));
  }
};

// Pair arithmetic of a walk, AR: 1 packed f32x2 instructions, 0 scalar
// pairs; FP64 pairs are always scalar.  Measured on GB300 the scalar form is
// the faster one for the HVP at large lattices: the odd column pairs a
// packed instruction needs as aligned register pairs cost moves that scalar
// operands do not (the compiler's float2 intrinsics behave like the inline
// PTX).
template <typename T, int AR>
struct PA {
  typedef PK<T> P;
};
template <>
struct PA<float, 0> {
  typedef PKs P;
};

// One staged row as seen from the column pair (x, x + 1): x[c + 2] holds the
// columns (x + c, x + 1 + c), c = -2 .. 2, of the x component (y, z alike).
template <typename T>
struct RowP {
  typename PK<T>::V x[5], y[5], z[5];
};

// Stencil weights in the field precision, formed on the host: -2 J_s per
// shell, D (= 2 D / 2), 2 D, 2 D sqrt(3)/2, and 2 K.
template <typename T>
struct Weights {
  T j0, j1, j2, dh, dh2, ds, twoK;
};

template <typename T>
Weights<T> make_weights(const ModelDev& md) {
  Weights<T> w;
  w.j0 = (T)(-2.0 * md.J[0]);
  w.j1 = (T)(md.n_shells > 1 ? -2.0 * md.J[1] : 0.0);
  w.j2 = (T)(md.n_shells > 2 ? -2.0 * md.J[2] : 0.0);
  w.dh = (T)md.D;
  w.dh2 = (T)(2.0 * md.D);
  w.ds = (T)(2.0 * md.D * 0.86602540378443864676);
  w.twoK = (T)(2.0 * md.K);
  return w;
}

// The weights as column pairs.
template <typename T>
struct WP {
  typename PK<T>::V j0, j1, j2, dh, dh2, ds, nds;
  __device__ __forceinline__ explicit WP(const Weights<T>& w) {
    typedef PK<T> P;
    j0 = P::bc(w.j0);
    j1 = P::bc(w.j1);
    j2 = P::bc(w.j2);
    dh = P::bc(w.dh);
    dh2 = P::bc(w.dh2);
    ds = P::bc(w.ds);
    nds = P::bc(-w.ds);
  }
};

// Adds to (hx, hy, hz) the contribution of a row at offset d2 (= row - site).
template <typename T, int D2, class P = PK<T>>
__device__ __forceinline__ void add_row(const RowP<T>& r, typename PK<T>::V& hx, typename PK<T>::V& hy,
                                        typename PK<T>::V& hz, const WP<T>& w) {
#define XC(c) r.x[(c) + 2]
#define YC(c) r.y[(c) + 2]
#define ZC(c) r.z[(c) + 2]
  if constexpr (D2 == -2) {  // (1,-2) s2; (0,-2), (2,-2) s3
    hx = P::fma(w.j1, XC(1), hx);
    hy = P::fma(w.j1, YC(1), hy);
    hz = P::fma(w.j1, ZC(1), hz);
    hx = P::fma(w.j2, P::add(XC(0), XC(2)), hx);
    hy = P::fma(w.j2, P::add(YC(0), YC(2)), hy);
    hz = P::fma(w.j2, P::add(ZC(0), ZC(2)), hz);
  } else if constexpr (D2 == -1) {  // (0,-1), (1,-1) s1; (-1,-1), (2,-1) s2
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
  } else if constexpr (D2 == 0) {  // (1,0), (-1,0) s1; (2,0), (-2,0) s3
    // DMI: (1,0) d_hat = (1, 0); (-1,0) d_hat = (-1, 0)
    hx = P::fma(w.j0, P::add(XC(1), XC(-1)), hx);
    hy = P::fma(w.j0, P::add(YC(1), YC(-1)), hy);
    hz = P::fma(w.j0, P::add(ZC(1), ZC(-1)), hz);
    hx = P::fma(w.j2, P::add(XC(2), XC(-2)), hx);
    hy = P::fma(w.j2, P::add(YC(2), YC(-2)), hy);
    hz = P::fma(w.j2, P::add(ZC(2), ZC(-2)), hz);
    hx = P::fma(w.dh2, P::sub(ZC(1), ZC(-1)), hx);
    hz = P::fma(w.dh2, P::sub(XC(-1), XC(1)), hz);
  } else if constexpr (D2 == 1) {  // (0,1), (-1,1) s1; (1,1), (-2,1) s2
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

// Row RR of the walk (the strip's sites are rows 2 .. SW + 1) meets strip
// site S at offset d2 = RR - 2 - S; the site's own row first goes to the hook.
template <typename T, int SW, int RR, int S, class P, class F>
__device__ __forceinline__ void scatter(const RowP<T>& r, typename PK<T>::V (&ax)[SW], typename PK<T>::V (&ay)[SW],
                                        typename PK<T>::V (&az)[SW], const WP<T>& w, F& f) {
  constexpr int D2 = RR - 2 - S;
  if constexpr (S >= 0 && S < SW && D2 >= -2 && D2 <= 2) {
    if constexpr (D2 == 0) f.template center<S>(r, ax[S], ay[S], az[S]);
    add_row<T, D2, P>(r, ax[S], ay[S], az[S], w);
  }
}

template <typename T, int SW, int RR, class P, class F>
__device__ __forceinline__ void scatter_row(const RowP<T>& r, typename PK<T>::V (&ax)[SW],
                                            typename PK<T>::V (&ay)[SW], typename PK<T>::V (&az)[SW],
                                            const WP<T>& w, F& f) {
  scatter<T, SW, RR, RR - 4, P>(r, ax, ay, az, w, f);
  scatter<T, SW, RR, RR - 3, P>(r, ax, ay, az, w, f);
  scatter<T, SW, RR, RR - 2, P>(r, ax, ay, az, w, f);
  scatter<T, SW, RR, RR - 1, P>(r, ax, ay, az, w, f);
  scatter<T, SW, RR, RR, P>(r, ax, ay, az, w, f);
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

// Walk of rows 0 .. RR of a strip starting at staged row row0 (the staged
// tile has SY rows per component plane).
template <typename T, int SW, int SY, int RR, class P>
struct SWalk {
  template <class F>
  static __device__ __forceinline__ void run(const T* __restrict__ tile, int row0, int lane,
                                             typename PK<T>::V (&ax)[SW], typename PK<T>::V (&ay)[SW],
                                             typename PK<T>::V (&az)[SW], const WP<T>& w, F& f) {
    SWalk<T, SW, SY, RR - 1, P>::run(tile, row0, lane, ax, ay, az, w, f);
    RowP<T> r;
    // staged column of x - 2 is 2 lane + kPadL - 2
    const T* p = tile + (size_t)(row0 + RR) * kSX + 2 * lane + kPadL - 2;
    read_pairs<T>(p, r.x);
    read_pairs<T>(p + (size_t)kSX * SY, r.y);
    read_pairs<T>(p + 2 * (size_t)kSX * SY, r.z);
    scatter_row<T, SW, RR, P>(r, ax, ay, az, w, f);
  }
};
template <typename T, int SW, int SY, class P>
struct SWalk<T, SW, SY, -1, P> {
  template <class F>
  static __device__ __forceinline__ void run(const T*, int, int, typename PK<T>::V (&)[SW],
                                             typename PK<T>::V (&)[SW], typename PK<T>::V (&)[SW], const WP<T>&,
                                             F&) {}
};

// The full walk of one strip: accumulators set to zero, rows 0 .. SW + 3;
// P: the pair arithmetic (PA).
template <typename T, int SW, int SY, class P = PK<T>, class F>
__device__ __forceinline__ void walk(const T* __restrict__ tile, int row0, int lane, typename PK<T>::V (&ax)[SW],
                                     typename PK<T>::V (&ay)[SW], typename PK<T>::V (&az)[SW], const WP<T>& w,
                                     F& f) {
#pragma unroll
  for (int k = 0; k < SW; ++k) ax[k] = ay[k] = az[k] = PK<T>::bc((T)0);
  SWalk<T, SW, SY, SW + 3, P>::run(tile, row0, lane, ax, ay, az, w, f);
}

// ---- asynchronous global -> shared copies (cp.async; 16-byte copies bypass L1)
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

// Periodic index for a coordinate at most one period outside [0, L) (the
// staged tiles reach a few sites past the lattice): two compares; a general
// modulo only for lattices smaller than the reach.
__device__ __forceinline__ int wrap_near(int a, int L) {
  if (a < 0) a += L;
  if (a >= L) a -= L;
  return (a >= 0 && a < L) ? a : wrap(a, L);
}

// Starts the copy of a field's staged tile: staged (ly, lx) holds lattice
// site (x0 - kPadL + lx, y0 - 2 + ly), periodic, for ly < SY.  `vec16`: the
// block's staged columns lie inside the lattice and every staged row starts
// on a 16-byte boundary, so rows go as 16-byte copies.  Commits one group.
template <typename T, int SY>
__device__ __forceinline__ void stage_tile(T* tile, const T* __restrict__ v, size_t N, int L1, int L2, int x0, int y0,
                                           bool vec16) {
  constexpr size_t kPlane = (size_t)kSX * SY;
  if (vec16) {
    constexpr int kE = 16 / (int)sizeof(T);  // elements per copy
    constexpr int kCh = kSX / kE;            // copies per staged row
    for (int idx = threadIdx.x; idx < 3 * SY * kCh; idx += blockDim.x) {
      const int comp = idx / (SY * kCh), rem = idx - comp * (SY * kCh);
      const int ly = rem / kCh, ch = rem - ly * kCh;
      const int gy = y0 - 2 + ly;
      const size_t g = (size_t)comp * N + (size_t)gy * L1 + (x0 - kPadL) + ch * kE;
      cp_async16(tile + comp * kPlane + (size_t)ly * kSX + ch * kE, v + g);
    }
  } else {
    for (int idx = threadIdx.x; idx < kSX * SY; idx += blockDim.x) {
      const int ly = idx / kSX, lx = idx - ly * kSX;
      const int gx = wrap_near(x0 - kPadL + lx, L1), gy = wrap_near(y0 - 2 + ly, L2);
      const size_t g = (size_t)gy * L1 + gx;
      cp_elem(tile + idx, v + g);
      cp_elem(tile + kPlane + idx, v + N + g);
      cp_elem(tile + 2 * kPlane + idx, v + 2 * N + g);
    }
  }
  cp_async_commit();
}

// The 16-byte copies of a staged tile whose rows lie inside the lattice
// (tile_inside), precomputed per thread: copy k of a thread is chunk
// idx = threadIdx.x + k B of the [3][SY][kSX] tile (destination idx kE
// elements in), its source offset relative to the field pointer kept in 32
// bits (3 N < 2^32: moto_create caps N at 2^30).  A block that stages the
// same tile of several fields (the HVP's vectors) computes the offsets once
// instead of two divisions and the address arithmetic per copy and field.
template <typename T, int SY, int B>
struct TileCopies {
  static constexpr int kE = 16 / (int)sizeof(T);
  static constexpr int kCh = kSX / kE;
  static constexpr int kTotal = 3 * SY * kCh;
  static constexpr int kN = (kTotal + B - 1) / B;
  uint32_t off[kN];
  __device__ __forceinline__ void init(size_t N, int L1, int x0, int y0) {
#pragma unroll
    for (int k = 0; k < kN; ++k) {
      const int idx = threadIdx.x + k * B;
      const int comp = idx / (SY * kCh), rem = idx - comp * (SY * kCh);
      const int ly = rem / kCh, ch = rem - ly * kCh;
      off[k] = (uint32_t)((size_t)comp * N + (size_t)(y0 - 2 + ly) * L1 + (x0 - kPadL) + ch * kE);
    }
  }
  // starts the copies of the tile of field v; commits one group
  __device__ __forceinline__ void stage(T* tile, const T* __restrict__ v) const {
#pragma unroll
    for (int k = 0; k < kN; ++k) {
      const int idx = threadIdx.x + k * B;
      if (k + 1 < kN || idx < kTotal) cp_async16(tile + (size_t)idx * kE, v + off[k]);
    }
    cp_async_commit();
  }
};

// Whether a tile at (x0, y0) stages with 16-byte copies.
template <int TY>
__device__ __forceinline__ bool tile_inside(int x0, int y0, int L1, int L2) {
  return x0 >= kPadL && y0 >= 2 && x0 + kTX + kPadL <= L1 && y0 + TY + 2 <= L2;
}

// Reduction type of a field precision: two-float sums for FP32 fields, FP64
// for FP64 fields.
template <typename T>
struct Red;
template <>
struct Red<float> {
  typedef F2 R;
  static __device__ __forceinline__ R of(float a) { return f2_of(a); }
  static __device__ __forceinline__ double value(R a) { return (double)a.hi + (double)a.lo; }
};
template <>
struct Red<double> {
  typedef double R;
  static __device__ __forceinline__ R of(double a) { return a; }
  static __device__ __forceinline__ double value(R a) { return a; }
};

}  // namespace strip
}  // namespace moto
