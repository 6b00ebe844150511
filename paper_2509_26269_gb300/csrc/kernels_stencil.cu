// Stencil kernels: energy + Riemannian gradient, tangent HVP dispatch,
// topological charge.
//
// The hot energy / gradient and charge kernels are persistent: a grid of a
// few blocks per SM (a multiple of the 152 SMs) walks the lattice's 64 x 16
// tiles, staging tile t + grid with asynchronous copies while tile t is
// computed, and evaluates the stencil with the register strips of strip.cuh
// (the staged spins serve both as the stencil field and as the on-site m_i).
// Per-site work and block sums stay in the field precision (two-float sums
// for FP32 fields): GB300's FP64 pipe is a small fraction of its FP32 rate,
// so FP64 appears only in the last block's total.  The older 32 x 32-tile
// kernel below evaluates the energy in FP64 arithmetic (moto_energy) and the
// Euclidean gradient of the autograd path.
#include <algorithm>
#include <mutex>
#include <vector>

#include "internal.h"
#include "stencil.cuh"
#include "strip.cuh"

namespace moto {

namespace {

template <typename T>
__device__ __forceinline__ T ld(const T* p) {
  return __ldg(p);
}

// Last-block reduction of two per-block values: a sum (slot 0) and a max
// (slot 1), in block-index order.
__device__ void finish_sum_max(const double* part, int nblocks, double* out, double sum_scale) {
  __shared__ double red[2 * 8];
  double a = 0.0, b = 0.0;
  for (int k = threadIdx.x; k < nblocks; k += blockDim.x) {
    a += __ldcg(part + 2 * k);
    b = fmax(b, __ldcg(part + 2 * k + 1));
  }
  double v[1] = {a};
  block_sum<1>(v, red);
  const double mx = block_max(b, red + 8);
  if (threadIdx.x == 0) {
    out[0] = v[0] * sum_scale;
    out[1] = mx;
  }
}

}  // namespace

// grad_i E = h_i(m) - muB z - 2 K m_iz z;  s_i = m_i . grad_i E;
// g_i = grad_i E - s_i m_i;  E = sum_i (s_i - muB m_iz) / 2 (E is quadratic in
// m: E = m^T (grad E + b) / 2 with b = -muB z summed over sites).  With euclid
// set, g receives grad_i E itself and out[1] its largest per-site norm.
template <typename T, typename A>
__global__ void __launch_bounds__(kThreads) energy_grad_kernel(ModelDev md, const T* __restrict__ m,
                                                               T* __restrict__ g, T* __restrict__ s,
                                                               double* part, unsigned* counter, double* out,
                                                               int* status, int euclid, size_t ws) {
  m = wofs(m, ws);
  g = wofs(g, ws);
  s = wofs(s, ws);
  part = wofs(part, ws);
  counter = wofs(counter, ws);
  out = wofs(out, ws);
  status = wofs(status, ws);
  __shared__ Tile<T> tile;
  const int x0 = blockIdx.x * kTileX, y0 = blockIdx.y * kTileY;
  load_tile(m, md.N, md.L1, md.L2, x0, y0, tile);
  __syncthreads();
  const int lx = threadIdx.x & 31, wy = threadIdx.x >> 5;
  // the thread's few sites are summed in the arithmetic precision A, the
  // block and the grid in FP64
  A esumA = (A)0, gmaxA = (A)0;
  bool bad = false;
  const size_t N = md.N;
#pragma unroll
  for (int r = 0; r < kTileRowsPerThread; ++r) {
    const int ly = wy * kTileRowsPerThread + r;
    const int gx = x0 + lx, gy = y0 + ly;
    if (gx < md.L1 && gy < md.L2) {
      A hx, hy, hz;
      linear_field<A>(md, tile, lx, ly, hx, hy, hz);
      const A mx = (A)tile.v[0][ly + kHalo][lx + kHalo];
      const A my = (A)tile.v[1][ly + kHalo][lx + kHalo];
      const A mz = (A)tile.v[2][ly + kHalo][lx + kHalo];
      hz += (A)(-md.muB) - (A)(2.0 * md.K) * mz;
      const A si = mx * hx + my * hy + mz * hz;
      const A pr = euclid ? (A)0 : si;
      const A gxv = hx - pr * mx, gyv = hy - pr * my, gzv = hz - pr * mz;
      const size_t i = (size_t)gy * md.L1 + gx;
      if (g) {
        g[i] = (T)gxv;
        g[N + i] = (T)gyv;
        g[2 * N + i] = (T)gzv;
      }
      if (s) s[i] = (T)si;
      esumA += (A)0.5 * (si - (A)md.muB * mz);
      gmaxA = fmax(gmaxA, gxv * gxv + gyv * gyv + gzv * gzv);
      bad |= !finite3(gxv, gyv, gzv);
    }
  }
  double esum = (double)esumA, gmax = (double)gmaxA;
  __shared__ double red[16];
  double v[1] = {esum};
  block_sum<1>(v, red);
  gmax = block_max(gmax, red + 8);
  const int nblocks = gridDim.x * gridDim.y;
  const int bid = blockIdx.y * gridDim.x + blockIdx.x;
  if (bad) atomicOr(status, kStatusNonfinite);
  if (!out) return;
  if (threadIdx.x == 0) {
    part[2 * bid] = v[0];
    part[2 * bid + 1] = gmax;
  }
  // grid_last_block uses gridDim.x only; flatten the check here
  __shared__ bool last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = (atomicAdd(counter, 1u) == (unsigned)nblocks - 1);
  __syncthreads();
  if (!last) return;
  __threadfence();
  finish_sum_max(part, nblocks, out, 1.0);
  if (threadIdx.x == 0) {
    out[1] = sqrt(out[1]);
    *counter = 0u;
  }
}

// (H v)_i = P_i [ h_i(v) - 2 K v_iz z - s_i v_i ] for nvec vectors.
template <typename T>
__global__ void __launch_bounds__(kThreads) hvp_kernel(ModelDev md, const T* __restrict__ m,
                                                       const T* __restrict__ s, const T* __restrict__ V,
                                                       size_t ldv, T* __restrict__ HV, size_t ldhv, int nvec,
                                                       const int* gate, int mask) {
  if (gate && (*gate & mask)) return;
  __shared__ Tile<T> tile;
  const int x0 = blockIdx.x * kTileX, y0 = blockIdx.y * kTileY;
  const int lx = threadIdx.x & 31, wy = threadIdx.x >> 5;
  const size_t N = md.N;
  T mr[kTileRowsPerThread][3], sr[kTileRowsPerThread];
  bool in[kTileRowsPerThread];
#pragma unroll
  for (int r = 0; r < kTileRowsPerThread; ++r) {
    const int gx = x0 + lx, gy = y0 + wy * kTileRowsPerThread + r;
    in[r] = gx < md.L1 && gy < md.L2;
    const size_t i = in[r] ? (size_t)gy * md.L1 + gx : 0;
    mr[r][0] = ld(m + i);
    mr[r][1] = ld(m + N + i);
    mr[r][2] = ld(m + 2 * N + i);
    sr[r] = ld(s + i);
  }
  for (int j = 0; j < nvec; ++j) {
    const T* v = V + (size_t)j * ldv;
    T* hv = HV + (size_t)j * ldhv;
    if (j > 0) __syncthreads();
    load_tile(v, md.N, md.L1, md.L2, x0, y0, tile);
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kTileRowsPerThread; ++r) {
      if (!in[r]) continue;
      const int ly = wy * kTileRowsPerThread + r;
      T hx, hy, hz;
      linear_field<T>(md, tile, lx, ly, hx, hy, hz);
      const T vx = tile.v[0][ly + kHalo][lx + kHalo];
      const T vy = tile.v[1][ly + kHalo][lx + kHalo];
      const T vz = tile.v[2][ly + kHalo][lx + kHalo];
      hz -= (T)(2.0 * md.K) * vz;
      hx -= sr[r] * vx;
      hy -= sr[r] * vy;
      hz -= sr[r] * vz;
      const T p = mr[r][0] * hx + mr[r][1] * hy + mr[r][2] * hz;
      const size_t i = (size_t)(y0 + ly) * md.L1 + (x0 + lx);
      hv[i] = hx - p * mr[r][0];
      hv[N + i] = hy - p * mr[r][1];
      hv[2 * N + i] = hz - p * mr[r][2];
    }
  }
}

// (hess E v)_i = h_i(v) - 2 K v_iz z for nvec vectors: the Euclidean Hessian
// of the quadratic energy, the same at every m (no projection, no s term).
template <typename T>
__global__ void __launch_bounds__(kThreads) euclid_hvp_kernel(ModelDev md, const T* __restrict__ V, size_t ldv,
                                                              T* __restrict__ HV, size_t ldhv, int nvec) {
  __shared__ Tile<T> tile;
  const int x0 = blockIdx.x * kTileX, y0 = blockIdx.y * kTileY;
  const int lx = threadIdx.x & 31, wy = threadIdx.x >> 5;
  const size_t N = md.N;
  for (int j = 0; j < nvec; ++j) {
    const T* v = V + (size_t)j * ldv;
    T* hv = HV + (size_t)j * ldhv;
    if (j > 0) __syncthreads();
    load_tile(v, md.N, md.L1, md.L2, x0, y0, tile);
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kTileRowsPerThread; ++r) {
      const int ly = wy * kTileRowsPerThread + r;
      if (x0 + lx >= md.L1 || y0 + ly >= md.L2) continue;
      T hx, hy, hz;
      linear_field<T>(md, tile, lx, ly, hx, hy, hz);
      hz -= (T)(2.0 * md.K) * tile.v[2][ly + kHalo][lx + kHalo];
      const size_t i = (size_t)(y0 + ly) * md.L1 + (x0 + lx);
      hv[i] = hx;
      hv[N + i] = hy;
      hv[2 * N + i] = hz;
    }
  }
}

// ---------------------------------------------------------------------------
// persistent strip kernels
// ---------------------------------------------------------------------------
namespace {

// on-site hook of the energy walk: keeps the spins of the strip's sites
template <typename T, int SW>
struct SpinsOnSite {
  typename strip::PK<T>::V mx[SW], my[SW], mz[SW];
  template <int S>
  __device__ __forceinline__ void center(const strip::RowP<T>& r, typename strip::PK<T>::V&,
                                         typename strip::PK<T>::V&, typename strip::PK<T>::V&) {
    mx[S] = r.x[2];
    my[S] = r.y[2];
    mz[S] = r.z[2];
  }
};

__device__ __forceinline__ void tile_origin(int t, int ntx, int ty_sites, int& x0, int& y0) {
  const int ty = t / ntx;
  x0 = (t - ty * ntx) * strip::kTX;
  y0 = ty * ty_sites;
}

// Tile ring of the persistent kernels: tile t + i grid is staged in buffer
// (it + i) % NST, so NST - 1 tiles are in flight while one is used.
// tc: the 16-byte copies' offsets relative to a tile's origin, computed once
// per block (interior tiles add the origin's offset to the field pointer)
template <typename T, int TY, class TC>
__device__ __forceinline__ void stage_one(T* tiles, const T* m, size_t N, int L1, int L2, int ntx, int t, int buf,
                                          int aligned, const TC& tc) {
  int x0, y0;
  tile_origin(t, ntx, TY, x0, y0);
  T* dst = tiles + (size_t)buf * strip::Dims<TY>::kTile;
  if (aligned && strip::tile_inside<TY>(x0, y0, L1, L2))
    tc.stage(dst, m + (size_t)(y0 - 2) * L1 + (x0 - strip::kPadL));
  else
    strip::stage_tile<T, strip::Dims<TY>::SY>(dst, m, N, L1, L2, x0, y0, false);
}

// the first NST - 1 tiles of the block
template <int NST, typename T, int TY, class TC>
__device__ __forceinline__ void stage_prologue(T* tiles, const T* m, size_t N, int L1, int L2, int ntx, int ntiles,
                                               int t0, int aligned, const TC& tc) {
#pragma unroll
  for (int i = 0; i < NST - 1; ++i) {
    const int t = t0 + i * (int)gridDim.x;
    if (t < ntiles) stage_one<T, TY>(tiles, m, N, L1, L2, ntx, t, i, aligned, tc);
  }
}

// Before using tile t (the block's it-th): stage the tile NST - 1 iterations
// ahead (its buffer was released by the barrier at the end of the previous
// iteration), then wait until tile t has landed: the copy groups issued after
// it may stay pending.
template <int NST, typename T, int TY, class TC>
__device__ __forceinline__ void stage_next(T* tiles, const T* m, size_t N, int L1, int L2, int ntx, int ntiles, int t,
                                           int it, int aligned, const TC& tc) {
  static_assert(NST >= 2 && NST <= 3, "two or three staged tiles");
  const int ahead = t + (NST - 1) * (int)gridDim.x;
  if (ahead < ntiles) stage_one<T, TY>(tiles, m, N, L1, L2, ntx, ahead, (it + NST - 1) % NST, aligned, tc);
  const int later = (ntiles - 1 - t) / (int)gridDim.x;  // tiles of this block after t
  const int pend = later < NST - 1 ? later : NST - 1;
  if (pend >= 2)
    strip::cp_async_wait<2>();
  else if (pend == 1)
    strip::cp_async_wait<1>();
  else
    strip::cp_async_wait<0>();
}

// Fixed-order sum of one value per thread over the block (result in thread
// 0): a shuffle tree per warp, then the warps in order.
template <typename R>
__device__ __forceinline__ R block_total(R v, R* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = radd(v, rshfl(v, o));
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  if (threadIdx.x == 0)
    for (int i = 1; i < nw; ++i) v = radd(v, sh[i]);
  __syncthreads();
  return v;
}

template <typename T>
__device__ __forceinline__ T block_maxv(T v, T* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  if (threadIdx.x == 0)
    for (int i = 1; i < nw; ++i) v = max(v, sh[i]);
  __syncthreads();
  return v;
}

// Last block: totals of the per-block partials, in an order fixed by (nb,
// blockDim): thread t adds blocks t, t + blockDim, ... in order, then the
// block tree.  Sums come as R (two-float or FP64), maxima as T.
template <typename T>
__device__ __forceinline__ void last_block_totals(const typename strip::Red<T>::R* psum, const double* pmax, int nb,
                                                  double* out_sum, double* out_max) {
  typedef strip::Red<T> RD;
  typedef typename RD::R R;
  __shared__ R shr[32];
  __shared__ double shm[32];
  R a = RD::of((T)0);
  double mx = 0.0;
  // eight blocks' partials in flight at a time (L2 latency, not arithmetic,
  // bounds this loop), added in block order
  int b = threadIdx.x;
  for (; b + 7 * (int)blockDim.x < nb; b += 8 * (int)blockDim.x) {
    R v[8];
    double w[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      v[u] = psum[b + u * blockDim.x];
      w[u] = pmax ? __ldcg(pmax + b + u * blockDim.x) : 0.0;
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      a = radd(a, v[u]);
      mx = fmax(mx, w[u]);
    }
  }
  for (; b < nb; b += blockDim.x) {
    a = radd(a, psum[b]);
    if (pmax) mx = fmax(mx, __ldcg(pmax + b));
  }
  a = block_total<R>(a, shr);
  if (pmax) mx = block_maxv<double>(mx, shm);
  if (threadIdx.x == 0) {
    *out_sum = RD::value(a);
    if (out_max) *out_max = mx;
  }
}

}  // namespace

// Energy and Riemannian gradient (the hot path: arithmetic in the field
// precision).  grad_i E = h_i(m) - muB z - 2 K m_iz z; s_i = m_i . grad_i E;
// g_i = grad_i E - s_i m_i; E = sum_i (s_i - muB m_iz) / 2 (E is quadratic in
// m).  out = [E, max_i |g_i|].  Partials: part[0 .. grid) the block energies
// (8-byte reduction values), part[grid .. 2 grid) the block maxima of |g|^2.
template <typename T, int SW, int WY, int NST, int MINB, int AR>
__global__ void __launch_bounds__(32 * WY, MINB) energy_grad_strip_kernel(ModelDev md, strip::Weights<T> hw, T muB,
                                                                    const T* __restrict__ m, T* __restrict__ g,
                                                                    T* __restrict__ s, double* part, unsigned* counter,
                                                                    double* out, int* status, int aligned, int ntx,
                                                                    int ntiles, size_t ws) {
  m = wofs(m, ws);
  g = wofs(g, ws);
  s = wofs(s, ws);
  part = wofs(part, ws);
  counter = wofs(counter, ws);
  out = wofs(out, ws);
  status = wofs(status, ws);
  using namespace strip;
  constexpr int TY = SW * WY;
  typedef Dims<TY> DM;
  typedef typename PA<T, AR>::P P;
  typedef typename PK<T>::V VP;
  typedef Red<T> RD;
  typedef typename RD::R R;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* tiles = reinterpret_cast<T*>(smem_raw);  // [NST][3][SY][kSX]
  __shared__ R shr[WY];
  __shared__ T shm[WY];
  const int lane = threadIdx.x & 31, wy = threadIdx.x >> 5;
  const int L1 = md.L1, L2 = md.L2;
  const size_t N = md.N;
  const WP<T> w(hw);
  const VP nmuB = P::bc(-muB), n2K = P::bc(-hw.twoK), half = P::bc((T)0.5), neg = P::bc((T)-1);
  R eacc = RD::of((T)0);
  T gmax = (T)0;
  bool bad = false;
  int t = blockIdx.x, x0, y0;
  TileCopies<T, DM::SY, 32 * WY> tc;
  tc.init(N, L1, kPadL, 2);  // offsets relative to a tile's origin
  stage_prologue<NST, T, TY>(tiles, m, N, L1, L2, ntx, ntiles, t, aligned, tc);
  for (int it = 0; t < ntiles; ++it, t += gridDim.x) {
    stage_next<NST, T, TY>(tiles, m, N, L1, L2, ntx, ntiles, t, it, aligned, tc);
    __syncthreads();
    tile_origin(t, ntx, TY, x0, y0);
    SpinsOnSite<T, SW> os;
    VP ax[SW], ay[SW], az[SW];
    walk<T, SW, DM::SY, P>(tiles + (size_t)(it % NST) * DM::kTile, wy * SW, lane, ax, ay, az, w, os);
    const int x = x0 + 2 * lane;
    const bool two = x + 1 < L1;
    const bool pair_store = aligned && two;
    T etile = (T)0;
    if (x < L1) {
#pragma unroll
      for (int k = 0; k < SW; ++k) {
        const int y = y0 + wy * SW + k;
        if (y >= L2) break;
        const VP m0 = os.mx[k], m1 = os.my[k], m2 = os.mz[k];
        const VP hx = ax[k], hy = ay[k];
        const VP hz = P::add(P::fma(n2K, m2, az[k]), nmuB);
        const VP si = P::fma(m2, hz, P::fma(m1, hy, P::mul(m0, hx)));
        const VP nsi = P::mul(si, neg);
        const VP gx = P::fma(nsi, m0, hx), gy = P::fma(nsi, m1, hy), gz = P::fma(nsi, m2, hz);
        const size_t i = (size_t)y * L1 + x;
        if (pair_store) {
          if (g) {
            *reinterpret_cast<VP*>(g + i) = gx;
            *reinterpret_cast<VP*>(g + N + i) = gy;
            *reinterpret_cast<VP*>(g + 2 * N + i) = gz;
          }
          if (s) *reinterpret_cast<VP*>(s + i) = si;
        } else {
          if (g) {
            g[i] = gx.x;
            g[N + i] = gy.x;
            g[2 * N + i] = gz.x;
          }
          if (s) s[i] = si.x;
          if (two) {
            if (g) {
              g[i + 1] = gx.y;
              g[N + i + 1] = gy.y;
              g[2 * N + i + 1] = gz.y;
            }
            if (s) s[i + 1] = si.y;
          }
        }
        const VP e = P::mul(half, P::fma(nmuB, m2, si));
        const VP g2 = P::fma(gz, gz, P::fma(gy, gy, P::mul(gx, gx)));
        etile += e.x;
        gmax = max(gmax, g2.x);
        bad |= !isfinite(g2.x);
        if (two) {
          etile += e.y;
          gmax = max(gmax, g2.y);
          bad |= !isfinite(g2.y);
        }
      }
    }
    eacc = radd(eacc, RD::of(etile));
    // every warp is done with this buffer before the copy of tile t + 2 grid
    // (issued in the next iteration) overwrites it
    __syncthreads();
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(status, kStatusNonfinite);
  if (!out) return;
  eacc = block_total<R>(eacc, shr);
  gmax = block_maxv<T>(gmax, shm);
  const int nb = gridDim.x;
  if (threadIdx.x == 0) {
    reinterpret_cast<R*>(part)[blockIdx.x] = eacc;
    part[nb + blockIdx.x] = (double)gmax;
  }
  if (!grid_last_block(counter)) return;
  last_block_totals<T>(reinterpret_cast<const R*>(part), part + nb, nb, out, out + 1);
  if (threadIdx.x == 0) {
    out[1] = sqrt(out[1]);
    *counter = 0u;
  }
}

// Berg-Luescher charge: per site the up triangle (i, i+a1, i+a2) and the down
// triangle (i+a1, i+a1+a2, i+a2), Omega = 2 atan2(a.(b x c), 1 + a.b + b.c +
// c.a), Q = -(1/4 pi) sum Omega.  Solid angles and the thread's sums in the
// field precision, block and grid sums as two-float (FP32) or FP64.
template <typename T>
__device__ __forceinline__ T solid_angle(T ax, T ay, T az, T bx, T by, T bz, T cx, T cy, T cz) {
  const T num = ax * (by * cz - bz * cy) + ay * (bz * cx - bx * cz) + az * (bx * cy - by * cx);
  const T den = (T)1 + (ax * bx + ay * by + az * bz) + (bx * cx + by * cy + bz * cz) + (cx * ax + cy * ay + cz * az);
  return (T)2 * atan2(num, den);
}

template <typename T, int SW, int WY, int NST, int MINB>
__global__ void __launch_bounds__(32 * WY, MINB) topo_strip_kernel(ModelDev md, const T* __restrict__ m, double* part,
                                                             unsigned* counter, double* out, int aligned, int ntx,
                                                             int ntiles, size_t ws) {
  m = wofs(m, ws);
  part = wofs(part, ws);
  counter = wofs(counter, ws);
  out = wofs(out, ws);
  using namespace strip;
  constexpr int TY = SW * WY;
  typedef Dims<TY> DM;
  typedef Red<T> RD;
  typedef typename RD::R R;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* tiles = reinterpret_cast<T*>(smem_raw);
  __shared__ R shr[WY];
  const int lane = threadIdx.x & 31, wy = threadIdx.x >> 5;
  const int L1 = md.L1, L2 = md.L2;
  const size_t N = md.N;
  R acc = RD::of((T)0);
  int t = blockIdx.x, x0, y0;
  TileCopies<T, DM::SY, 32 * WY> tc;
  tc.init(N, L1, kPadL, 2);  // offsets relative to a tile's origin
  stage_prologue<NST, T, TY>(tiles, m, N, L1, L2, ntx, ntiles, t, aligned, tc);
  for (int it = 0; t < ntiles; ++it, t += gridDim.x) {
    stage_next<NST, T, TY>(tiles, m, N, L1, L2, ntx, ntiles, t, it, aligned, tc);
    __syncthreads();
    tile_origin(t, ntx, TY, x0, y0);
    const T* tile = tiles + (size_t)(it % NST) * DM::kTile;
    const int x = x0 + 2 * lane;
    T qt = (T)0;
    if (x < L1) {
      const bool two = x + 1 < L1;
      // staged column of x is 2 lane + kPadL, staged row of y is y - y0 + 2;
      // the walk holds columns x, x + 1, x + 2 of the current and next rows
      T c[2][3][3];
      const int lx = 2 * lane + kPadL;
#pragma unroll
      for (int k = 0; k <= SW; ++k) {
        const int ly = wy * SW + k + 2;
        const int cur = k & 1;
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          const T* row = tile + (size_t)q * DM::kPlane + (size_t)ly * kSX + lx;
          const typename PK<T>::V p01 = *reinterpret_cast<const typename PK<T>::V*>(row);
          c[cur][q][0] = p01.x;
          c[cur][q][1] = p01.y;
          c[cur][q][2] = row[2];
        }
        if (k > 0) {
          const int y = y0 + wy * SW + k - 1;
          if (y < L2) {
            const int pr = cur ^ 1;  // row y; cur holds row y + 1
#define M_(r, col) c[r][0][col], c[r][1][col], c[r][2][col]
            qt += solid_angle<T>(M_(pr, 0), M_(pr, 1), M_(cur, 0)) + solid_angle<T>(M_(pr, 1), M_(cur, 1), M_(cur, 0));
            if (two)
              qt += solid_angle<T>(M_(pr, 1), M_(pr, 2), M_(cur, 1)) +
                    solid_angle<T>(M_(pr, 2), M_(cur, 2), M_(cur, 1));
#undef M_
          }
        }
      }
    }
    acc = radd(acc, RD::of(qt));
    __syncthreads();
  }
  acc = block_total<R>(acc, shr);
  const int nb = gridDim.x;
  if (threadIdx.x == 0) reinterpret_cast<R*>(part)[blockIdx.x] = acc;
  if (!grid_last_block(counter)) return;
  double q = 0.0;
  last_block_totals<T>(reinterpret_cast<const R*>(part), nullptr, nb, &q, nullptr);
  if (threadIdx.x == 0) {
    out[0] = -q / (4.0 * 3.14159265358979323846);
    *counter = 0u;
  }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
static dim3 tile_grid(const ModelDev& md) {
  return dim3((md.L1 + kTileX - 1) / kTileX, (md.L2 + kTileY - 1) / kTileY);
}

// persistent strip kernels: at most this many blocks an SM
constexpr int kStripMaxBps = 8;
constexpr int kStripSW = 4, kStripWY = 4;  // 64 x 16-site tiles, 128 threads

long long stencil_blocks(int L1, int L2) {
  const long long old_tiles = (((long long)L1 + kTileX - 1) / kTileX) * (((long long)L2 + kTileY - 1) / kTileY);
  const long long strip_tiles = (((long long)L1 + strip::kTX - 1) / strip::kTX) *
                                (((long long)L2 + kStripSW * kStripWY - 1) / (kStripSW * kStripWY));
  return std::max(old_tiles, std::min(strip_tiles, (long long)kSMs * kStripMaxBps));
}

int tile_blocks(const ModelDev& md) { return (int)stencil_blocks(md.L1, md.L2); }

namespace {

// Blocks an SM of a persistent strip kernel (occupancy with its shared
// memory, at most kStripMaxBps), queried once per kernel.
template <typename K>
int strip_bps(K kernel, int threads, size_t smem, int& cache) {
  if (cache == 0) {
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kernel, threads, smem) != cudaSuccess || b < 1) b = 1;
    cache = std::min(b, kStripMaxBps);
  }
  return cache;
}

template <typename T>
bool al16(const void* p) {
  return p == nullptr || ((uintptr_t)p % 16) == 0;
}

// The persistent stencils' variants: (staged tiles, blocks an SM the
// registers must allow, FP32 pair arithmetic: PA).  The per-site arithmetic
// is the same in all; the block partition, and so the order of the energy's
// sum, follows the grid.
template <typename T, int NST, int MINB, int AR0>
void energy_strip_v(const ModelDev& md, const T* m, T* g, T* s, double* part, unsigned* counter, double* out,
                    int* status, cudaStream_t st) {
  constexpr int AR = sizeof(T) == 4 ? AR0 : 1;  // FP64 pairs are scalar in every form
  constexpr int SW = kStripSW, WY = kStripWY, TY = SW * WY;
  const int ntx = (md.L1 + strip::kTX - 1) / strip::kTX, nty = (md.L2 + TY - 1) / TY;
  const int ntiles = ntx * nty;
  const size_t smem = NST * strip::Dims<TY>::kTile * sizeof(T);
  static int bps_cache = 0;
  const int bps = strip_bps(energy_grad_strip_kernel<T, SW, WY, NST, MINB, AR>, 32 * WY, smem, bps_cache);
  const int grid = std::min(ntiles, kSMs * bps);
  constexpr int kE = 16 / (int)sizeof(T);
  const int aligned = (md.L1 % kE == 0) && al16<T>(m) && al16<T>(g) && al16<T>(s);
  energy_grad_strip_kernel<T, SW, WY, NST, MINB, AR><<<wgrid(grid), 32 * WY, smem, st>>>(
      md, strip::make_weights<T>(md), (T)md.muB, m, g, s, part, counter, out, status, aligned, ntx, ntiles,
      walker_ws());
}

template <typename T, int NST, int MINB>
void topo_strip_v(const ModelDev& md, const T* m, double* part, unsigned* counter, double* out, cudaStream_t st) {
  constexpr int SW = kStripSW, WY = kStripWY, TY = SW * WY;
  const int ntx = (md.L1 + strip::kTX - 1) / strip::kTX, nty = (md.L2 + TY - 1) / TY;
  const int ntiles = ntx * nty;
  const size_t smem = NST * strip::Dims<TY>::kTile * sizeof(T);
  static int bps_cache = 0;
  const int bps = strip_bps(topo_strip_kernel<T, SW, WY, NST, MINB>, 32 * WY, smem, bps_cache);
  const int grid = std::min(ntiles, kSMs * bps);
  constexpr int kE = 16 / (int)sizeof(T);
  const int aligned = (md.L1 % kE == 0) && al16<T>(m);
  topo_strip_kernel<T, SW, WY, NST, MINB><<<wgrid(grid), 32 * WY, smem, st>>>(md, m, part, counter, out, aligned,
                                                                             ntx, ntiles, walker_ws());
}

// Process-wide choices of the autotuner: (L1, L2, element size) -> variant.
struct StencilChoice {
  int L1, L2, esize, variant;
};
std::mutex g_stencil_mutex;
std::vector<StencilChoice> g_stencil_choices;

int stencil_choice(int L1, int L2, int esize) {
  std::lock_guard<std::mutex> lock(g_stencil_mutex);
  for (const StencilChoice& c : g_stencil_choices)
    if (c.L1 == L1 && c.L2 == L2 && c.esize == esize) return c.variant;
  return -1;
}

template <typename T>
void launch_energy_grad_strip(const ModelDev& md, const T* m, T* g, T* s, double* part, unsigned* counter,
                              double* out, int* status, cudaStream_t st, int variant) {
  if (variant < 0) variant = std::max(0, stencil_choice(md.L1, md.L2, (int)sizeof(T)));
  switch (variant) {
    case 1: energy_strip_v<T, 2, 5, 0>(md, m, g, s, part, counter, out, status, st); break;
    case 2: energy_strip_v<T, 3, 1, 1>(md, m, g, s, part, counter, out, status, st); break;
    case 3: energy_strip_v<T, 2, 5, 1>(md, m, g, s, part, counter, out, status, st); break;
    default: energy_strip_v<T, 3, 1, 0>(md, m, g, s, part, counter, out, status, st); break;
  }
}

}  // namespace

template <typename T>
void launch_energy_grad(const ModelDev& md, const T* m, T* g, T* s, double* part, unsigned* counter, double* out,
                        int* status, bool fp64_arith, cudaStream_t st, bool euclid) {
  if (md.npairs > 0) {
    launch_pair_energy_grad<T>(md, m, g, s, part, counter, out, status, fp64_arith, euclid, st);
    return;
  }
  if (!fp64_arith && !euclid) {
    launch_energy_grad_strip<T>(md, m, g, s, part, counter, out, status, st, -1);
    return;
  }
  const int e = euclid ? 1 : 0;
  if (fp64_arith)
    energy_grad_kernel<T, double><<<wgrid(tile_grid(md)), kThreads, 0, st>>>(md, m, g, s, part, counter, out, status, e, walker_ws());
  else
    energy_grad_kernel<T, T><<<wgrid(tile_grid(md)), kThreads, 0, st>>>(md, m, g, s, part, counter, out, status, e, walker_ws());
}

template <typename T>
void launch_euclid_hvp(const ModelDev& md, const T* V, size_t ldv, T* HV, size_t ldhv, int nvec, cudaStream_t st) {
  if (md.npairs > 0) {
    launch_pair_hvp<T>(md, nullptr, nullptr, V, ldv, HV, ldhv, nvec, true, nullptr, 0, st);
    return;
  }
  euclid_hvp_kernel<T><<<tile_grid(md), kThreads, 0, st>>>(md, V, ldv, HV, ldhv, nvec);
}

template <typename T>
void launch_hvp(const ModelDev& md, const T* m, const T* s, const T* V, size_t ldv, T* HV, size_t ldhv, int nvec,
                const int* gate, int mask, cudaStream_t st) {
  if (md.npairs > 0) {
    launch_pair_hvp<T>(md, m, s, V, ldv, HV, ldhv, nvec, false, gate, mask, st);
    return;
  }
  launch_hvp_strip<T>(md, m, s, V, ldv, HV, ldhv, nvec, gate, mask, st);
}

template <typename T>
void launch_topo(const ModelDev& md, const T* m, double* part, unsigned* counter, double* out, cudaStream_t st) {
  // the charge has no pair walk: variants 1 and 3 share its two-tile layout
  const int v = stencil_choice(md.L1, md.L2, (int)sizeof(T));
  if (v == 1 || v == 3)
    topo_strip_v<T, 2, 5>(md, m, part, counter, out, st);
  else
    topo_strip_v<T, 3, 1>(md, m, part, counter, out, st);
}

int stencil_variant_count() { return 4; }
int stencil_tuned_variant(int L1, int L2, int esize) { return stencil_choice(L1, L2, esize); }
void stencil_record_variant(int L1, int L2, int esize, int variant) {
  std::lock_guard<std::mutex> lock(g_stencil_mutex);
  for (StencilChoice& c : g_stencil_choices)
    if (c.L1 == L1 && c.L2 == L2 && c.esize == esize) {
      c.variant = variant;
      return;
    }
  g_stencil_choices.push_back(StencilChoice{L1, L2, esize, variant});
}

template <typename T>
void launch_energy_grad_variant(int variant, const ModelDev& md, const T* m, T* g, T* s, double* part,
                                unsigned* counter, double* out, int* status, cudaStream_t st) {
  launch_energy_grad_strip<T>(md, m, g, s, part, counter, out, status, st, variant);
}

#define INST(T)                                                                                               \
  template void launch_energy_grad<T>(const ModelDev&, const T*, T*, T*, double*, unsigned*, double*, int*,  \
                                      bool, cudaStream_t, bool);                                              \
  template void launch_euclid_hvp<T>(const ModelDev&, const T*, size_t, T*, size_t, int, cudaStream_t);      \
  template void launch_hvp<T>(const ModelDev&, const T*, const T*, const T*, size_t, T*, size_t, int,        \
                              const int*, int, cudaStream_t);                                                 \
  template void launch_topo<T>(const ModelDev&, const T*, double*, unsigned*, double*, cudaStream_t);        \
  template void launch_energy_grad_variant<T>(int, const ModelDev&, const T*, T*, T*, double*, unsigned*,    \
                                              double*, int*, cudaStream_t);
INST(float)
INST(double)
#undef INST

}  // namespace moto
