// Stencil kernels: energy + Riemannian gradient, tangent HVP, topological charge.
//
// Every kernel maps one 32 x 32 tile of sites to a 256-thread block (warp w
// owns rows 4w..4w+3, lane = column), stages the field it differentiates in a
// shared-memory tile with a 2-site periodic halo, and keeps the on-site
// vectors (m_i, s_i) in registers.
#include "internal.h"
#include "stencil.cuh"

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
                                                               int* status, int euclid) {
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

// Berg-Luescher charge: per site the up triangle (i, i+a1, i+a2) and the down
// triangle (i+a1, i+a1+a2, i+a2); Omega = 2 atan2(a.(b x c), 1+a.b+b.c+c.a);
// Q = -(1/4 pi) sum Omega.
template <typename T, typename A>
__device__ __forceinline__ A solid_angle(const A* a, const A* b, const A* c) {
  const A num = a[0] * (b[1] * c[2] - b[2] * c[1]) + a[1] * (b[2] * c[0] - b[0] * c[2]) +
                a[2] * (b[0] * c[1] - b[1] * c[0]);
  const A den = (A)1 + (a[0] * b[0] + a[1] * b[1] + a[2] * b[2]) + (b[0] * c[0] + b[1] * c[1] + b[2] * c[2]) +
                (c[0] * a[0] + c[1] * a[1] + c[2] * a[2]);
  return (A)2 * atan2(num, den);
}

template <typename T>
__global__ void __launch_bounds__(kThreads) topo_kernel(ModelDev md, const T* __restrict__ m, double* part,
                                                        unsigned* counter, double* out) {
  typedef T A;
  __shared__ Tile<T> tile;
  const int x0 = blockIdx.x * kTileX, y0 = blockIdx.y * kTileY;
  load_tile(m, md.N, md.L1, md.L2, x0, y0, tile);
  __syncthreads();
  const int lx = threadIdx.x & 31, wy = threadIdx.x >> 5;
  double acc = 0.0;
#pragma unroll
  for (int r = 0; r < kTileRowsPerThread; ++r) {
    const int ly = wy * kTileRowsPerThread + r;
    if (x0 + lx < md.L1 && y0 + ly < md.L2) {
      const int cx = lx + kHalo, cy = ly + kHalo;
      A m0[3], m1[3], m2[3], m3[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        m0[c] = tile.v[c][cy][cx];
        m1[c] = tile.v[c][cy][cx + 1];
        m2[c] = tile.v[c][cy + 1][cx];
        m3[c] = tile.v[c][cy + 1][cx + 1];
      }
      acc += (double)solid_angle<T, A>(m0, m1, m2) + (double)solid_angle<T, A>(m1, m3, m2);
    }
  }
  __shared__ double red[8];
  double v[1] = {acc};
  block_sum<1>(v, red);
  const int nblocks = gridDim.x * gridDim.y;
  const int bid = blockIdx.y * gridDim.x + blockIdx.x;
  if (threadIdx.x == 0) part[bid] = v[0];
  __shared__ bool last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = (atomicAdd(counter, 1u) == (unsigned)nblocks - 1);
  __syncthreads();
  if (!last) return;
  __threadfence();
  double a = 0.0;
  for (int k = threadIdx.x; k < nblocks; k += blockDim.x) a += __ldcg(part + k);
  double w[1] = {a};
  block_sum<1>(w, red);
  if (threadIdx.x == 0) {
    out[0] = -w[0] / (4.0 * 3.14159265358979323846);
    *counter = 0u;
  }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
static dim3 tile_grid(const ModelDev& md) {
  return dim3((md.L1 + kTileX - 1) / kTileX, (md.L2 + kTileY - 1) / kTileY);
}

long long stencil_blocks(int L1, int L2) {
  return (((long long)L1 + kTileX - 1) / kTileX) * (((long long)L2 + kTileY - 1) / kTileY);
}

int tile_blocks(const ModelDev& md) { return (int)stencil_blocks(md.L1, md.L2); }

template <typename T>
void launch_energy_grad(const ModelDev& md, const T* m, T* g, T* s, double* part, unsigned* counter, double* out,
                        int* status, bool fp64_arith, cudaStream_t st, bool euclid) {
  if (md.npairs > 0) {
    launch_pair_energy_grad<T>(md, m, g, s, part, counter, out, status, fp64_arith, euclid, st);
    return;
  }
  const int e = euclid ? 1 : 0;
  if (fp64_arith)
    energy_grad_kernel<T, double><<<tile_grid(md), kThreads, 0, st>>>(md, m, g, s, part, counter, out, status, e);
  else
    energy_grad_kernel<T, T><<<tile_grid(md), kThreads, 0, st>>>(md, m, g, s, part, counter, out, status, e);
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
  topo_kernel<T><<<tile_grid(md), kThreads, 0, st>>>(md, m, part, counter, out);
}

#define INST(T)                                                                                               \
  template void launch_energy_grad<T>(const ModelDev&, const T*, T*, T*, double*, unsigned*, double*, int*,  \
                                      bool, cudaStream_t, bool);                                              \
  template void launch_euclid_hvp<T>(const ModelDev&, const T*, size_t, T*, size_t, int, cudaStream_t);      \
  template void launch_hvp<T>(const ModelDev&, const T*, const T*, const T*, size_t, T*, size_t, int,        \
                              const int*, int, cudaStream_t);                                                 \
  template void launch_topo<T>(const ModelDev&, const T*, double*, unsigned*, double*, cudaStream_t);
INST(float)
INST(double)
#undef INST

}  // namespace moto
