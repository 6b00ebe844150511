// Stencil kernels of a general pair-list Hamiltonian (an extension beyond the
// three-shell Neel model: the many-shell DFT parameterisations the paper
// tabulates for Pd/Fe/Ir(111) have ~20 shells and full DMI vectors)
//   E = - sum_i sum_p [ J_p m_i . m_{i+d_p} + D_p . (m_i x m_{i+d_p}) ]
//       - muB sum_i m_iz - K sum_i m_iz^2,
// the pair list closed under d -> -d with J_{-d} = J_d and D_{-d} = -D_d, so
// every bond enters twice as in Eq. param-hamiltonian.  With that closure the
// linear part of the gradient needs the +d neighbours only:
//   h_i(x) = grad_i E_lin(x) = -2 sum_p [ J_p x_{i+d_p} + x_{i+d_p} x D_p ],
// and energy, gradient, tangent HVP and the Euclidean derivatives follow
// exactly as for the shell model (see kernels_stencil.cu).
//
// A 256-thread block owns a 32 x 8 tile of sites (a thread per site), stages
// the differentiated field with a periodic halo of `reach` sites on every side
// and the pair list in shared memory.
#include "internal.h"

namespace moto {

namespace {
constexpr int kPX = 32, kPY = 8;  // sites per block tile

template <typename T>
struct PairSm {
  int d1, d2;
  T J, Dx, Dy, Dz;
};

template <typename T>
__device__ __forceinline__ void stage_pairs(const ModelDev& md, PairSm<T>* ps) {
  for (int p = threadIdx.x; p < md.npairs; p += blockDim.x) {
    const double* q = md.pairs + 6 * (size_t)p;
    ps[p].d1 = (int)q[0];
    ps[p].d2 = (int)q[1];
    ps[p].J = (T)q[2];
    ps[p].Dx = (T)q[3];
    ps[p].Dy = (T)q[4];
    ps[p].Dz = (T)q[5];
  }
}

// field x at (x0 - R .. x0 + kPX + R) x (y0 - R .. y0 + kPY + R), periodic
template <typename T>
__device__ __forceinline__ void stage_halo(const T* __restrict__ x, const ModelDev& md, int x0, int y0, int R,
                                           T* tile) {
  const int SX = kPX + 2 * R, SY = kPY + 2 * R;
  const size_t N = md.N;
  for (int idx = threadIdx.x; idx < SX * SY; idx += blockDim.x) {
    const int ly = idx / SX, lx = idx - ly * SX;
    const int gx = wrap(x0 - R + lx, md.L1), gy = wrap(y0 - R + ly, md.L2);
    const size_t g = (size_t)gy * md.L1 + gx;
    tile[idx] = x[g];
    tile[SX * SY + idx] = x[N + g];
    tile[2 * SX * SY + idx] = x[2 * N + g];
  }
}

// h = -2 sum_p [J_p x_{+d} + x_{+d} x D_p] at tile-local site (lx, ly)
template <typename A, typename T>
__device__ __forceinline__ void pair_field(const T* tile, const PairSm<T>* ps, int np, int R, int lx, int ly, A& hx,
                                           A& hy, A& hz) {
  const int SX = kPX + 2 * R, SY = kPY + 2 * R;
  A ax = 0, ay = 0, az = 0;
  for (int p = 0; p < np; ++p) {
    const int t = (ly + R + ps[p].d2) * SX + (lx + R + ps[p].d1);
    const A x = (A)tile[t], y = (A)tile[SX * SY + t], z = (A)tile[2 * SX * SY + t];
    const A J = (A)ps[p].J, Dx = (A)ps[p].Dx, Dy = (A)ps[p].Dy, Dz = (A)ps[p].Dz;
    ax += J * x + (y * Dz - z * Dy);
    ay += J * y + (z * Dx - x * Dz);
    az += J * z + (x * Dy - y * Dx);
  }
  hx = (A)-2 * ax;
  hy = (A)-2 * ay;
  hz = (A)-2 * az;
}

__device__ __forceinline__ bool finite3p(double a, double b, double c) {
  return isfinite(a) && isfinite(b) && isfinite(c);
}
}  // namespace

template <typename T, typename A>
__global__ void __launch_bounds__(kThreads) pair_energy_grad_kernel(ModelDev md, const T* __restrict__ m, T* g, T* s,
                                                                    double* part, unsigned* counter, double* out,
                                                                    int* status, int euclid) {
  extern __shared__ __align__(16) unsigned char pr_raw[];
  PairSm<T>* ps = reinterpret_cast<PairSm<T>*>(pr_raw);
  T* tile = reinterpret_cast<T*>(pr_raw + MOTO_MAX_PAIRS * sizeof(PairSm<T>));
  const int R = md.reach;
  const int x0 = blockIdx.x * kPX, y0 = blockIdx.y * kPY;
  stage_pairs(md, ps);
  stage_halo(m, md, x0, y0, R, tile);
  __syncthreads();
  const int lx = threadIdx.x % kPX, ly = threadIdx.x / kPX;
  const int gx = x0 + lx, gy = y0 + ly;
  const int SX = kPX + 2 * R, SY = kPY + 2 * R;
  double esum = 0.0, gmax = 0.0;
  bool bad = false;
  const size_t N = md.N;
  if (gx < md.L1 && gy < md.L2) {
    A hx, hy, hz;
    pair_field<A, T>(tile, ps, md.npairs, R, lx, ly, hx, hy, hz);
    const int t = (ly + R) * SX + lx + R;
    const A mx = (A)tile[t], my = (A)tile[SX * SY + t], mz = (A)tile[2 * SX * SY + t];
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
    esum = 0.5 * ((double)si - md.muB * (double)mz);
    gmax = (double)(gxv * gxv + gyv * gyv + gzv * gzv);
    bad = !finite3p((double)gxv, (double)gyv, (double)gzv);
  }
  __shared__ double red[16];
  double v[1] = {esum};
  block_sum<1>(v, red);
  gmax = block_max(gmax, red + 8);
  if (bad) atomicOr(status, kStatusNonfinite);
  if (!out) return;
  const int nblocks = gridDim.x * gridDim.y;
  const int bid = blockIdx.y * gridDim.x + blockIdx.x;
  if (threadIdx.x == 0) {
    part[2 * bid] = v[0];
    part[2 * bid + 1] = gmax;
  }
  __shared__ bool last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = (atomicAdd(counter, 1u) == (unsigned)nblocks - 1);
  __syncthreads();
  if (!last) return;
  __threadfence();
  double a = 0.0, b = 0.0;
  for (int k = threadIdx.x; k < nblocks; k += blockDim.x) {
    a += __ldcg(part + 2 * k);
    b = fmax(b, __ldcg(part + 2 * k + 1));
  }
  double w[1] = {a};
  block_sum<1>(w, red);
  const double mx = block_max(b, red + 8);
  if (threadIdx.x == 0) {
    out[0] = w[0];
    out[1] = sqrt(mx);
    *counter = 0u;
  }
}

// euclid == 0: (H v)_i = P_i [ h_i(v) - 2 K v_iz z - s_i v_i ];
// euclid == 1: (hess E v)_i = h_i(v) - 2 K v_iz z (m, s unused)
template <typename T>
__global__ void __launch_bounds__(kThreads) pair_hvp_kernel(ModelDev md, const T* __restrict__ m,
                                                            const T* __restrict__ s, const T* __restrict__ V,
                                                            size_t ldv, T* __restrict__ HV, size_t ldhv, int nvec,
                                                            int euclid, const int* gate, int mask) {
  if (gate && (*gate & mask)) return;
  extern __shared__ __align__(16) unsigned char pr_raw[];
  PairSm<T>* ps = reinterpret_cast<PairSm<T>*>(pr_raw);
  T* tile = reinterpret_cast<T*>(pr_raw + MOTO_MAX_PAIRS * sizeof(PairSm<T>));
  const int R = md.reach;
  const int x0 = blockIdx.x * kPX, y0 = blockIdx.y * kPY;
  const int lx = threadIdx.x % kPX, ly = threadIdx.x / kPX;
  const int gx = x0 + lx, gy = y0 + ly;
  const bool in = gx < md.L1 && gy < md.L2;
  const size_t N = md.N;
  const size_t i = in ? (size_t)gy * md.L1 + gx : 0;
  T m0 = 0, m1 = 0, m2 = 0, si = 0;
  if (!euclid && in) {
    m0 = m[i];
    m1 = m[N + i];
    m2 = m[2 * N + i];
    si = s[i];
  }
  const int SX = kPX + 2 * R, SY = kPY + 2 * R;
  const T twoK = (T)(2.0 * md.K);
  stage_pairs(md, ps);
  for (int j = 0; j < nvec; ++j) {
    if (j > 0) __syncthreads();
    stage_halo(V + (size_t)j * ldv, md, x0, y0, R, tile);
    __syncthreads();
    if (!in) continue;
    T hx, hy, hz;
    pair_field<T, T>(tile, ps, md.npairs, R, lx, ly, hx, hy, hz);
    const int t = (ly + R) * SX + lx + R;
    const T vx = tile[t], vy = tile[SX * SY + t], vz = tile[2 * SX * SY + t];
    hz -= twoK * vz;
    T* hv = HV + (size_t)j * ldhv;
    if (euclid) {
      hv[i] = hx;
      hv[N + i] = hy;
      hv[2 * N + i] = hz;
    } else {
      hx -= si * vx;
      hy -= si * vy;
      hz -= si * vz;
      const T p = m0 * hx + m1 * hy + m2 * hz;
      hv[i] = hx - p * m0;
      hv[N + i] = hy - p * m1;
      hv[2 * N + i] = hz - p * m2;
    }
  }
}

namespace {
template <typename T>
size_t pair_smem(int R) {
  return MOTO_MAX_PAIRS * sizeof(PairSm<T>) + 3 * (size_t)(kPX + 2 * R) * (kPY + 2 * R) * sizeof(T);
}
dim3 pair_grid(const ModelDev& md) { return dim3((md.L1 + kPX - 1) / kPX, (md.L2 + kPY - 1) / kPY); }
}  // namespace

int pair_blocks(const ModelDev& md) {
  const dim3 g = pair_grid(md);
  return (int)(g.x * g.y);
}

template <typename T>
void launch_pair_energy_grad(const ModelDev& md, const T* m, T* g, T* s, double* part, unsigned* counter,
                             double* out, int* status, bool fp64_arith, bool euclid, cudaStream_t st) {
  const size_t smem = pair_smem<T>(md.reach);
  const int e = euclid ? 1 : 0;
  if (fp64_arith) {
    cudaFuncSetAttribute(pair_energy_grad_kernel<T, double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)pair_smem<T>(MOTO_MAX_REACH));
    pair_energy_grad_kernel<T, double><<<pair_grid(md), kThreads, smem, st>>>(md, m, g, s, part, counter, out,
                                                                              status, e);
  } else {
    cudaFuncSetAttribute(pair_energy_grad_kernel<T, T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)pair_smem<T>(MOTO_MAX_REACH));
    pair_energy_grad_kernel<T, T><<<pair_grid(md), kThreads, smem, st>>>(md, m, g, s, part, counter, out, status,
                                                                         e);
  }
}

template <typename T>
void launch_pair_hvp(const ModelDev& md, const T* m, const T* s, const T* V, size_t ldv, T* HV, size_t ldhv,
                     int nvec, bool euclid, const int* gate, int mask, cudaStream_t st) {
  cudaFuncSetAttribute(pair_hvp_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)pair_smem<T>(MOTO_MAX_REACH));
  pair_hvp_kernel<T><<<pair_grid(md), kThreads, pair_smem<T>(md.reach), st>>>(md, m, s, V, ldv, HV, ldhv, nvec,
                                                                             euclid ? 1 : 0, gate, mask);
}

#define INST(T)                                                                                                 \
  template void launch_pair_energy_grad<T>(const ModelDev&, const T*, T*, T*, double*, unsigned*, double*, int*, \
                                           bool, bool, cudaStream_t);                                           \
  template void launch_pair_hvp<T>(const ModelDev&, const T*, const T*, const T*, size_t, T*, size_t, int, bool, \
                                   const int*, int, cudaStream_t);
INST(float)
INST(double)
#undef INST

}  // namespace moto
