// Lattice stencil of the spin Hamiltonian: the linear field
//   h_i(x) = -2 sum_s J_s sum_{d in shell s} x_{i+d}
//            - 2 D sum_{d in shell 1} [ z (x_{i+d} . d_hat) - d_hat x_{i+d,z} ]
// which is grad_i E without its on-site terms when x = m (Eq. param-hamiltonian,
// ordered-pair sums, Neel DMI D_ij = D z x r_hat_ij), and the off-site part of
// (hess E x)_i for any x.  Evaluated from a shared-memory tile that holds the
// block's sites plus a 2-site periodic halo in index space (shell 3 reaches
// offsets of +-2).
#pragma once

#include "common.cuh"

namespace moto {

constexpr int kTileX = 32;             // sites along a1 per block (one warp)
constexpr int kTileRowsPerThread = 4;  // rows along a2 per thread
constexpr int kTileY = 8 * kTileRowsPerThread;  // 8 warps per block
constexpr int kHalo = 2;
constexpr int kTX = kTileX + 2 * kHalo;  // 36
constexpr int kTY = kTileY + 2 * kHalo;  // 36

template <typename T>
struct Tile {
  T v[3][kTY][kTX];
};

// Cooperative load of the halo'd tile of a 3N field with origin (x0, y0).
template <typename T>
__device__ __forceinline__ void load_tile(const T* __restrict__ x, int N, int L1, int L2, int x0, int y0,
                                          Tile<T>& t) {
  const bool interior = (x0 >= kHalo) && (y0 >= kHalo) && (x0 + kTileX + kHalo <= L1) && (y0 + kTileY + kHalo <= L2);
  for (int idx = threadIdx.x; idx < kTX * kTY; idx += blockDim.x) {
    const int ly = idx / kTX, lx = idx - ly * kTX;
    int gx = x0 + lx - kHalo, gy = y0 + ly - kHalo;
    if (!interior) {
      gx = wrap(gx, L1);
      gy = wrap(gy, L2);
    }
    const size_t g = (size_t)gy * L1 + gx;
    t.v[0][ly][lx] = __ldg(x + g);
    t.v[1][ly][lx] = __ldg(x + N + g);
    t.v[2][ly][lx] = __ldg(x + 2 * (size_t)N + g);
  }
}

// h = linear field at tile-local site (lx, ly) (without halo offset).
template <typename A, typename T>
__device__ __forceinline__ void linear_field(const ModelDev& md, const Tile<T>& t, int lx, int ly, A& hx, A& hy,
                                             A& hz) {
  const int cx = lx + kHalo, cy = ly + kHalo;
#define X_(c, d1, d2) ((A)t.v[c][cy + (d2)][cx + (d1)])
  A ax, ay, az;
  // shell 1: +-(1,0), +-(0,1), +-(-1,1)
  ax = X_(0, 1, 0) + X_(0, -1, 0) + X_(0, 0, 1) + X_(0, 0, -1) + X_(0, -1, 1) + X_(0, 1, -1);
  ay = X_(1, 1, 0) + X_(1, -1, 0) + X_(1, 0, 1) + X_(1, 0, -1) + X_(1, -1, 1) + X_(1, 1, -1);
  az = X_(2, 1, 0) + X_(2, -1, 0) + X_(2, 0, 1) + X_(2, 0, -1) + X_(2, -1, 1) + X_(2, 1, -1);
  const A j0 = (A)(-2.0 * md.J[0]);
  hx = j0 * ax;
  hy = j0 * ay;
  hz = j0 * az;
  if (md.n_shells > 1) {
    // shell 2: +-(1,1), +-(-1,2), +-(-2,1)
    ax = X_(0, 1, 1) + X_(0, -1, -1) + X_(0, -1, 2) + X_(0, 1, -2) + X_(0, -2, 1) + X_(0, 2, -1);
    ay = X_(1, 1, 1) + X_(1, -1, -1) + X_(1, -1, 2) + X_(1, 1, -2) + X_(1, -2, 1) + X_(1, 2, -1);
    az = X_(2, 1, 1) + X_(2, -1, -1) + X_(2, -1, 2) + X_(2, 1, -2) + X_(2, -2, 1) + X_(2, 2, -1);
    const A j1 = (A)(-2.0 * md.J[1]);
    hx += j1 * ax;
    hy += j1 * ay;
    hz += j1 * az;
  }
  if (md.n_shells > 2) {
    // shell 3: +-(2,0), +-(0,2), +-(-2,2)
    ax = X_(0, 2, 0) + X_(0, -2, 0) + X_(0, 0, 2) + X_(0, 0, -2) + X_(0, -2, 2) + X_(0, 2, -2);
    ay = X_(1, 2, 0) + X_(1, -2, 0) + X_(1, 0, 2) + X_(1, 0, -2) + X_(1, -2, 2) + X_(1, 2, -2);
    az = X_(2, 2, 0) + X_(2, -2, 0) + X_(2, 0, 2) + X_(2, 0, -2) + X_(2, -2, 2) + X_(2, 2, -2);
    const A j2 = (A)(-2.0 * md.J[2]);
    hx += j2 * ax;
    hy += j2 * ay;
    hz += j2 * az;
  }
  // Neel DMI, shell 1, pairing +d with -d (d_hat(-d) = -d_hat(d)):
  //   in-plane: +2D sum_half d_hat (x_{+d,z} - x_{-d,z})
  //   z:        -2D sum_half d_hat . (x_{+d} - x_{-d})
  // half shell d = (1,0) d_hat = (1, 0); (0,1): (1/2, s); (-1,1): (-1/2, s); s = sqrt(3)/2
  const A s3 = (A)0.86602540378443864676;
  const A h = (A)0.5;
  const A dz1 = X_(2, 1, 0) - X_(2, -1, 0);
  const A dz2 = X_(2, 0, 1) - X_(2, 0, -1);
  const A dz3 = X_(2, -1, 1) - X_(2, 1, -1);
  const A dx1 = X_(0, 1, 0) - X_(0, -1, 0);
  const A dx2 = X_(0, 0, 1) - X_(0, 0, -1);
  const A dx3 = X_(0, -1, 1) - X_(0, 1, -1);
  const A dy2 = X_(1, 0, 1) - X_(1, 0, -1);
  const A dy3 = X_(1, -1, 1) - X_(1, 1, -1);
  const A twoD = (A)(2.0 * md.D);
  hx += twoD * (dz1 + h * (dz2 - dz3));
  hy += twoD * (s3 * (dz2 + dz3));
  hz -= twoD * (dx1 + h * (dx2 - dx3) + s3 * (dy2 + dy3));
#undef X_
}

}  // namespace moto
