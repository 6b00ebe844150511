// Estimated loss of orthogonality of block Lanczos, for selective (partial)
// reorthogonalisation.
//
// Block Lanczos satisfies H Q_k = Q_{k-1} B_k^T + Q_k A_k + Q_{k+1} B_{k+1} up
// to rounding, with A_k = T(k, k) symmetric and B_{k+1} = T(k+1, k) the upper
// triangular factor of the new block.  Writing W_{i,k} = Q_i^T Q_k and using
// the symmetry of H (Q_j^T H Q_k = (Q_k^T H Q_j)^T) gives the block form of
// Simon's omega recurrence (Simon 1984):
//   B_{j+1}^T W_{j+1,k} = W_{j,k+1} B_{k+1} + W_{j,k} A_k - A_j W_{j,k}
//                         + W_{j,k-1} B_k^T - B_j W_{j-1,k}        (k < j)
// with W_{k,k} = I.  The estimates add, with the sign of each entry, a
// rounding term nu = eps |T| / min diag(B_{j+1}) (the size of the local
// rounding error of one step magnified by B_{j+1}^{-1}), and take
// W_{j+1,j} = nu for the local orthogonality the three-term pass and the
// Cholesky QR keep.  When the largest |W_{j+1,k}| exceeds sqrt(eps) (or the
// previous step was reorthogonalised because of the estimate: Simon's rule
// of two consecutive blocks) the new block gets the full pass against the
// basis; its estimates then restart at nu.
//
// The estimates live in an MOTO_MAX_BASIS x MOTO_MAX_BASIS FP64 matrix Om
// (block (i, k) at rows i b .., columns k b ..); the decision is the gate bit
// kGateNoReorth, which the full-pass launches of the step test.  The
// recurrence itself runs in FP32: its values are order-of-magnitude bounds
// compared with sqrt(eps) (>= 1e-8), far inside FP32's range, and on GB300
// a chain of dependent FP64 operations costs ~100 cycles a link against a
// few for FP32.
#include "internal.h"

namespace moto {

namespace {
constexpr int kLdO = MOTO_MAX_BASIS;

__device__ __forceinline__ double tblk(const double* T, int ldT, int b, int i, int k, int r, int c) {
  return T[(size_t)(i * b + r) * ldT + k * b + c];
}
}  // namespace

// Block row j + 1 of the estimates from rows j and j - 1 (k < j), the
// decision, and W_{j+1,j} = nu.  Rn: the (tentative) B_{j+1}, b x b row-major.
// One block of 1024 threads; thread (k, r, c) forms one entry of the
// right-hand side, thread (k, c) solves one column of the triangular system.
__global__ void __launch_bounds__(1024) omega_estimate_kernel(int b, int j, const double* T, int ldT,
                                                              const double* Rn, double* Om, double* rlog,
                                                              DevState* st, double eps, size_t ws) {
  T = wofs(T, ws);
  Rn = wofs(Rn, ws);
  Om = wofs(Om, ws);
  rlog = wofs(rlog, ws);
  st = wofs(st, ws);
  if (st->gate & (kGateKrylov | kGateDone)) return;
  __shared__ float Bn[MOTO_MAX_K][MOTO_MAX_K];
  __shared__ float binv[MOTO_MAX_K];  // 1 / B_{j+1}(r, r), +inf where not positive
  __shared__ float M[MOTO_MAX_BASIS * MOTO_MAX_K];  // [k][r][c], k < j
  // the operands, staged in one round trip: block rows j - 1 and j of the
  // estimates (columns 0 .. (j + 1) b) and the blocks of T the recurrence
  // reads, Td[k] = T(k, k) for k <= j and Tl[k] = T(k + 1, k) for k < j
  __shared__ float Os[2 * MOTO_MAX_K][MOTO_MAX_BASIS];
  // (j + 1) b <= MOTO_MAX_BASIS, so (j + 1) b^2 <= MOTO_MAX_BASIS MOTO_MAX_K
  __shared__ float Td[MOTO_MAX_BASIS * MOTO_MAX_K];
  __shared__ float Tl[MOTO_MAX_BASIS * MOTO_MAX_K];
  __shared__ float nu_s, wmax[32];
  const int bb = b * b, t = threadIdx.x;
  if (t < bb) Bn[t / b][t % b] = (float)Rn[t];
  if (t < b) {
    const double d = Rn[t * b + t];
    binv[t] = d > 0.0 ? (float)(1.0 / d) : __int_as_float(0x7f800000);
  }
  const int ncol = (j + 1) * b;
  for (int e = t; e < 2 * b * ncol; e += blockDim.x) {
    const int rr = e / ncol, cc = e - rr * ncol;  // rr < b: block row j - 1
    const int grow = (j - 1) * b + rr;
    Os[rr][cc] = grow >= 0 ? (float)Om[(size_t)grow * kLdO + cc] : 0.f;
  }
  for (int e = t; e < (2 * j + 1) * bb; e += blockDim.x) {
    const int kb = e / bb, q = e - kb * bb, r = q / b, c = q - r * b;
    if (kb <= j)
      Td[kb * bb + q] = (float)tblk(T, ldT, b, kb, kb, r, c);
    else
      Tl[(kb - j - 1) * bb + q] = (float)tblk(T, ldT, b, kb - j, kb - j - 1, r, c);
  }
  __syncthreads();
  // staged views: W_{j,x} row r at Os[b + r][x], W_{j-1,x} row r at Os[r][x]
#define OMJ(r, col) Os[b + (r)][col]
#define OMJ1(r, col) Os[(r)][col]
#define TD(k, r, c) Td[(k) * bb + (r) * b + (c)]
#define TL(k, r, c) Tl[(k) * bb + (r) * b + (c)]
  if (t == 0) {
    float dmin = __int_as_float(0x7f800000);
    for (int r = 0; r < b; ++r) dmin = fminf(dmin, Bn[r][r]);
    const float tn = (float)fmax(st->tnorm, 1e-30);
    nu_s = dmin > 0.f ? (float)eps * tn / dmin : __int_as_float(0x7f800000);
  }
  // right-hand sides
  for (int e = t; e < j * bb; e += blockDim.x) {
    const int k = e / bb, r = (e % bb) / b, c = e % b;
    float a = 0.f;
    for (int q = 0; q < b; ++q) {
      // W_{j,k+1} B_{k+1}   (W_{j,j} = I)
      const float wjk1 = (k + 1 == j) ? (r == q ? 1.f : 0.f) : OMJ(r, (k + 1) * b + q);
      a += wjk1 * TL(k, q, c);
      // W_{j,k} A_k - A_j W_{j,k}
      a += OMJ(r, k * b + q) * TD(k, q, c);
      a -= TD(j, r, q) * OMJ(q, k * b + c);
      // W_{j,k-1} B_k^T
      if (k > 0) a += OMJ(r, (k - 1) * b + q) * TL(k - 1, c, q);
      // - B_j W_{j-1,k}   (W_{j-1,j-1} = I)
      const float wj1k = (k == j - 1) ? (q == c ? 1.f : 0.f) : OMJ1(q, k * b + c);
      a -= TL(j - 1, r, q) * wj1k;
    }
    M[e] = a;
  }
#undef OMJ
#undef OMJ1
#undef TD
#undef TL
  __syncthreads();
  const float nu = nu_s;
  float mx = 0.f;
  // B_{j+1}^T X = M, B upper triangular: forward substitution down each column
  for (int e = t; e < j * b; e += blockDim.x) {
    const int k = e / b, c = e % b;
    float x[MOTO_MAX_K];
    for (int r = 0; r < b; ++r) {
      float a = M[k * bb + r * b + c];
      for (int q = 0; q < r; ++q) a -= Bn[q][r] * x[q];
      x[r] = a * binv[r];
    }
    for (int r = 0; r < b; ++r) {
      const float v = x[r] + copysignf(nu, x[r]);
      Om[(size_t)((j + 1) * b + r) * kLdO + k * b + c] = (double)v;
      mx = fmaxf(mx, fabsf(v));
    }
  }
  for (int e = t; e < bb; e += blockDim.x)
    Om[(size_t)((j + 1) * b + e / b) * kLdO + j * b + e % b] = (double)nu;
  // block maximum, then the decision (a factor without a positive diagonal,
  // nu = inf, always asks for the pass)
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((t & 31) == 0) wmax[t >> 5] = mx;
  __syncthreads();
  if (t == 0) {
    float m2 = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m2 = fmaxf(m2, wmax[w]);
    const bool forced = st->pad[3] != 0;
    const bool need = forced || !(nu < __int_as_float(0x7f800000)) || !(m2 <= (float)sqrt(eps));
    st->pad[5] = forced ? 1 : 0;
    rlog[j] = need ? 1.0 : 0.0;  // for the launch profiler: did step j take the full pass
    if (need)
      st->gate &= ~kGateNoReorth;
    else
      st->gate |= kGateNoReorth;
  }
}

// After a full pass of step j (runs only when the step was reorthogonalised):
// the estimates of block row j + 1 restart at nu; a pass the estimate asked
// for forces one on the next step too, a forced pass does not.
__global__ void omega_reset_kernel(int b, int j, const double* Rn, double* Om, DevState* st, double eps, size_t ws) {
  Rn = wofs(Rn, ws);
  Om = wofs(Om, ws);
  st = wofs(st, ws);
  if (st->gate & (kGateKrylov | kGateDone | kGateNoReorth)) return;
  __shared__ double nu_s;
  const int t = threadIdx.x;
  if (t == 0) {
    double dmin = 1e300;
    for (int r = 0; r < b; ++r) dmin = fmin(dmin, Rn[r * b + r]);
    nu_s = dmin > 0.0 ? eps * fmax(st->tnorm, 1e-300) / dmin : 1e300;
  }
  __syncthreads();
  for (int e = t; e < (j + 1) * b * b; e += blockDim.x) {
    const int k = e / (b * b), r = (e % (b * b)) / b, c = e % b;
    Om[(size_t)((j + 1) * b + r) * kLdO + k * b + c] = nu_s;
  }
  if (t == 0) {
    st->pad[3] = st->pad[5] ? 0 : 1;
    st->pad[4] += 1;  // reorthogonalised steps of this solve
  }
}

void launch_omega_estimate(int b, int j, const double* T, int ldT, const double* Rn, double* Om, double* rlog,
                           DevState* st, double eps, cudaStream_t s) {
  omega_estimate_kernel<<<wgrid(1), 1024, 0, s>>>(b, j, T, ldT, Rn, Om, rlog, st, eps, walker_ws());
}

void launch_omega_reset(int b, int j, const double* Rn, double* Om, DevState* st, double eps, cudaStream_t s) {
  omega_reset_kernel<<<wgrid(1), 256, 0, s>>>(b, j, Rn, Om, st, eps, walker_ws());
}

}  // namespace moto
