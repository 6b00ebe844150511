// Eigenpairs of the projected block-Lanczos matrix T (n <= 96, symmetric, band
// width b) on one block.  GB300 executes FP64 slowly (a thin pipe shared by the
// SM, and dependent chains on one thread are slower still), so FP64 is kept
// where it buys accuracy and the context precision R does the rest:
//   1. Householder reduction to tridiagonal form Q^T T Q = tridiag(d, e) in R
//      (skipped for b = 1, where T is tridiagonal); three barriers per
//      reflector: warp 0 forms it, every warp applies it to its rows;
//   2. the lowest 16 eigenvalues located by FP32 multisection on the Sturm
//      sequence of the characteristic polynomials
//      p_r = (d_r - x) p_{r-1} - e_{r-1}^2 p_{r-2} (sign changes count the
//      eigenvalues below x; rescaled to stay in range), 16 lanes each;
//   3. each eigenvector of the tridiagonal matrix by inverse iteration in R
//      (LU with partial pivoting, three sweeps), one lane each, vectors
//      orthogonalised within clusters of close eigenvalues, and FP64
//      Rayleigh quotients;
//   4. back-transformation of the k lowest eigenvectors in R (one warp per
//      vector) and, for them, FP64 Rayleigh quotients with the original T.
// Golub & Van Loan, Matrix Computations, sec. 8.3 (tridiagonalisation), 8.4
// (bisection), 8.2 (inverse iteration, Rayleigh quotient).
#include "internal.h"

namespace moto {

namespace {
constexpr int kN = MOTO_MAX_BASIS;
constexpr int kLdA = kN + 1;
constexpr int kNE = 16;  // lowest Ritz values computed; higher entries of theta stay +inf
constexpr int kIW = kN + 1;  // padded stride of the per-lane inverse-iteration arrays

template <typename R>
__device__ __forceinline__ R warp_sum_r(R v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// start vector of inverse iteration: a fixed hash of (row, eigenvalue index)
// in [0.75, 1.25)
__device__ __forceinline__ float start_entry(int r, int i) {
  unsigned h = (unsigned)r * 0x9E3779B1u ^ (unsigned)(i + 1) * 0x85EBCA77u;
  h ^= h >> 15;
  h *= 0x2C1B3C6Du;
  h ^= h >> 12;
  return 0.75f + 0.5f * (float)(h >> 8) * (1.0f / 16777216.0f);
}

template <typename R>
size_t eig_smem_bytes() {
  return (3 * kN + (size_t)kNE * kN) * sizeof(double) +
         ((size_t)kN * kLdA + 2 * kN + 5 * (size_t)kNE * kIW + (size_t)kNE * kN) * sizeof(R) + (size_t)kNE * kIW;
}
}  // namespace

template <typename R>
__global__ void __launch_bounds__(256) tridiag_eig_kernel(const double* __restrict__ Tm, int ldT, int band,
                                                          double* theta, double* Y, int k, DevState* st, size_t ws) {
  Tm = wofs(Tm, ws);
  theta = wofs(theta, ws);
  Y = wofs(Y, ws);
  st = wofs(st, ws);
  if (st->gate & kGateDone) return;
  extern __shared__ double sm[];
  double* d = sm;                              // diagonal
  double* e = d + kN;                          // off-diagonal
  double* lam = e + kN;                        // eigenvalues
  double* vec = lam + kN;                      // kNE x n eigenvectors of the tridiagonal matrix
  R* A = reinterpret_cast<R*>(vec + (size_t)kNE * kN);  // n x (n+1), Householder vectors below the subdiagonal
  R* beta = A + (size_t)kN * kLdA;             // reflector scales
  R* pv = beta + kN;                           // p = b A22 v
  R* iw = pv + kN;                             // inverse iteration: [dg, su, s2, lm, x] x kNE x kIW
  R* vr = iw + 5 * (size_t)kNE * kIW;          // kNE x n vectors in R for the back-transformation
  unsigned char* piv = reinterpret_cast<unsigned char*>(vr + (size_t)kNE * kN);  // pivot flags
  __shared__ float shift[kNE];
  __shared__ float df[kN], ef[kN], e2f[kN];
  __shared__ R sh_alpha, sh_beta;
  __shared__ double sh_tn;
  const int n = st->nT;
  const int tid = threadIdx.x, nth = blockDim.x;
  const int wp = tid >> 5, ln = tid & 31, nw = nth >> 5;

  for (int i = tid; i < MOTO_MAX_BASIS; i += nth) theta[i] = 1.0 / 0.0;
  if (n <= 0) return;
#pragma unroll 4
  for (int idx = tid; idx < n * n; idx += nth) {
    const int r = idx / n, c = idx - r * n;
    A[r * kLdA + c] = (R)(0.5 * (Tm[(size_t)r * ldT + c] + Tm[(size_t)c * ldT + r]));
  }
  __syncthreads();

  // ---- 1. tridiagonalisation (precision R) -------------------------------------
  if (band > 1) {
    for (int j = 0; j + 2 < n; ++j) {
      const int m0 = j + 1;
      if (wp == 0) {  // reflector of column j below the diagonal
        R s = 0;
        for (int r = m0 + ln; r < n; r += 32) {
          const R a = A[r * kLdA + j];
          s += a * a;
        }
        const R norm2 = warp_sum_r(s);
        if (ln == 0) {
          const R x0 = A[m0 * kLdA + j];
          if (norm2 - x0 * x0 <= (R)1e-30 * (norm2 + (R)1e-30)) {
            sh_beta = 0;
            sh_alpha = x0;
          } else {
            const R alpha = -copysign(sqrt(norm2), x0);
            const R v0 = x0 - alpha;
            const R vtv = v0 * v0 + (norm2 - x0 * x0);
            sh_alpha = alpha;
            sh_beta = (R)2 / vtv;
            A[m0 * kLdA + j] = v0;
          }
          e[j] = (double)sh_alpha;
          beta[j] = sh_beta;
        }
      }
      __syncthreads();
      const R b = sh_beta;
      if (b == (R)0) {
        __syncthreads();
        continue;
      }
      // p = b A22 v: two threads a row (adjacent lanes, alternate columns),
      // four partial sums each
      for (int idx = tid; idx < 2 * (n - m0); idx += nth) {
        const int r = m0 + (idx >> 1), h = idx & 1;
        R a0 = 0, a1 = 0, a2 = 0, a3 = 0;
        int c2 = m0 + h;
        for (; c2 + 6 < n; c2 += 8) {
          a0 += A[r * kLdA + c2] * A[c2 * kLdA + j];
          a1 += A[r * kLdA + c2 + 2] * A[(c2 + 2) * kLdA + j];
          a2 += A[r * kLdA + c2 + 4] * A[(c2 + 4) * kLdA + j];
          a3 += A[r * kLdA + c2 + 6] * A[(c2 + 6) * kLdA + j];
        }
        for (; c2 < n; c2 += 2) a0 += A[r * kLdA + c2] * A[c2 * kLdA + j];
        R a = (a0 + a1) + (a2 + a3);
        a += __shfl_xor_sync(3u << (ln & 30), a, 1);
        if (h == 0) pv[r] = b * a;
      }
      __syncthreads();
      // K = b v^T p / 2, summed by every warp in the same order; the update
      // A22 -= v w^T + w v^T with w = p - K v formed on the fly
      R q = 0;
      for (int r = m0 + ln; r < n; r += 32) q += A[r * kLdA + j] * pv[r];
      const R K = (R)0.5 * b * warp_sum_r(q);
      // the lane's column terms (at most three columns) do not depend on the row
      R vcol[3], wcol[3];
#pragma unroll
      for (int u = 0; u < 3; ++u) {
        const int c2 = m0 + ln + 32 * u;
        vcol[u] = c2 < n ? A[c2 * kLdA + j] : (R)0;
        wcol[u] = c2 < n ? pv[c2] - K * vcol[u] : (R)0;
      }
#pragma unroll 2
      for (int r = m0 + wp; r < n; r += nw) {
        const R vr_ = A[r * kLdA + j];
        const R wr = pv[r] - K * vr_;
#pragma unroll
        for (int u = 0; u < 3; ++u) {
          const int c2 = m0 + ln + 32 * u;
          if (c2 < n) A[r * kLdA + c2] -= vr_ * wcol[u] + wr * vcol[u];
        }
      }
      __syncthreads();
    }
    if (tid == 0) {
      for (int i = 0; i < n; ++i) d[i] = (double)A[i * kLdA + i];
      if (n >= 2) e[n - 2] = (double)A[(n - 1) * kLdA + (n - 2)];
      e[n - 1] = 0.0;
      for (int i = (n >= 2 ? n - 2 : 0); i < n; ++i) beta[i] = 0;
    }
  } else {
    for (int i = tid; i < n; i += nth) {
      d[i] = 0.5 * (Tm[(size_t)i * ldT + i] + Tm[(size_t)i * ldT + i]);
      e[i] = (i + 1 < n) ? 0.5 * (Tm[(size_t)(i + 1) * ldT + i] + Tm[(size_t)i * ldT + i + 1]) : 0.0;
      beta[i] = 0;
    }
  }
  __syncthreads();

  // ---- 2. FP32 bisection for the lowest ne eigenvalues --------------------------
  for (int r = tid; r < n; r += nth) {
    df[r] = (float)d[r];
    ef[r] = (float)fabs(e[r]);
    e2f[r] = (float)(e[r] * e[r]);
  }
  if (wp == 0) {  // |T| estimate (largest row sum of the tridiagonal matrix)
    double t = 0.0;
    for (int i = ln; i < n; i += 32) {
      const double rs = (i > 0 ? fabs(e[i - 1]) : 0.0) + (i + 1 < n ? fabs(e[i]) : 0.0);
      t = fmax(t, fabs(d[i]) + rs);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t = fmax(t, __shfl_xor_sync(0xffffffffu, t, o));
    if (ln == 0) sh_tn = fmax(t, 1e-300);
  }
  __syncthreads();
  const double tn = sh_tn;
  const int ne = n < kNE ? n : kNE;
  {
    // multisection: half-warp h of warp w brackets eigenvalue 2w + h; its 16
    // lanes count the eigenvalues below 16 interior points of the bracket
    // (Sturm sequence), which shrinks the bracket 17-fold per round
    const int half = ln >> 4, sl = ln & 15;
    const int i = 2 * wp + half;
    const bool act = i < ne;
    float lo = 1e30f, hi = -1e30f;
    for (int r = 0; r < n; ++r) {
      const float rr = (r > 0 ? ef[r - 1] : 0.f) + (r + 1 < n ? ef[r] : 0.f);
      lo = fminf(lo, df[r] - rr);
      hi = fmaxf(hi, df[r] + rr);
    }
    float a = lo - 1e-6f * (float)tn, bb = hi + 1e-6f * (float)tn;
    for (int round = 0; round < 24; ++round) {
      const bool open = act && (bb - a) > 4e-7f * fmaxf(fabsf(a), fabsf(bb)) + 2e-7f * (float)tn;
      if (!__any_sync(0xffffffffu, open)) break;
      const float x = a + (bb - a) * (float)(sl + 1) * (1.0f / 17.0f);
      float pm = 1.f, p = df[0] - x;
      if (p == 0.f) p = -1e-30f;
      int cnt = (p < 0.f) ? 1 : 0;
      for (int r = 1; r < n; ++r) {
        float pn = (df[r] - x) * p - e2f[r - 1] * pm;
        if (pn == 0.f) pn = -copysignf(1e-30f, p);
        cnt += ((pn < 0.f) != (p < 0.f)) ? 1 : 0;
        pm = p;
        p = pn;
        const float ap = fabsf(p);
        if (ap > 1e18f || (ap < 1e-18f && fabsf(pm) < 1e-18f)) {
          const float sc = ap > 1e18f ? 1e-18f : 1e18f;
          p *= sc;
          pm *= sc;
        }
      }
      const unsigned above = (__ballot_sync(0xffffffffu, cnt > i) >> (16 * half)) & 0xFFFFu;
      if (open) {
        // counts grow with x: the first point above eigenvalue i closes the bracket
        const float w = bb - a;
        if (above == 0u) {
          a = a + w * (16.0f / 17.0f);
        } else {
          const int f = __ffs(above) - 1;
          const float na = f == 0 ? a : a + w * (float)f * (1.0f / 17.0f);
          bb = a + w * (float)(f + 1) * (1.0f / 17.0f);
          a = na;
        }
      }
    }
    if (act && sl == 0) shift[i] = 0.5f * (a + bb);
  }
  __syncthreads();

  // ---- 3. inverse iteration (precision R), one lane per eigenvalue -------------
  if (tid < ne) {
    const int i = tid;
    R* dg = iw + (size_t)i * kIW;
    R* su = dg + (size_t)kNE * kIW;
    R* s2 = su + (size_t)kNE * kIW;
    R* lm = s2 + (size_t)kNE * kIW;
    R* x = lm + (size_t)kNE * kIW;
    unsigned char* pivot = piv + (size_t)i * kIW;
    const R sigma = (R)shift[i];
    const R tiny = (R)((sizeof(R) == 4 ? 1e-7 : 1e-14) * tn);
    for (int r = 0; r < n; ++r) {
      dg[r] = (R)d[r] - sigma;
      su[r] = (r + 1 < n) ? (R)e[r] : (R)0;
      s2[r] = 0;
    }
    for (int r = 0; r + 1 < n; ++r) {
      const R sub = (R)e[r];
      if (fabs(dg[r]) >= fabs(sub)) {
        pivot[r] = 0;
        const R l = (dg[r] != (R)0) ? sub / dg[r] : (R)0;
        lm[r] = l;
        dg[r + 1] -= l * su[r];
      } else {
        pivot[r] = 1;
        const R l = dg[r] / sub;
        lm[r] = l;
        const R d1 = dg[r + 1], u1 = su[r + 1], old_su = su[r];
        dg[r] = sub;
        su[r] = d1;
        s2[r] = u1;
        dg[r + 1] = old_su - l * d1;
        su[r + 1] = -l * u1;
      }
    }
    for (int r = 0; r < n; ++r) {
      if (fabs(dg[r]) < tiny) dg[r] = (dg[r] < (R)0 ? -tiny : tiny);
      dg[r] = (R)1 / dg[r];  // the sweeps multiply by the reciprocal pivots
    }
    for (int r = 0; r < n; ++r) x[r] = (R)start_entry(r, i);
    for (int sweep = 0; sweep < 3; ++sweep) {
      for (int r = 0; r + 1 < n; ++r) {
        if (pivot[r]) {
          const R t = x[r];
          x[r] = x[r + 1];
          x[r + 1] = t - lm[r] * x[r + 1];
        } else {
          x[r + 1] -= lm[r] * x[r];
        }
      }
      for (int r = n - 1; r >= 0; --r) {
        R a = x[r];
        if (r + 1 < n) a -= su[r] * x[r + 1];
        if (r + 2 < n) a -= s2[r] * x[r + 2];
        x[r] = a * dg[r];
      }
      R nn = 0;
      for (int r = 0; r < n; ++r) nn += x[r] * x[r];
      nn = (R)1 / sqrt(nn);
      for (int r = 0; r < n; ++r) x[r] *= nn;
    }
    for (int r = 0; r < n; ++r) vec[i * kN + r] = (double)x[r];
  }
  __syncthreads();
  // clusters: orthogonalise (modified Gram-Schmidt), then Rayleigh quotients
  if (wp == 0) {  // warp 0: lanes split the rows, fixed shuffle trees
    for (int i = 1; i < ne; ++i) {
      bool touched = false;
      for (int j = 0; j < i; ++j) {
        if (fabs((double)shift[i] - (double)shift[j]) > 1e-5 * tn) continue;
        double dot = 0.0;
        for (int r = ln; r < n; r += 32) dot += vec[i * kN + r] * vec[j * kN + r];
        dot = warp_sum(dot);
        for (int r = ln; r < n; r += 32) vec[i * kN + r] -= dot * vec[j * kN + r];
        __syncwarp();
        touched = true;
      }
      if (touched) {
        double nn = 0.0;
        for (int r = ln; r < n; r += 32) nn += vec[i * kN + r] * vec[i * kN + r];
        nn = 1.0 / sqrt(warp_sum(nn));
        for (int r = ln; r < n; r += 32) vec[i * kN + r] *= nn;
        __syncwarp();
      }
    }
  }
  __syncthreads();
  for (int i = wp; i < ne; i += nw) {  // lambda_i = x^T tridiag x, a warp per vector
    const double* x = vec + i * kN;
    double a = 0.0;
    for (int r = ln; r < n; r += 32) {
      double t = d[r] * x[r];
      if (r > 0) t += e[r - 1] * x[r - 1];
      if (r + 1 < n) t += e[r] * x[r + 1];
      a += x[r] * t;
    }
    a = warp_sum(a);
    if (ln == 0) lam[i] = a;
  }
  __syncthreads();
  // order (inverse iteration keeps the bisection order except inside clusters)
  if (tid == 0) {
    for (int i = 1; i < ne; ++i)
      for (int j = i; j > 0 && lam[j] < lam[j - 1]; --j) {
        const double t = lam[j];
        lam[j] = lam[j - 1];
        lam[j - 1] = t;
        for (int r = 0; r < n; ++r) {
          const double u = vec[j * kN + r];
          vec[j * kN + r] = vec[(j - 1) * kN + r];
          vec[(j - 1) * kN + r] = u;
        }
      }
  }
  __syncthreads();
  // The returned vectors, mutually orthogonalised in FP64: inverse iteration
  // in FP32 leaves vectors of close (but not clustered) eigenvalues with
  // overlaps of order eps |T| / gap, up to ~1e-4 on the dense low end of the
  // spectrum.  One classical Gram-Schmidt pass removes them to O(overlap^2):
  // the dots in parallel (a warp per pair), the updates from the unchanged
  // vectors (thread per entry), then the norms.
  {
    const int kr = k < ne ? k : ne;
    __shared__ double ov[MOTO_MAX_K][MOTO_MAX_K];
    double* nv = reinterpret_cast<double*>(iw);  // kr x kN scratch (inverse-iteration workspace)
    for (int pr = wp; pr < kr * kr; pr += nw) {
      const int i = pr / kr, j = pr - i * kr;
      if (j >= i) continue;
      double a = 0.0;
      for (int r = ln; r < n; r += 32) a += vec[i * kN + r] * vec[j * kN + r];
      a = warp_sum(a);
      if (ln == 0) ov[i][j] = a;
    }
    __syncthreads();
    for (int idx = tid; idx < kr * n; idx += nth) {
      const int i = idx / n, r = idx - i * n;
      double x = vec[i * kN + r];
      for (int j = 0; j < i; ++j) x -= ov[i][j] * vec[j * kN + r];
      nv[i * kN + r] = x;
    }
    __syncthreads();
    for (int i = wp; i < kr; i += nw) {
      double a = 0.0;
      for (int r = ln; r < n; r += 32) a += nv[i * kN + r] * nv[i * kN + r];
      const double f = 1.0 / sqrt(warp_sum(a));
      for (int r = ln; r < n; r += 32) vec[i * kN + r] = nv[i * kN + r] * f;
    }
    __syncthreads();
  }

  // ---- 4. back-transformation x <- H_0 ... H_{n-3} x in R (a warp per vector,
  //         the reflectors read-only), then FP64 Rayleigh quotients with the
  //         original T ---------------------------------------------------------------
  const int kk = k < ne ? k : ne;
  if (band > 1) {
    // the band of the symmetrised T for the Rayleigh quotients, read in one
    // round trip by all threads (the inverse-iteration workspace is free now)
    const int bw = 2 * band + 1;
    double* Tb = reinterpret_cast<double*>(iw);
#pragma unroll 4
    for (int idx = tid; idx < n * bw; idx += nth) {
      const int r = idx / bw, c2 = r - band + (idx - r * bw);
      Tb[idx] = (c2 >= 0 && c2 < n) ? 0.5 * (Tm[(size_t)r * ldT + c2] + Tm[(size_t)c2 * ldT + r]) : 0.0;
    }
    __syncthreads();
    for (int vi = wp; vi < kk; vi += nw) {
      R* x = vr + (size_t)vi * kN;
      for (int r = ln; r < n; r += 32) x[r] = (R)vec[vi * kN + r];
      __syncwarp();
      for (int j = n - 3; j >= 0; --j) {
        const R b = beta[j];
        if (b == (R)0) continue;
        const int m0 = j + 1;
        R dot = 0;
        for (int r = m0 + ln; r < n; r += 32) dot += A[r * kLdA + j] * x[r];
        dot = warp_sum_r(dot) * b;
        for (int r = m0 + ln; r < n; r += 32) x[r] -= dot * A[r * kLdA + j];
        __syncwarp();
      }
      double a = 0.0, nn = 0.0;
      for (int r = ln; r < n; r += 32) {
        double t = 0.0;
        const int c0 = r - band < 0 ? 0 : r - band, c1 = r + band + 1 > n ? n : r + band + 1;
        for (int c2 = c0; c2 < c1; ++c2) t += Tb[r * bw + (c2 - r + band)] * (double)x[c2];
        a += (double)x[r] * t;
        nn += (double)x[r] * (double)x[r];
      }
      a = warp_sum(a);
      nn = warp_sum(nn);
      if (ln == 0) lam[vi] = a / nn;
      for (int r = ln; r < n; r += 32) vec[vi * kN + r] = (double)x[r];
    }
    __syncthreads();
  }
  for (int i = tid; i < ne; i += nth) theta[i] = lam[i];
  for (int idx = tid; idx < n * kk; idx += nth) {
    const int r = idx / kk, i = idx - r * kk;
    Y[(size_t)r * k + i] = vec[i * kN + r];
  }
}

void launch_tridiag_eig(const double* T, int ldT, int band, int fp64, double* theta, double* Y, int k, DevState* st,
                        cudaStream_t s) {
  if (fp64) {
    static bool attr = false;
    if (!attr) {
      cudaFuncSetAttribute(tridiag_eig_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)eig_smem_bytes<double>());
      attr = true;
    }
    tridiag_eig_kernel<double><<<wgrid(1), 256, eig_smem_bytes<double>(), s>>>(T, ldT, band, theta, Y, k, st, walker_ws());
  } else {
    static bool attr = false;
    if (!attr) {
      cudaFuncSetAttribute(tridiag_eig_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)eig_smem_bytes<float>());
      attr = true;
    }
    tridiag_eig_kernel<float><<<wgrid(1), 256, eig_smem_bytes<float>(), s>>>(T, ldT, band, theta, Y, k, st, walker_ws());
  }
}

}  // namespace moto
