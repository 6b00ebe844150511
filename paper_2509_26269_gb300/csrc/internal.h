// Internal launchers shared by the C-ABI implementation and the kernel files.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

#include "common.cuh"

namespace moto {

// ---- walker batches ----
// The sequences of a walker group set the calling thread's current walker
// grid: every launch then gets gridDim.z = nw and the slice stride ws (bytes)
// as its last argument; kernels offset their pointers with wofs().  Single
// contexts run with {1, 0}.
struct WalkerGrid {
  int nw;
  size_t ws;
};
WalkerGrid& walker_grid();
inline dim3 wgrid(dim3 g) {
  g.z = (unsigned)walker_grid().nw;
  return g;
}
inline dim3 wgrid(int x) { return wgrid(dim3((unsigned)x)); }
inline dim3 wgrid(unsigned x) { return wgrid(dim3(x)); }
inline size_t walker_ws() { return walker_grid().ws; }

// ---- gate bits: kernels given (gate, mask) return at once if (*gate & mask) ----
enum : int {
  kGateKrylov = 1,  // the Krylov recurrence broke down; skip its remaining steps
  kGateDone = 2,    // the ascent / descent has converged; skip the rest
  kGateNoReorth = 4,  // selective reorthogonalisation: this step keeps the local pass only
};

// Device-side bookkeeping of one eigensolve / optimisation, in device memory.
struct DevState {
  int gate;        // kGate* bits
  int status;      // kStatus* bits (sticky until cleared)
  int steps;       // Krylov blocks in the basis (block Lanczos)
  int nT;          // order of the projected matrix
  int iters;       // iterations (LOBPCG) or steps done
  int lb_head;     // L-BFGS ring: next slot
  int lb_count;    // L-BFGS ring: pairs held
  int lb_have_prev;
  int converged;   // 1 once the stopping test passed
  int pad[7];      // pad[0]: current LOBPCG set; pad[1]: outer steps taken;
                   // pad[2]: CG restart; pad[3]: force a full pass on the next
                   // Lanczos step; pad[4]: steps reorthogonalised in full this
                   // solve; pad[5]: the current step's full pass was forced
  double tnorm;    // running estimate of |T| (largest row sum seen)
  double hnorm;    // LOBPCG: largest |theta| seen
  double scale;    // step scale of the current direction
  double dot;      // g . v1 of the current step
};

int tile_blocks(const ModelDev& md);
// blocks (and so partial-sum slots) of an energy / gradient / charge launch on
// an L1 x L2 lattice, in 64-bit so that no lattice size overflows it
long long stencil_blocks(int L1, int L2);
int pair_blocks(const ModelDev& md);
// pair-list stencils (kernels_pairs.cu); launch_energy_grad, launch_hvp and
// launch_euclid_hvp forward to them when md.npairs > 0
template <typename T>
void launch_pair_energy_grad(const ModelDev& md, const T* m, T* g, T* s, double* part, unsigned* counter,
                             double* out, int* status, bool fp64_arith, bool euclid, cudaStream_t st);
template <typename T>
void launch_pair_hvp(const ModelDev& md, const T* m, const T* s, const T* V, size_t ldv, T* HV, size_t ldhv,
                     int nvec, bool euclid, const int* gate, int mask, cudaStream_t st);

// euclid: g receives grad E itself instead of the Riemannian gradient
template <typename T>
void launch_energy_grad(const ModelDev& md, const T* m, T* g, T* s, double* part, unsigned* counter, double* out,
                        int* status, bool fp64_arith, cudaStream_t st, bool euclid = false);
// Euclidean Hessian-vector product (hess E v)_i = h_i(v) - 2 K v_iz z
template <typename T>
void launch_euclid_hvp(const ModelDev& md, const T* V, size_t ldv, T* HV, size_t ldhv, int nvec, cudaStream_t st);
template <typename T>
void launch_hvp(const ModelDev& md, const T* m, const T* s, const T* V, size_t ldv, T* HV, size_t ldhv, int nvec,
                const int* gate, int mask, cudaStream_t st);
// register-blocked column-strip HVP (kernels_hvp.cu); launch_hvp uses it with
// the variant the autotuner recorded for the lattice (variant 0 without one)
template <typename T>
void launch_hvp_strip(const ModelDev& md, const T* m, const T* s, const T* V, size_t ldv, T* HV, size_t ldhv,
                      int nvec, const int* gate, int mask, cudaStream_t st);
// The strip HVP variants (strip length, warps per block, m held in
// registers): all give bit-identical results; only their speed differs.
int hvp_variant_count();
template <typename T>
void launch_hvp_strip_variant(int variant, const ModelDev& md, const T* m, const T* s, const T* V, size_t ldv, T* HV,
                              size_t ldhv, int nvec, const int* gate, int mask, cudaStream_t st);
// The persistent energy / gradient and charge stencils come in variants
// (staged tiles, blocks an SM); the autotuner records one per lattice and
// precision (-1: none, variant 0 used).  g and s are bit-identical across
// variants; the energy's sum follows the grid.
int stencil_variant_count();
int stencil_tuned_variant(int L1, int L2, int esize);
void stencil_record_variant(int L1, int L2, int esize, int variant);
template <typename T>
void launch_energy_grad_variant(int variant, const ModelDev& md, const T* m, T* g, T* s, double* part,
                                unsigned* counter, double* out, int* status, cudaStream_t st);
// process-wide autotuner record: (L1, L2, element size, nvec) -> variant (-1: none)
int hvp_tuned_variant(int L1, int L2, int esize, int nvec);
void hvp_record_variant(int L1, int L2, int esize, int nvec, int variant);
template <typename T>
void launch_topo(const ModelDev& md, const T* m, double* part, unsigned* counter, double* out, cudaStream_t st);

// out[r*ny + c] = sum_e X_r[e] Y_c[e] over n elements, r < nx <= 96, c < ny <= 8.
// Aligned fields go to the streaming kernel (mode 0: FP32 runs, then
// two-float sums); otherwise FP32 products are summed in FP32 over at most
// 16 x (tile share) elements, then promoted to FP64 for every cross-thread
// and cross-block sum (T = float); all-FP64 for T = double.
template <typename T>
void launch_gram(const T* X, size_t ldx, int nx, const T* Y, size_t ldy, int ny, size_t n, double* out,
                 double* part, unsigned* counter, const int* gate, int mask, cudaStream_t st);
int gram_blocks();
// Streaming reorthogonalisation kernels (kernels_tile.cu), modes
//   0: out = X^T Y;  1: Y <- Y - X[u0, u0 + nu) C, out = X^T Y;
//   2: Y <- Y - X C, out = Y^T Y;  3: Yout <- X C, out = Yout^T Yout
// over n elements (fields X at stride ldx, Y at ldy; updated fields go to Yout
// at stride ldo, Yout == Y for modes 1 and 2; C is nu x ny in mode 1, nx x ny
// in modes 2 and 3).  Modes 1 and 3 with Yout == nullptr store nothing: the
// Gram sees the updated fields, memory keeps the old ones.  Mode 2 may add Cadd
// (nadd x ny) to rows uadd .. uadd + nadd - 1 of C.  Returns false (nothing
// launched) when a base address or stride breaks the TMA alignment rules; the
// caller then uses combine + the plain Gram kernel.  polls > 0 replaces the
// bound of the consumer warps' waits for a filled stage (polls non-blocking
// tests instead of ~2^22 blocking ones), so that a test can make them give
// up; 0 keeps the default.
template <typename T>
bool launch_tile(int mode, const T* X, size_t ldx, int nx, int u0, int nu, const T* Y, size_t ldy, int ny, size_t n,
                 const double* C, T* Yout, size_t ldo, double* out, double* part, unsigned* counter, const int* gate,
                 int mask, int* status, cudaStream_t st, const double* Cadd = nullptr, int uadd = 0, int nadd = 0,
                 int polls = 0);
// Cholesky QR applied twice without storing X R1^{-1} (kernels_vec.cu): with
// gram, S2 = (X P1)^T (X P1); without, Q = (X P1) P2, projected on the tangent
// planes of m when m != NULL.  X: nx <= 8 fields; P1, P2: nx x nx FP64.  Both
// form X P1 with the same FMA chain, so they see the same rounded values.
template <typename T>
bool launch_chol2(const T* X, size_t ldx, int nx, const double* P1, const double* P2, T* Q, size_t ldq, const T* m,
                  int N, double* S2, double* part, unsigned* counter, const int* gate, int mask, bool gram,
                  cudaStream_t st);
// Block Lanczos: T(j, j) = sym of block row jr of the local Gram G1 (b x b
// blocks, row jr holding Q_j^T H Q_j).
void launch_arnoldi_diag(const double* G1, int b, int jr, int j, double* T, int ldT, DevState* st, cudaStream_t s);
// status word of the last context that set one (timeouts of bounded waits)
void set_gram_status(int* status);

// Site-wise combination of vector fields (3N elements, component-major):
//   out_c = beta * Y_c + sigma * sum_{r < nx} X_r C[r*ny + c]      (c < ny <= 8)
// nx is read from *nx_dev when nx_dev != NULL (then nx_max bounds it).
// If m != NULL the result is projected on the tangent planes of m.
// Y may alias out (in-place), X must not.
template <typename T>
void launch_combine(const T* X, size_t ldx, int nx, const int* nx_dev, const double* C, int ny, const T* Y,
                    size_t ldy, double beta, double sigma, T* out, size_t ldo, const T* m, int N, const int* gate,
                    int mask, cudaStream_t st);

// out_j = P(in_j) for nvec fields (in may alias out).
template <typename T>
void launch_project(const T* m, const T* in, size_t ldi, T* out, size_t ldo, int nvec, int N, const int* gate,
                    int mask, cudaStream_t st);

// Ritz finishing: V_c <- P(V_c) / |P(V_c)| * sign, sign making the entry of
// largest magnitude positive (lowest flat index on ties).  Two launches.
template <typename T>
void launch_finish(const T* m, T* V, size_t ldv, int k, int N, double* part, unsigned* counter, double* scal,
                   const int* gate, int mask, cudaStream_t st);

// ---- small dense FP64 steps, one block each ----
// Block Lanczos, after A = Q_j^T H Q_j: symmetrise into T(j,j), build the
// three-term coefficients [R_j^T ; A] (rows for Q_{j-1}, Q_j) into C3.
void launch_lanczos_coeffs(const double* A, int b, int j, double* T, int ldT, double* C3, DevState* st,
                           cudaStream_t s);
// Cholesky QR step on G (b x b): writes Rinv (b x b, coefficient matrix) and
// accumulates R.  second != 0: final pass of CholQR2; then R is placed at
// T(j+1, j) / T(j, j+1) (when j >= 0) and st->steps advanced.  Breakdown sets
// kGateKrylov.
void launch_cholqr(const double* G, int b, int second, int j, double* Rinv, double* Racc, double* T, int ldT,
                   DevState* st, double rel_tol, cudaStream_t s, int skip = 0);
// Selective reorthogonalisation (kernels_omega.cu): estimates of Q_{j+1}^T Q_k
// from the block recurrence, the decision (gate bit kGateNoReorth), and the
// restart of the estimates after a full pass.  Om: MOTO_MAX_BASIS^2 doubles.
void launch_omega_estimate(int b, int j, const double* T, int ldT, const double* Rn, double* Om, double* rlog,
                           DevState* st, double eps, cudaStream_t s);
void launch_omega_reset(int b, int j, const double* Rn, double* Om, DevState* st, double eps, cudaStream_t s);
// Symmetric eigensolver (cyclic Jacobi, FP64) on the leading nT x nT block of
// T (nT read from st->nT, <= 96): theta ascending (MOTO_MAX_BASIS entries,
// +inf padded) and the first k eigenvectors as an (nT x k) coefficient matrix Y.
void launch_small_eig(const double* T, int ldT, double* theta, double* Y, int k, DevState* st, cudaStream_t s);
// Same contract, by Householder tridiagonalisation (skipped for band 1),
// Sturm bisection and inverse iteration (kernels_eig.cu).
void launch_tridiag_eig(const double* T, int ldT, int band, int fp64, double* theta, double* Y, int k, DevState* st,
                        cudaStream_t s);

// LOBPCG small steps (see kernels_vec.cu)
void launch_lob_rr(const double* Gb, const double* Mb, int k, int nb, double drop, double* Cx, double* Cp,
                   double* theta, DevState* st, cudaStream_t s);
void launch_lob_check(const double* Gw, int k, double tol, const double* theta, DevState* st, cudaStream_t s);
// mode 0: out = diag(src[0..k));  mode 1: out = diag(1 / sqrt(src[j*k + j]))
void launch_diag(const double* src, int k, int mode, double* out, const DevState* st, int mask, cudaStream_t s);

// ---- L-BFGS / MMF ----
// G = g - 2 sum_c dots[c] V_c over nv fields of V (nv = 0: G = g), and
// fmax_out = max_i |G_i|
template <typename T>
void launch_mmf_force(const T* g, const T* V, size_t ldv, int nv, const double* dots, T* G, int N, double* part,
                      unsigned* counter, double* fmax_out, const int* gate, int mask, cudaStream_t st);
// Nonlinear CG (Polak-Ribiere+).  cg (doubles): [0..8] the 3 x 3 Gram of
// [G, s, y] (row-major: G.G at 0, s.s at 4, s.y at 5, y.G at 6, y.y at 8),
// [9] |G_prev|^2 (kept), [10] beta, [11] step length.  cg_coeffs forms beta and the length and sets
// lb_have_prev; cg_direction writes p = -G + beta P p (p: the previous
// direction on entry) and decides restart (pad[2]) and the capped scale;
// cg_retract takes d = scale * (restart ? -G : p) and retracts.
void launch_cg_coeffs(double* cg, double gamma0, DevState* dst, cudaStream_t st);
template <typename T>
void launch_cg_direction(const T* m, const T* G, T* p, int N, const double* cg, double theta_max, double* part,
                         unsigned* counter, DevState* dst, const int* gate, int mask, cudaStream_t st);
template <typename T>
void launch_cg_retract(T* m, const T* G, T* p, T* d, const DevState* dst, int N, const int* gate, int mask,
                       cudaStream_t st);
template <typename T>
void launch_lbfgs_pair(const T* m, const T* d_prev, const T* G_prev, const T* G, T* ring, size_t ld, T* stage,
                       const DevState* dst, int N, const int* gate, int mask, cudaStream_t st);
void launch_lbfgs_solve(double* M, int mem, const double* newdots, double gamma0, double* coef, DevState* dst,
                        cudaStream_t st);
template <typename T>
void launch_lbfgs_direction(const T* basis, size_t ld, int nb, const double* coef, const T* m, T* d, int N,
                            double theta_max, double* part, unsigned* counter, DevState* dst, const int* gate,
                            int mask, cudaStream_t st);
template <typename T>
void launch_retract(T* m, T* d, const DevState* dst, int N, const int* gate, int mask, cudaStream_t st);
template <typename T>
void launch_descent_seed(const T* m, const T* v1, double eta_theta, double sign, T* out, int N, double* part,
                         unsigned* counter, double* scal, cudaStream_t st);
// ---- explorer front-end (kernels_explorer.cu) ----
// out_j = R_x0(P_mask P_x0 delta_j), j < count (mask: N bytes, NULL = all)
template <typename T>
void launch_perturb(const T* x0, const unsigned char* mask, const T* delta, size_t ldd, int count, T* out,
                    size_t ldo, int N, cudaStream_t st);
// D (P x P) = pairwise L1 distances of P <= MOTO_MAX_POP fields of n
// elements; false (nothing launched) when P or the scratch is out of range
template <typename T>
bool launch_pairwise_l1(const T* X, size_t ldx, int P, size_t n, double* part, size_t part_cap, unsigned* counter,
                        double* D, cudaStream_t st);

// Damped spin dynamics (Heun): predictor mp = unit(m + dt f(m, g)); corrector
// m <- unit(m + dt/2 (f(m, g0) + f(mp, g1))), f(m, g) = (m x g - alpha g) /
// (1 + alpha^2) with g the Riemannian gradient
template <typename T>
void launch_llg_predict(const T* m, const T* g, T* mp, double alpha, double dt, int N, const int* gate, int mask,
                        cudaStream_t st);
template <typename T>
void launch_llg_correct(T* m, const T* g0, const T* mp, const T* g1, double alpha, double dt, int N,
                        const int* gate, int mask, cudaStream_t st);

// indexed > 0: out6 is a trace of `indexed` rows, the record goes to row
// min(outer steps taken, indexed - 1); 0: out6 is the record itself
void launch_saddle_test(const double* eg_out, const double* fmax, const double* lam, const double* gdot,
                        double tau_F, double tau_lambda, double* out6, int* status_out, DevState* dst, int ascent,
                        int last, int indexed, cudaStream_t st);

}  // namespace moto
