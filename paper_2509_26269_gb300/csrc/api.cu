// C ABI of the minimum-mode kernel: context and workspace management and the
// host-side sequencing of the device steps.  Control stays on the device
// (gate bits, step counters, convergence flags); the host only enqueues
// launches, except moto_ascend / moto_descend / moto_status which read a
// status word back.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <tuple>
#include <vector>

#include "internal.h"

using namespace moto;

namespace moto {
WalkerGrid& walker_grid() {
  thread_local WalkerGrid g{1, 0};
  return g;
}
}  // namespace moto

struct moto_ctx {
  ModelDev md;
  double* pairs;  // pair-list storage, MOTO_MAX_PAIRS x [d1, d2, J, Dx, Dy, Dz]
  int dtype;
  size_t esize;
  moto_params p;  // sizing parameters given at creation
  int N;
  size_t n3;  // 3N
  size_t ld;  // element stride of internal vector fields
  // device scratch
  void* basis;  // MOTO_MAX_BASIS fields
  void* W;      // MOTO_MAX_K fields
  void* Wt;     // MOTO_MAX_K fields
  void* g;      // gradient
  void* s;      // s_i (N)
  void* ring;   // L-BFGS: 2(mem+1) pair slots, G, G_prev, d, 2 staging
  void* lob;    // LOBPCG blocks: 2 sets x [X, W, P, AX, AW, AP] (12 x MOTO_MAX_K fields)
  double* dsm;  // small dense area
  double* part;
  unsigned* counter;
  DevState* st;
  size_t part_len;
  size_t bytes;
  // launch profiler (moto_profile_*): events around each launch of the
  // Krylov / optimiser sequences, tagged with a kernel class and the
  // algorithmic bytes that launch moves
  int prof_on, prof_n, prof_cap;
  cudaEvent_t* prof_ev;
  int* prof_kind;
  double* prof_bytes;
  int* prof_cond;    // >= 0: the launch ran only if step prof_cond's full pass was taken
  int prof_cond_cur;  // the step of the conditional launches being enqueued (-1: none)
  cudaStream_t prof_stream;
  // bound of the streaming kernel's consumer waits (moto_set_wait_limit; 0 = default)
  int wait_polls;
  // HVP variant: forced by moto_set_hvp_variant (>= 0) or the autotuner's
  // choice; per-variant times of the autotuner run that chose it
  int hvp_force;
  int hvp_nvec;
  float hvp_ms[16];
  int hvp_tuned_here;
  // energy / gradient stencil variant: forced (>= 0) or the autotuner's
  int stencil_force;
  float stencil_ms[8];
  int stencil_tuned_here;
  int last_selective;  // the last block Lanczos solve reorthogonalised selectively
  // walker group (batches): nw walkers whose scratch and fields lie in
  // equally sized slices (wstride bytes) of one allocation, `arena`; the
  // pointers above address slice 0.  Slots for the walkers' spins, modes and
  // descent copies follow the scratch in each slice.
  int nw;
  size_t wstride;
  void* arena;
  void *mslot, *Vslot, *mpslot, *mmslot;
  // moto_mmf_step replayed as a CUDA graph when the same arguments come back:
  // the key of the last call, how many calls in a row had it, the captured
  // step (on a private stream), and a generation that every setter of a
  // captured launch parameter bumps
  int gen;
  int step_seen;
  int step_gen;
  void *step_m, *step_V;
  double* step_out;
  int* step_status;
  moto_params step_p;
  cudaStream_t step_stream;
  cudaGraphExec_t step_exec;
};

namespace {
struct ProfScope {
  moto_ctx* c;
  bool on;
  ProfScope(moto_ctx* c_, int kind, double bytes, cudaStream_t st) : c(c_), on(false) {
    if (c->prof_on && c->prof_n < c->prof_cap) {
      on = true;
      c->prof_kind[c->prof_n] = kind;
      c->prof_bytes[c->prof_n] = bytes;
      c->prof_cond[c->prof_n] = c->prof_cond_cur;
      cudaEventRecord(c->prof_ev[2 * c->prof_n], st);
      c->prof_stream = st;
    }
  }
  ~ProfScope() {
    if (on) {
      cudaEventRecord(c->prof_ev[2 * c->prof_n + 1], c->prof_stream);
      c->prof_n += 1;
    }
  }
};
}  // namespace
#define MOTO_CAT2(a, b) a##b
#define MOTO_CAT(a, b) MOTO_CAT2(a, b)
#define PROF(kind, bytes) ProfScope MOTO_CAT(prof_scope_, __LINE__)(c, (kind), (double)(bytes), st)

// kernel classes of the profiler
enum {
  kPkHvp = 0,
  kPkGram = 1,
  kPkCombine = 2,
  kPkStencil = 3,
  kPkSmall = 4,
  kPkVec = 5,
  kPkEig = 6,
  kPkReorthGram = 7,
  kPkReorthUpd = 8,
  kPkChol2 = 9,
  kPkCount = 10
};

namespace {
// Profiled launch wrappers: same arguments as the launchers, plus the context.
// Bytes are the algorithmic traffic of the launch (each field read or written
// once).
template <typename T>
void P_gram(moto_ctx* c, const T* X, size_t ldx, int nx, const T* Y, size_t ldy, int ny, size_t n, double* out,
            double* part, unsigned* counter, const int* gate, int mask, cudaStream_t st) {
  PROF(kPkGram, (double)((X == Y) ? nx : nx + ny) * n * sizeof(T));
  set_gram_status(&c->st->status);
  launch_gram<T>(X, ldx, nx, Y, ldy, ny, n, out, part, counter, gate, mask, st);
}
template <typename T>
void P_combine(moto_ctx* c, const T* X, size_t ldx, int nx, const int* nx_dev, const double* C, int ny, const T* Y,
               size_t ldy, double beta, double sigma, T* out, size_t ldo, const T* m, int N, const int* gate, int mask,
               cudaStream_t st) {
  const double f = 3.0 * N * sizeof(T);
  PROF(kPkCombine, f * (nx + ny + (beta != 0.0 ? ny : 0) + (m ? 1 : 0)));
  launch_combine<T>(X, ldx, nx, nx_dev, C, ny, Y, ldy, beta, sigma, out, ldo, m, N, gate, mask, st);
}
template <typename T>
void P_hvp(moto_ctx* c, const ModelDev& md, const T* m, const T* s, const T* V, size_t ldv, T* HV, size_t ldhv,
           int nvec, const int* gate, int mask, cudaStream_t st) {
  PROF(kPkHvp, (4.0 + 6.0 * nvec) * md.N * sizeof(T));
  if (c->hvp_force >= 0 && md.npairs == 0)
    launch_hvp_strip_variant<T>(c->hvp_force, md, m, s, V, ldv, HV, ldhv, nvec, gate, mask, st);
  else
    launch_hvp<T>(md, m, s, V, ldv, HV, ldhv, nvec, gate, mask, st);
}
template <typename T>
void P_energy_grad(moto_ctx* c, const ModelDev& md, const T* m, T* g, T* s, double* part, unsigned* counter,
                   double* out, int* status, bool fp64, cudaStream_t st) {
  PROF(kPkStencil, (3.0 + (g ? 3.0 : 0.0) + (s ? 1.0 : 0.0)) * md.N * sizeof(T));
  if (c->stencil_force >= 0 && md.npairs == 0 && !fp64)
    launch_energy_grad_variant<T>(c->stencil_force, md, m, g, s, part, counter, out, status, st);
  else
    launch_energy_grad<T>(md, m, g, s, part, counter, out, status, fp64, st);
}
template <typename T>
void P_project(moto_ctx* c, const T* m, const T* in, size_t ldi, T* out, size_t ldo, int nvec, int N, const int* gate,
               int mask, cudaStream_t st) {
  PROF(kPkVec, (3.0 + 6.0 * nvec) * N * sizeof(T));
  launch_project<T>(m, in, ldi, out, ldo, nvec, N, gate, mask, st);
}
template <typename T>
void P_finish(moto_ctx* c, const T* m, T* V, size_t ldv, int k, int N, double* part, unsigned* counter, double* scal,
              const int* gate, int mask, cudaStream_t st) {
  PROF(kPkVec, (6.0 + 9.0 * k) * N * sizeof(T));
  launch_finish<T>(m, V, ldv, k, N, part, counter, scal, gate, mask, st);
}
template <typename T>
void P_mmf_force(moto_ctx* c, const T* g, const T* V, size_t ldv, int nv, const double* dots, T* G, int N,
                 double* part, unsigned* counter, double* fmax_out, const int* gate, int mask, cudaStream_t st) {
  PROF(kPkVec, (6.0 + 3.0 * nv) * N * sizeof(T));
  launch_mmf_force<T>(g, V, ldv, nv, dots, G, N, part, counter, fmax_out, gate, mask, st);
}
template <typename T>
void P_llg_predict(moto_ctx* c, const T* m, const T* g, T* mp, double alpha, double dt, int N, const int* gate,
                   int mask, cudaStream_t st) {
  PROF(kPkVec, 9.0 * N * sizeof(T));
  launch_llg_predict<T>(m, g, mp, alpha, dt, N, gate, mask, st);
}
template <typename T>
void P_llg_correct(moto_ctx* c, T* m, const T* g0, const T* mp, const T* g1, double alpha, double dt, int N,
                   const int* gate, int mask, cudaStream_t st) {
  PROF(kPkVec, 15.0 * N * sizeof(T));
  launch_llg_correct<T>(m, g0, mp, g1, alpha, dt, N, gate, mask, st);
}
template <typename T>
void P_cg_direction(moto_ctx* c, const T* m, const T* G, T* p, int N, const double* cg, double theta_max,
                    double* part, unsigned* counter, DevState* dst, const int* gate, int mask, cudaStream_t st) {
  PROF(kPkVec, 12.0 * N * sizeof(T));
  launch_cg_direction<T>(m, G, p, N, cg, theta_max, part, counter, dst, gate, mask, st);
}
template <typename T>
void P_cg_retract(moto_ctx* c, T* m, const T* G, T* p, T* d, const DevState* dst, int N, const int* gate, int mask,
                  cudaStream_t st) {
  PROF(kPkVec, 18.0 * N * sizeof(T));
  launch_cg_retract<T>(m, G, p, d, dst, N, gate, mask, st);
}
template <typename T>
void P_lbfgs_pair(moto_ctx* c, const T* m, const T* d_prev, const T* G_prev, const T* G, T* ring, size_t ld, T* stage,
                  const DevState* dst, int N, const int* gate, int mask, cudaStream_t st) {
  PROF(kPkVec, 24.0 * N * sizeof(T));
  launch_lbfgs_pair<T>(m, d_prev, G_prev, G, ring, ld, stage, dst, N, gate, mask, st);
}
template <typename T>
void P_lbfgs_direction(moto_ctx* c, const T* basis, size_t ld, int nb, const double* coef, const T* m, T* d, int N,
                       double theta_max, double* part, unsigned* counter, DevState* dst, const int* gate, int mask,
                       cudaStream_t st) {
  PROF(kPkVec, (3.0 * nb + 6.0) * N * sizeof(T));
  launch_lbfgs_direction<T>(basis, ld, nb, coef, m, d, N, theta_max, part, counter, dst, gate, mask, st);
}
template <typename T>
void P_retract(moto_ctx* c, T* m, T* d, const DevState* dst, int N, const int* gate, int mask, cudaStream_t st) {
  PROF(kPkVec, 12.0 * N * sizeof(T));
  launch_retract<T>(m, d, dst, N, gate, mask, st);
}
// Streaming reorthogonalisation step (see internal.h, modes 0-3) with the
// combine + Gram fallback for fields that break the TMA alignment rules.  In
// mode 1 only X rows u0 .. u0 + nu - 1 take part in the update.
template <typename T>
void P_tile(moto_ctx* c, int mode, const T* X, int nx, int u0, int nu, T* Y, int ny, const double* C, T* Yout,
            double* out, const int* gate, int mask, cudaStream_t st, const double* Cadd = nullptr, int uadd = 0,
            int nadd = 0) {
  const size_t ld = c->ld;
  const int N = c->N;
  bool done;
  {
    const double f = 3.0 * N * sizeof(T);
    const double fields = (mode == 0 || (mode == 1 && !Yout)) ? nx + ny : (mode == 3 ? nx + ny : nx + 2.0 * ny);
    PROF(mode == 1 ? kPkReorthGram : (mode == 2 ? kPkReorthUpd : kPkGram), f * fields);
    set_gram_status(&c->st->status);
    done = launch_tile<T>(mode, X, ld, nx, u0, nu, Y, ld, ny, c->n3, C, Yout, ld, out, c->part, c->counter, gate,
                          mask, &c->st->status, st, Cadd, uadd, nadd, c->wait_polls);
  }
  if (done) return;
  switch (mode) {
    case 0:
      P_gram<T>(c, X, ld, nx, Y, ld, ny, c->n3, out, c->part, c->counter, gate, mask, st);
      break;
    case 1: {
      // unstored update: the updated fields go to the scratch block
      T* U = Yout ? Y : static_cast<T*>(c->Wt);
      P_combine<T>(c, X + (size_t)u0 * ld, ld, nu, nullptr, C, ny, Y, ld, 1.0, -1.0, U, ld, nullptr, N, gate, mask,
                   st);
      P_gram<T>(c, X, ld, nx, U, ld, ny, c->n3, out, c->part, c->counter, gate, mask, st);
      break;
    }
    case 2:
      if (Cadd)
        P_combine<T>(c, X + (size_t)uadd * ld, ld, nadd, nullptr, Cadd, ny, Y, ld, 1.0, -1.0, Y, ld, nullptr, N, gate,
                     mask, st);
      P_combine<T>(c, X, ld, nx, nullptr, C, ny, Y, ld, 1.0, -1.0, Y, ld, nullptr, N, gate, mask, st);
      P_gram<T>(c, Y, ld, ny, Y, ld, ny, c->n3, out, c->part, c->counter, gate, mask, st);
      break;
    default:
      P_combine<T>(c, X, ld, nx, nullptr, C, ny, nullptr, 0, 0.0, 1.0, Yout, ld, nullptr, N, gate, mask, st);
      P_gram<T>(c, Yout, ld, ny, Yout, ld, ny, c->n3, out, c->part, c->counter, gate, mask, st);
      break;
  }
}

__global__ void set_status_kernel(DevState* st, int bits, size_t ws) {
  st = wofs(st, ws);
  if (threadIdx.x == 0) st->status |= bits;
}

// Cholesky QR, second pass: Gram of W R1^{-1} (read-only sweep) and the
// final combination Q = (W R1^{-1}) R2^{-1} (projected), W R1^{-1} never stored.
template <typename T>
void P_chol2_gram(moto_ctx* c, const T* W, int b, const double* R1inv, double* S2, const int* gate, int mask,
                  cudaStream_t st) {
  PROF(kPkChol2, (double)b * 3.0 * c->N * sizeof(T));
  if (!launch_chol2<T>(W, c->ld, b, R1inv, nullptr, nullptr, 0, nullptr, c->N, S2, c->part, c->counter, gate, mask,
                       true, st))
    set_status_kernel<<<wgrid(1), 1, 0, st>>>(c->st, kStatusNotSPD, walker_ws());
}
template <typename T>
void P_combine2(moto_ctx* c, const T* W, int b, const double* R1inv, const double* R2inv, T* Q, const T* m,
                const int* gate, int mask, cudaStream_t st) {
  PROF(kPkCombine, (2.0 * b + (m ? 1 : 0)) * 3.0 * c->N * sizeof(T));
  launch_chol2<T>(W, c->ld, b, R1inv, R2inv, Q, c->ld, m, c->N, nullptr, nullptr, nullptr, gate, mask, false, st);
}

#define SMALL_WRAP(name)                                                 \
  template <typename... A>                                               \
  void P_##name(moto_ctx* c, A... args) {                                \
    cudaStream_t st = std::get<sizeof...(A) - 1>(std::make_tuple(args...)); \
    PROF(kPkSmall, 0.0);                                                 \
    launch_##name(args...);                                              \
  }
SMALL_WRAP(lanczos_coeffs)
SMALL_WRAP(cholqr)
SMALL_WRAP(small_eig)
SMALL_WRAP(lob_rr)
SMALL_WRAP(lob_check)
SMALL_WRAP(diag)
SMALL_WRAP(lbfgs_solve)
SMALL_WRAP(saddle_test)
SMALL_WRAP(cg_coeffs)
SMALL_WRAP(arnoldi_diag)
SMALL_WRAP(omega_estimate)
SMALL_WRAP(omega_reset)
#undef SMALL_WRAP
// Cholesky QR pass that also skips when a gate bit of `skip` is set
void P_cholqr_skip(moto_ctx* c, const double* G, int b, int second, int j, double* Rinv, double* Racc, double* T,
                   int ldT, DevState* dst, double rel, int skip, cudaStream_t st) {
  PROF(kPkSmall, 0.0);
  launch_cholqr(G, b, second, j, Rinv, Racc, T, ldT, dst, rel, st, skip);
}
void P_tridiag_eig(moto_ctx* c, const double* T, int ldT, int band, double* theta, double* Y, int k, DevState* dst,
                   cudaStream_t st) {
  PROF(kPkEig, 0.0);
  launch_tridiag_eig(T, ldT, band, c->dtype == MOTO_F64 ? 1 : 0, theta, Y, k, dst, st);
}
}  // namespace

namespace {

// small dense layout (doubles)
constexpr size_t kT = 0;                                           // T: MAX_BASIS^2
constexpr size_t kTheta = kT + MOTO_MAX_BASIS * MOTO_MAX_BASIS;    // MAX_BASIS
constexpr size_t kY = kTheta + MOTO_MAX_BASIS;                     // MAX_BASIS * MAX_K
constexpr size_t kC = kY + MOTO_MAX_BASIS * MOTO_MAX_K;            // MAX_BASIS * MAX_K
constexpr size_t kC3 = kC + MOTO_MAX_BASIS * MOTO_MAX_K;           // 2K * K
constexpr size_t kC2 = kC3 + 2 * MOTO_MAX_K * MOTO_MAX_K;          // MAX_BASIS * MAX_K (second CGS pass)
constexpr size_t kRinv2 = kC2 + MOTO_MAX_BASIS * MOTO_MAX_K;       // K*K (second Cholesky QR factor)
constexpr size_t kG = kRinv2 + MOTO_MAX_K * MOTO_MAX_K;            // K*K
constexpr size_t kRinv = kG + MOTO_MAX_K * MOTO_MAX_K;             // K*K
constexpr size_t kRacc = kRinv + MOTO_MAX_K * MOTO_MAX_K;          // K*K
constexpr size_t kEG = kRacc + MOTO_MAX_K * MOTO_MAX_K;            // 2: [E, gmax]
constexpr size_t kFmax = kEG + 2;                                  // 1
constexpr size_t kScal = kFmax + 1;                                // MAX_K
constexpr size_t kLbM = kScal + MOTO_MAX_K;                        // (2(mem+1)+1)^2
constexpr size_t kLbMsz = (2 * MOTO_MAX_MEM + 3) * (2 * MOTO_MAX_MEM + 3);
constexpr size_t kLbNew = kLbM + kLbMsz;                           // 3 * (2(mem+1)+1)
constexpr size_t kLbCoef = kLbNew + 3 * (2 * MOTO_MAX_MEM + 3);    // 2(mem+1)+1
constexpr size_t kTmp = kLbCoef + (2 * MOTO_MAX_MEM + 3);          // 8 scratch doubles
constexpr size_t kLobG = kTmp + 8;                                 // 3K x 3K (LOBPCG Gram)
constexpr size_t kLobM = kLobG + 9 * MOTO_MAX_K * MOTO_MAX_K;      // 3K x 3K
constexpr size_t kLobC = kLobM + 9 * MOTO_MAX_K * MOTO_MAX_K;      // 3K x 2K coefficient blocks
constexpr size_t kLobAux = kLobC + 6 * MOTO_MAX_K * MOTO_MAX_K;    // 64 aux
constexpr size_t kMmfDots = kLobAux + 64 * MOTO_MAX_K;             // MAX_K: g . V_c (subspace force)
constexpr size_t kCg = kMmfDots + MOTO_MAX_K;                      // 12: Gram of [G, s, y], |G_prev|^2, beta, alpha
constexpr size_t kOm = kCg + 12;                                   // MAX_BASIS^2: orthogonality estimates
constexpr size_t kBout = kOm + MOTO_MAX_BASIS * MOTO_MAX_BASIS;  // 8: a batch walker's descent record
constexpr size_t kRlog = kBout + 8;                                // MAX_BASIS: full pass taken at step j (1/0)
constexpr size_t kDsmSize = kRlog + MOTO_MAX_BASIS;

constexpr int kLd = MOTO_MAX_BASIS;  // leading dimension of T

// A failed CUDA call makes the entry point return MOTO_ERR_CUDA; with the
// environment variable MOTO_DEBUG set, its error string and site go to stderr.
inline int cuda_fail(cudaError_t e, const char* what, int line) {
  static const bool dbg = getenv("MOTO_DEBUG") != nullptr;
  if (dbg) fprintf(stderr, "moto: %s failed at api.cu:%d: %s\n", what, line, cudaGetErrorString(e));
  return MOTO_ERR_CUDA;
}
#define CK(x)                                                    \
  do {                                                           \
    cudaError_t e_ = (x);                                        \
    if (e_ != cudaSuccess) return cuda_fail(e_, #x, __LINE__);   \
  } while (0)

inline cudaStream_t S(void* s) { return (cudaStream_t)s; }

template <typename T>
T* F(void* base, size_t ld, int j) {
  return static_cast<T*>(base) + (size_t)j * ld;
}

__global__ void state_kernel(DevState* st, int op, size_t ws) {
  st = wofs(st, ws);
  if (threadIdx.x != 0) return;
  switch (op) {
    case 0:  // begin Krylov solve
      st->gate &= ~(kGateKrylov | kGateNoReorth);
      st->pad[3] = 0;
      st->pad[4] = 0;
      st->pad[5] = 0;
      st->steps = 0;
      st->nT = 0;
      st->tnorm = 0.0;
      st->iters = 0;
      break;
    case 1:  // reset optimiser (ascent or descent start)
      st->gate = 0;
      st->pad[1] = 0;
      st->lb_head = 0;
      st->lb_count = 0;
      st->lb_have_prev = 0;
      st->converged = 0;
      st->iters = 0;
      break;
    case 2:  // clear status
      st->status = 0;
      break;
    case 3:  // begin LOBPCG
      st->gate &= ~kGateKrylov;
      st->steps = 0;
      st->iters = 0;
      st->hnorm = 0.0;
      st->pad[0] = 0;
      break;
    case 4:  // a standalone solve: an earlier ascent or descent may have left its done bit
      st->gate &= ~kGateDone;
      break;
  }
}

__global__ void info_kernel(const DevState* st, int* info, size_t ws) {
  st = wofs(st, ws);
  info = wofs(info, ws);
  if (threadIdx.x != 0) return;
  info[0] = st->steps + st->iters;  // block steps (Lanczos) or iterations (LOBPCG)
  info[1] = st->status;
}

__global__ void count_step_kernel(DevState* st) {
  if (threadIdx.x == 0 && !(st->gate & kGateDone)) st->iters += 1;
}

int check_params(const moto_params* p) {
  if (!p) return MOTO_ERR_ARG;
  if (p->k < 1 || p->k > MOTO_MAX_K) return MOTO_ERR_ARG;
  if (p->solver != MOTO_SOLVER_LANCZOS && p->solver != MOTO_SOLVER_LOBPCG) return MOTO_ERR_ARG;
  if (p->solver == MOTO_SOLVER_LANCZOS) {
    if (p->block < p->k || p->block > MOTO_MAX_K) return MOTO_ERR_ARG;
    if (p->krylov_steps < 1 || p->block * p->krylov_steps > MOTO_MAX_BASIS) return MOTO_ERR_ARG;
    if (p->block * p->krylov_steps < 2) return MOTO_ERR_ARG;
  } else {
    if (p->max_iter < 0) return MOTO_ERR_ARG;
  }
  if (p->lbfgs_mem < 1 || p->lbfgs_mem > MOTO_MAX_MEM) return MOTO_ERR_ARG;
  if (!(p->theta_max > 0.0) || !(p->gamma0 > 0.0) || !(p->tau_F >= 0.0) || !(p->eta_theta > 0.0))
    return MOTO_ERR_ARG;
  if (p->max_steps < 0 || p->descent_max_steps < 0) return MOTO_ERR_ARG;
  if (p->optimizer != MOTO_OPT_LBFGS && p->optimizer != MOTO_OPT_CG) return MOTO_ERR_ARG;
  if (p->subspace != 0 && p->subspace != 1) return MOTO_ERR_ARG;
  if (p->descent != MOTO_DESCENT_OPT && p->descent != MOTO_DESCENT_LLG) return MOTO_ERR_ARG;
  if (!(p->llg_alpha >= 0.0) || !(p->llg_dt > 0.0) || !(p->llg_time >= 0.0)) return MOTO_ERR_ARG;
  if (p->descent == MOTO_DESCENT_LLG && p->llg_time / p->llg_dt > 1e8) return MOTO_ERR_ARG;
  if (p->reorth != MOTO_REORTH_FULL && p->reorth != MOTO_REORTH_SELECTIVE) return MOTO_ERR_ARG;
  if (!(p->tau_lambda >= 0.0) || !std::isfinite(p->tau_lambda)) return MOTO_ERR_ARG;
  return MOTO_OK;
}

// ----------------------------------------------------------------------------
// block Lanczos (block size b, `steps` block steps), Ritz vectors of the
// nout lowest Ritz values into V
// ----------------------------------------------------------------------------
template <typename T>
void block_lanczos(moto_ctx* c, const T* m, const T* s, const T* v0, size_t ld0, int b, int steps, T* V, size_t ldv,
                   int nout, double* lam, cudaStream_t st, bool selective = false) {
  const int N = c->N;
  const size_t n3 = c->n3, ld = c->ld;
  T* Q = static_cast<T*>(c->basis);
  T* W = static_cast<T*>(c->W);
  double* D = c->dsm;
  int* gate = &c->st->gate;
  const int mk = kGateKrylov | kGateDone;
  const double rel = (c->dtype == MOTO_F64) ? 1e-12 : 1e-6;
  // unit roundoff of the stored fields (selective reorthogonalisation)
  const double eps = (c->dtype == MOTO_F64) ? 0x1p-53 : 0x1p-24;
  c->last_selective = selective ? 1 : 0;
  state_kernel<<<wgrid(1), 32, 0, st>>>(c->st, 0, walker_ws());
  // start block: project, Cholesky QR twice
  P_project<T>(c, m, v0, ld0, W, ld, b, N, gate, kGateDone, st);
  P_gram<T>(c, W, ld, b, W, ld, b, n3, D + kG, c->part, c->counter, gate, mk, st);
  P_cholqr(c, D + kG, b, 0, -1, D + kRinv, D + kRacc, D + kT, kLd, c->st, rel, st);
  P_chol2_gram<T>(c, W, b, D + kRinv, D + kG, gate, mk, st);
  P_cholqr(c, D + kG, b, 1, -1, D + kRinv2, D + kRacc, D + kT, kLd, c->st, rel, st);
  P_combine2<T>(c, W, b, D + kRinv, D + kRinv2, Q, nullptr, gate, mk, st);
  // Block Lanczos step j, reorthogonalised twice: W = H Q_j; A = Q_j^T W gives
  // T(j, j) = sym(A); the local pass W1 = W - Q_j T(j, j) - Q_{j-1} R_j^T (the
  // three-term recurrence) is formed in registers only, for G2 = Q^T W1 over
  // the whole basis (a read-only sweep); the full pass then writes
  // W <- W - [Q_{j-1}, Q_j] C3 - Q G2 (= W1 - Q G2) with S = W^T W in the same
  // sweep; Cholesky QR of W (twice) gives Q_{j+1} and R_{j+1} = T(j+1, j).  The
  // new block is re-projected on the tangent planes in its final combination
  // (a small beta would otherwise magnify rounding-level normal components
  // step after step).  The basis is read twice per step, W written once.
  for (int j = 0; j < steps; ++j) {
    T* Qj = Q + (size_t)j * b * ld;
    const int nq = (j + 1) * b;
    const int jl = j > 0 ? 1 : 0;  // local block rows: Q_{j-1} (if any), Q_j
    P_hvp<T>(c, c->md, m, s, Qj, ld, W, ld, b, gate, mk, st);
    P_tile<T>(c, 0, Qj, b, 0, 0, W, b, nullptr, nullptr, D + kC, gate, mk, st);
    // T(j, j) = sym(Q_j^T H Q_j); local coefficients [R_j^T; T(j, j)]
    P_lanczos_coeffs(c, D + kC, b, j, D + kT, kLd, D + kC3, c->st, st);
    if (j == steps - 1) break;
    if (selective) {
      // local three-term pass, stored, with the Gram of its result; the
      // tentative factor feeds the orthogonality estimate, which decides
      // whether the full pass against the basis (mode-0 Gram, then the
      // update with the Cholesky Gram) runs this step
      P_tile<T>(c, 2, Q + (size_t)(j - jl) * b * ld, (jl + 1) * b, 0, 0, W, b, D + kC3, W, D + kG, gate, mk, st);
      P_cholqr(c, D + kG, b, 0, j, D + kRinv, D + kRacc, D + kT, kLd, c->st, rel, st);
      P_omega_estimate(c, b, j, D + kT, kLd, D + kRacc, D + kOm, D + kRlog, c->st, eps, st);
      c->prof_cond_cur = j;  // the launches below do their work only if the estimate asked
      P_tile<T>(c, 0, Q, nq, 0, 0, W, b, nullptr, nullptr, D + kC2, gate, mk | kGateNoReorth, st);
      P_tile<T>(c, 2, Q, nq, 0, nq, W, b, D + kC2, W, D + kG, gate, mk | kGateNoReorth, st);
      P_cholqr_skip(c, D + kG, b, 0, j, D + kRinv, D + kRacc, D + kT, kLd, c->st, rel, kGateNoReorth, st);
      P_omega_reset(c, b, j, D + kRacc, D + kOm, c->st, eps, st);
      c->prof_cond_cur = -1;
    } else {
      P_tile<T>(c, 1, Q, nq, (j - jl) * b, (jl + 1) * b, W, b, D + kC3, nullptr, D + kC2, gate, mk, st);
      P_tile<T>(c, 2, Q, nq, 0, nq, W, b, D + kC2, W, D + kG, gate, mk, st, D + kC3, (j - jl) * b, (jl + 1) * b);
      P_cholqr(c, D + kG, b, 0, j, D + kRinv, D + kRacc, D + kT, kLd, c->st, rel, st);
    }
    P_chol2_gram<T>(c, W, b, D + kRinv, D + kG, gate, mk, st);
    P_cholqr(c, D + kG, b, 1, j, D + kRinv2, D + kRacc, D + kT, kLd, c->st, rel, st);
    P_combine2<T>(c, W, b, D + kRinv, D + kRinv2, Q + (size_t)(j + 1) * b * ld, m, gate, mk, st);
  }
  P_tridiag_eig(c, D + kT, kLd, b, lam, D + kY, nout, c->st, st);
  P_combine<T>(c, Q, ld, b * steps, &c->st->nT, D + kY, nout, nullptr, 0, 0.0, 1.0, V, ldv, nullptr, N,
                    gate, kGateDone, st);
  P_finish<T>(c, m, V, ldv, nout, N, c->part, c->counter, D + kScal, gate, kGateDone, st);
  (void)n3;
}


// ----------------------------------------------------------------------------
// LOBPCG (block size k).  Two sets of blocks, each [X, W, P, AX, AW, AP] of k
// fields; the set holding the current X is tracked on the device (st->pad[0])
// so that a convergence stop in any iteration leaves the right block behind.
// ----------------------------------------------------------------------------
__global__ void fill_inf_kernel(double* lam, int from) {
  for (int i = from + threadIdx.x; i < MOTO_MAX_BASIS; i += blockDim.x) lam[i] = 1.0 / 0.0;
}

__global__ void lob_swap_kernel(DevState* st, int mask) {
  if (threadIdx.x == 0 && !(st->gate & mask)) st->pad[0] ^= 1;
}

template <typename T>
__global__ void copy_current_kernel(const T* set0, const T* set1, size_t n, const DevState* st, T* out, size_t ld,
                                    int k, size_t ldo) {
  if (st->gate & kGateDone) return;
  const T* src = st->pad[0] ? set1 : set0;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
    for (int c = 0; c < k; ++c) out[(size_t)c * ldo + e] = src[(size_t)c * ld + e];
}

template <typename T>
void lobpcg(moto_ctx* c, const T* m, const T* s, const T* v0, size_t ld0, int k, int max_iter, double tol, T* V,
            size_t ldv, double* lam, cudaStream_t st) {
  const int N = c->N;
  const size_t n3 = c->n3, ld = c->ld;
  double* D = c->dsm;
  int* gate = &c->st->gate;
  const int mk = kGateKrylov | kGateDone;
  // SVQB drop level: a kept direction with scaled Gram eigenvalue w magnifies
  // the rounding of AS (~eps |H|) by 1/w in the projected matrix, so FP32
  // fields keep only directions with w > 1e-3
  const double drop = (c->dtype == MOTO_F64) ? 1e-12 : 1e-3;
  T* base = static_cast<T*>(c->lob);
  T* Wt = static_cast<T*>(c->Wt);
  auto SET = [&](int a) { return base + (size_t)a * 6 * MOTO_MAX_K * ld; };
  auto blk = [&](T* S, int j) { return S + (size_t)j * k * ld; };  // 0 X, 1 W, 2 P, 3 AX, 4 AW, 5 AP
  double* Gb = D + kLobG;
  double* Mb = D + kLobM;
  double* Cx = D + kLobC;
  double* Cp = Cx + 3 * k * k;
  state_kernel<<<wgrid(1), 32, 0, st>>>(c->st, 3, walker_ws());
  fill_inf_kernel<<<1, 128, 0, st>>>(lam, k);
  // initial Rayleigh-Ritz on span(P v0)
  T* A = SET(0);
  T* B = SET(1);
  P_project<T>(c, m, v0, ld0, blk(A, 0), ld, k, N, gate, kGateDone, st);
  P_hvp<T>(c, c->md, m, s, blk(A, 0), ld, blk(A, 3), ld, k, gate, mk, st);
  P_gram<T>(c, blk(A, 0), ld, k, blk(A, 0), ld, k, n3, Gb, c->part, c->counter, gate, mk, st);
  P_gram<T>(c, blk(A, 0), ld, k, blk(A, 3), ld, k, n3, Mb, c->part, c->counter, gate, mk, st);
  P_lob_rr(c, Gb, Mb, k, 1, drop, Cx, Cp, lam, c->st, st);
  P_combine<T>(c, blk(A, 0), ld, k, nullptr, Cx, k, nullptr, 0, 0.0, 1.0, blk(B, 0), ld, nullptr, N, gate, mk, st);
  P_combine<T>(c, blk(A, 3), ld, k, nullptr, Cx, k, nullptr, 0, 0.0, 1.0, blk(B, 3), ld, nullptr, N, gate, mk, st);
  lob_swap_kernel<<<1, 32, 0, st>>>(c->st, mk);
  int a = 1;
  bool haveP = false;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(st, &cap);
  for (int it = 1; it <= max_iter; ++it) {
    A = SET(a);
    B = SET(1 - a);
    // residuals R = AX - X theta, projected
    P_diag(c, lam, k, 0, D + kC3, c->st, mk, st);
    P_combine<T>(c, blk(A, 0), ld, k, nullptr, D + kC3, k, blk(A, 3), ld, 1.0, -1.0, blk(A, 1), ld, m, N, gate, mk,
                      st);
    P_gram<T>(c, blk(A, 1), ld, k, blk(A, 1), ld, k, n3, D + kG, c->part, c->counter, gate, mk, st);
    P_lob_check(c, D + kG, k, tol, lam, c->st, st);
    // W <- orthonormal basis of (I - X X^T) R
    P_gram<T>(c, blk(A, 0), ld, k, blk(A, 1), ld, k, n3, D + kC, c->part, c->counter, gate, mk, st);
    P_combine<T>(c, blk(A, 0), ld, k, nullptr, D + kC, k, blk(A, 1), ld, 1.0, -1.0, blk(A, 1), ld, nullptr, N, gate,
                      mk, st);
    P_gram<T>(c, blk(A, 1), ld, k, blk(A, 1), ld, k, n3, D + kG, c->part, c->counter, gate, mk, st);
    P_cholqr(c, D + kG, k, 0, -2, D + kRinv, D + kRacc, D + kT, kLd, c->st, 0.0, st);
    P_combine<T>(c, blk(A, 1), ld, k, nullptr, D + kRinv, k, nullptr, 0, 0.0, 1.0, Wt, ld, nullptr, N, gate, mk, st);
    P_gram<T>(c, Wt, ld, k, Wt, ld, k, n3, D + kG, c->part, c->counter, gate, mk, st);
    P_cholqr(c, D + kG, k, 1, -2, D + kRinv, D + kRacc, D + kT, kLd, c->st, 0.0, st);
    P_combine<T>(c, Wt, ld, k, nullptr, D + kRinv, k, nullptr, 0, 0.0, 1.0, blk(A, 1), ld, nullptr, N, gate, mk, st);
    P_hvp<T>(c, c->md, m, s, blk(A, 1), ld, blk(A, 4), ld, k, gate, mk, st);
    if (haveP) {
      P_gram<T>(c, blk(A, 2), ld, k, blk(A, 2), ld, k, n3, D + kG, c->part, c->counter, gate, mk, st);
      P_diag(c, D + kG, k, 1, D + kC3, c->st, mk, st);
      P_combine<T>(c, blk(A, 2), ld, k, nullptr, D + kC3, k, nullptr, 0, 0.0, 1.0, blk(A, 2), ld, nullptr, N, gate,
                        mk, st);
      P_combine<T>(c, blk(A, 5), ld, k, nullptr, D + kC3, k, nullptr, 0, 0.0, 1.0, blk(A, 5), ld, nullptr, N, gate,
                        mk, st);
    }
    const int nb = haveP ? 3 : 2;
    const int nS = nb * k;
    for (int jb = 0; jb < nb; ++jb) {
      P_gram<T>(c, A, ld, nS, blk(A, jb), ld, k, n3, Gb + (size_t)jb * nS * k, c->part, c->counter, gate, mk, st);
      P_gram<T>(c, A, ld, nS, blk(A, 3 + jb), ld, k, n3, Mb + (size_t)jb * nS * k, c->part, c->counter, gate, mk,
                     st);
    }
    P_lob_rr(c, Gb, Mb, k, nb, drop, Cx, Cp, lam, c->st, st);
    P_combine<T>(c, A, ld, nS, nullptr, Cx, k, nullptr, 0, 0.0, 1.0, blk(B, 0), ld, nullptr, N, gate, mk, st);
    P_combine<T>(c, blk(A, 3), ld, nS, nullptr, Cx, k, nullptr, 0, 0.0, 1.0, blk(B, 3), ld, nullptr, N, gate, mk,
                      st);
    P_combine<T>(c, A, ld, nS, nullptr, Cp, k, nullptr, 0, 0.0, 1.0, blk(B, 2), ld, nullptr, N, gate, mk, st);
    P_combine<T>(c, blk(A, 3), ld, nS, nullptr, Cp, k, nullptr, 0, 0.0, 1.0, blk(B, 5), ld, nullptr, N, gate, mk,
                      st);
    lob_swap_kernel<<<1, 32, 0, st>>>(c->st, mk);
    haveP = true;
    a = 1 - a;
    if (cap == cudaStreamCaptureStatusNone && it % 10 == 0) {
      DevState h;
      if (cudaMemcpyAsync(&h, c->st, sizeof(h), cudaMemcpyDeviceToHost, st) == cudaSuccess &&
          cudaStreamSynchronize(st) == cudaSuccess && (h.gate & mk))
        break;
    }
  }
  copy_current_kernel<T><<<(unsigned)std::min<size_t>((n3 + 255) / 256, 4096), 256, 0, st>>>(
      blk(SET(0), 0), blk(SET(1), 0), n3, c->st, V, ld, k, ldv);
  P_finish<T>(c, m, V, ldv, k, N, c->part, c->counter, D + kScal, gate, kGateDone, st);
}

}  // namespace

// ----------------------------------------------------------------------------
// Autotuner: the strip HVP comes in bit-identical variants whose speed depends
// on the lattice and the number of vectors per call.  At context creation the
// variants are timed once on the context's own scratch (CUDA events, one
// warm-up launch and three timed launches each, vectors as many as the solver
// passes per call) and the fastest is recorded process-wide for (L1, L2,
// precision, vectors); later contexts of the same lattice reuse the record.
// MOTO_AUTOTUNE=0 in the environment records variant 0 instead.
// ----------------------------------------------------------------------------
template <typename T>
int autotune_hvp(moto_ctx* c) {
  const int nvec = c->p.solver == MOTO_SOLVER_LANCZOS ? c->p.block : c->p.k;
  c->hvp_nvec = nvec;
  const int esz = (int)sizeof(T);
  if (hvp_tuned_variant(c->md.L1, c->md.L2, esz, nvec) >= 0) return MOTO_OK;
  const char* env = getenv("MOTO_AUTOTUNE");
  const int nv = hvp_variant_count();
  if (env && strcmp(env, "0") == 0) {
    hvp_record_variant(c->md.L1, c->md.L2, esz, nvec, 0);
    return MOTO_OK;
  }
  T* V = static_cast<T*>(c->basis);
  T* HV = V + (size_t)nvec * c->ld;
  const T* m = static_cast<const T*>(c->W);
  const T* s = static_cast<const T*>(c->s);
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  int best = 0;
  float best_ms = 0.f;
  for (int v = 0; v < nv && v < 16; ++v) {
    launch_hvp_strip_variant<T>(v, c->md, m, s, V, c->ld, HV, c->ld, nvec, nullptr, 0, 0);
    cudaEventRecord(e0, 0);
    for (int r = 0; r < 3; ++r)
      launch_hvp_strip_variant<T>(v, c->md, m, s, V, c->ld, HV, c->ld, nvec, nullptr, 0, 0);
    cudaEventRecord(e1, 0);
    float ms = 0.f;
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      return cuda_fail(cudaGetLastError(), "autotuner timing", __LINE__);
    }
    c->hvp_ms[v] = ms / 3.f;
    if (v == 0 || c->hvp_ms[v] < best_ms) {
      best = v;
      best_ms = c->hvp_ms[v];
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  hvp_record_variant(c->md.L1, c->md.L2, esz, nvec, best);
  c->hvp_tuned_here = 1;
  return MOTO_OK;
}

// The persistent energy / gradient stencil's variants, timed like the HVP's
// (gradient and s stored, one warm-up and three timed launches each) and
// recorded process-wide for (L1, L2, precision).
template <typename T>
int autotune_stencil(moto_ctx* c) {
  const int esz = (int)sizeof(T);
  if (stencil_tuned_variant(c->md.L1, c->md.L2, esz) >= 0) return MOTO_OK;
  const char* env = getenv("MOTO_AUTOTUNE");
  if (env && strcmp(env, "0") == 0) {
    stencil_record_variant(c->md.L1, c->md.L2, esz, 0);
    return MOTO_OK;
  }
  const T* m = static_cast<const T*>(c->W);
  T* g = static_cast<T*>(c->g);
  T* s = static_cast<T*>(c->s);
  double* out = c->dsm + kTmp;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  int best = 0;
  float best_ms = 0.f;
  for (int v = 0; v < stencil_variant_count() && v < 8; ++v) {
    launch_energy_grad_variant<T>(v, c->md, m, g, s, c->part, c->counter, out, &c->st->status, 0);
    cudaEventRecord(e0, 0);
    for (int r = 0; r < 3; ++r)
      launch_energy_grad_variant<T>(v, c->md, m, g, s, c->part, c->counter, out, &c->st->status, 0);
    cudaEventRecord(e1, 0);
    float ms = 0.f;
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      return cuda_fail(cudaGetLastError(), "autotuner timing", __LINE__);
    }
    c->stencil_ms[v] = ms / 3.f;
    if (v == 0 || c->stencil_ms[v] < best_ms) {
      best = v;
      best_ms = c->stencil_ms[v];
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  stencil_record_variant(c->md.L1, c->md.L2, esz, best);
  c->stencil_tuned_here = 1;
  return MOTO_OK;
}

// ----------------------------------------------------------------------------
// Context creation.  nw == 0: one walker, every scratch area its own
// allocation, sized for any parameters the solvers accept.  nw >= 1: a walker
// group, its scratch sized for `params` (basis block * steps fields, LOBPCG
// sets only for LOBPCG) plus slots for each walker's spins, modes and descent
// copies, in nw slices of one allocation (slice stride a multiple of 256 B).
// ----------------------------------------------------------------------------
int create_ctx(const moto_model* model, int dtype, const moto_params* params, int nw, moto_ctx** out) {
  if (!model || !out || !params || nw < 0) return MOTO_ERR_ARG;
  *out = nullptr;
  if (model->L1 < 5 || model->L2 < 5) return MOTO_ERR_ARG;
  if (model->n_shells < 1 || model->n_shells > 3) return MOTO_ERR_ARG;
  if (dtype != MOTO_F32 && dtype != MOTO_F64) return MOTO_ERR_ARG;
  if ((long long)model->L1 * model->L2 > (1LL << 30)) return MOTO_ERR_ARG;
  int rc = check_params(params);
  if (rc) return rc;
  moto_ctx* c = new moto_ctx();
  memset(c, 0, sizeof(*c));
  c->prof_cond_cur = -1;
  c->md.L1 = model->L1;
  c->md.L2 = model->L2;
  c->md.N = model->L1 * model->L2;
  c->md.n_shells = model->n_shells;
  for (int i = 0; i < 3; ++i) c->md.J[i] = i < model->n_shells ? model->J[i] : 0.0;
  c->md.D = model->D;
  c->md.K = model->K;
  c->md.muB = model->muB;
  c->dtype = dtype;
  c->esize = dtype == MOTO_F64 ? 8 : 4;
  c->p = *params;
  c->N = c->md.N;
  c->n3 = 3 * (size_t)c->N;
  c->ld = (c->n3 + 63) / 64 * 64;
  c->nw = nw > 0 ? nw : 1;
  const size_t vb = c->ld * c->esize;
  const int R = MOTO_MAX_MEM + 1;
  size_t tb = (size_t)tile_blocks(c->md);
  size_t part = std::max<size_t>(2 * tb, (size_t)kStreamBlocks * MOTO_MAX_BASIS * MOTO_MAX_K);
  part = std::max<size_t>(part, (size_t)kSMs * 8 * MOTO_MAX_K * 4);
  part = std::max<size_t>(part, (size_t)kStreamBlocks * 9 * MOTO_MAX_K * MOTO_MAX_K * 2);
  part = std::max<size_t>(part, 2 * (size_t)pair_blocks(c->md));
  c->part_len = part;
  const bool group = nw > 0;
  const int nbasis = group ? std::max(16, params->block * params->krylov_steps) : MOTO_MAX_BASIS;
  const size_t nlob = (!group || params->solver == MOTO_SOLVER_LOBPCG) ? 12 * MOTO_MAX_K : 0;
  const int nv = std::max(params->k, params->block);
  struct A {
    void** p;
    size_t n;
  } allocs[] = {
      {&c->basis, vb * nbasis},
      {&c->W, vb * MOTO_MAX_K},
      {&c->Wt, vb * MOTO_MAX_K},
      {&c->g, vb},
      {&c->s, c->ld * c->esize},
      {&c->ring, vb * (2 * R + 5)},
      {&c->lob, vb * nlob},  // two sets of [X, W, P, AX, AW, AP]
      {(void**)&c->dsm, kDsmSize * sizeof(double)},
      {(void**)&c->pairs, (size_t)MOTO_MAX_PAIRS * 6 * sizeof(double)},
      {(void**)&c->part, part * sizeof(double)},
      {(void**)&c->counter, 64 * sizeof(unsigned)},
      {(void**)&c->st, sizeof(DevState)},
      {&c->mslot, group ? vb : 0},
      {&c->Vslot, group ? vb * nv : 0},
      {&c->mpslot, group ? vb : 0},
      {&c->mmslot, group ? vb : 0},
  };
  if (!group) {
    for (auto& a : allocs) {
      if (a.n == 0) continue;
      if (cudaMalloc(a.p, a.n) != cudaSuccess) {
        moto_destroy(c);
        return MOTO_ERR_NOMEM;
      }
      c->bytes += a.n;
      cudaMemset(*a.p, 0, a.n);
    }
  } else {
    size_t off = 0;
    for (auto& a : allocs) off += (a.n + 255) / 256 * 256;
    c->wstride = off;
    if (cudaMalloc(&c->arena, off * (size_t)nw) != cudaSuccess) {
      c->arena = nullptr;
      moto_destroy(c);
      return MOTO_ERR_NOMEM;
    }
    off = 0;
    for (auto& a : allocs) {
      *a.p = a.n ? static_cast<char*>(c->arena) + off : nullptr;
      off += (a.n + 255) / 256 * 256;
    }
    c->bytes = off * (size_t)nw;
  }
  if (cudaDeviceSynchronize() != cudaSuccess) {
    moto_destroy(c);
    return MOTO_ERR_CUDA;
  }
  c->hvp_force = -1;
  c->stencil_force = -1;
  rc = dtype == MOTO_F32 ? autotune_hvp<float>(c) : autotune_hvp<double>(c);
  if (rc == MOTO_OK) rc = dtype == MOTO_F32 ? autotune_stencil<float>(c) : autotune_stencil<double>(c);
  if (rc == MOTO_OK) {
    // the timing launches wrote the scratch: give the solvers zeroed fields again
    if (group)
      cudaMemset(c->arena, 0, c->bytes);
    else
      cudaMemset(c->basis, 0, vb * nbasis);
    if (cudaDeviceSynchronize() != cudaSuccess) rc = MOTO_ERR_CUDA;
  }
  if (rc != MOTO_OK) {
    moto_destroy(c);
    return rc;
  }
  *out = c;
  return MOTO_OK;
}

// The calling thread's walker grid follows a context for a scope: a group of
// several walkers launches every kernel over all of them.
struct WalkerScope {
  WalkerGrid saved;
  explicit WalkerScope(const moto_ctx* c) : saved(walker_grid()) {
    walker_grid() = WalkerGrid{c->nw, c->nw > 1 ? c->wstride : 0};
  }
  ~WalkerScope() { walker_grid() = saved; }
};

// dst <- src (bytes per walker), for every walker of the current grid
cudaError_t copy_walkers(void* dst, const void* src, size_t bytes, cudaStream_t st) {
  const WalkerGrid wg = walker_grid();
  if (wg.nw > 1 && wg.ws)
    return cudaMemcpy2DAsync(dst, wg.ws, src, wg.ws, bytes, (size_t)wg.nw, cudaMemcpyDeviceToDevice, st);
  return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, st);
}

// ============================================================================
// C ABI
// ============================================================================
extern "C" {

void moto_default_params(moto_params* p) {
  if (!p) return;
  p->k = 1;
  p->solver = MOTO_SOLVER_LANCZOS;
  p->block = 1;
  p->krylov_steps = 60;
  p->max_iter = 200;
  p->tol = 1e-6;
  p->lbfgs_mem = 5;
  p->theta_max = 0.2;
  p->gamma0 = 0.02;
  p->tau_F = 1e-3;
  p->eta_theta = 0.1;
  p->max_steps = 300;
  p->descent_max_steps = 5000;
  p->optimizer = MOTO_OPT_LBFGS;
  p->subspace = 0;
  p->descent = MOTO_DESCENT_OPT;
  p->llg_alpha = 1.0;
  p->llg_dt = 0.01;
  p->llg_time = 50.0 / 0.6582119569;  // 50 ps in hbar/meV
  p->reorth = MOTO_REORTH_FULL;
  p->tau_lambda = 0.0;
}

const char* moto_status_string(int code) {
  switch (code) {
    case MOTO_OK: return "ok";
    case MOTO_NOT_CONVERGED: return "not converged (iteration cap reached)";
    case MOTO_ERR_ARG: return "invalid argument";
    case MOTO_ERR_CUDA: return "CUDA runtime error";
    case MOTO_ERR_NUMERIC: return "numerical breakdown (Krylov or small Gram matrix)";
    case MOTO_ERR_NONFINITE: return "non-finite value met on the device";
    case MOTO_ERR_TIMEOUT: return "bounded device wait timed out";
    case MOTO_ERR_NOMEM: return "out of device memory";
    default: return "unknown status";
  }
}

int moto_create(const moto_model* model, int dtype, const moto_params* params, moto_ctx** out) {
  return create_ctx(model, dtype, params, 0, out);
}

void moto_destroy(moto_ctx* c) {
  if (!c) return;
  cudaDeviceSynchronize();
  if (c->step_exec) cudaGraphExecDestroy(c->step_exec);
  if (c->step_stream) cudaStreamDestroy(c->step_stream);
  if (c->arena) {
    cudaFree(c->arena);
  } else {
    void* ptrs[] = {c->basis, c->W, c->Wt, c->g, c->s, c->ring, c->lob, c->dsm, c->pairs, c->part, c->counter, c->st};
    for (void* p : ptrs)
      if (p) cudaFree(p);
  }
  delete c;
}

int moto_set_hvp_variant(moto_ctx* c, int variant) {
  if (!c || variant < -1 || variant >= hvp_variant_count()) return MOTO_ERR_ARG;
  c->hvp_force = variant;
  c->gen += 1;
  return MOTO_OK;
}

int moto_hvp_tuning(const moto_ctx* c, int* variant, float* ms, int cap) {
  if (!c) return MOTO_ERR_ARG;
  const int nv = hvp_variant_count();
  if (variant) {
    const int t = hvp_tuned_variant(c->md.L1, c->md.L2, (int)c->esize, c->hvp_nvec);
    *variant = c->hvp_force >= 0 ? c->hvp_force : (t < 0 ? 0 : t);
  }
  if (ms)
    for (int v = 0; v < cap && v < nv; ++v) ms[v] = c->hvp_tuned_here ? c->hvp_ms[v] : 0.f;
  return nv;
}

int moto_set_stencil_variant(moto_ctx* c, int variant) {
  if (!c || variant < -1 || variant >= stencil_variant_count()) return MOTO_ERR_ARG;
  c->stencil_force = variant;
  c->gen += 1;
  return MOTO_OK;
}

int moto_stencil_tuning(const moto_ctx* c, int* variant, float* ms, int cap) {
  if (!c) return MOTO_ERR_ARG;
  const int nv = stencil_variant_count();
  if (variant) {
    const int t = stencil_tuned_variant(c->md.L1, c->md.L2, (int)c->esize);
    *variant = c->stencil_force >= 0 ? c->stencil_force : (t < 0 ? 0 : t);
  }
  if (ms)
    for (int v = 0; v < cap && v < nv; ++v) ms[v] = c->stencil_tuned_here ? c->stencil_ms[v] : 0.f;
  return nv;
}

int moto_krylov_basis(moto_ctx* c, const void** basis_dev, size_t* ld, int* nvec, int* reorth_steps,
                      void* stream) {
  if (!c) return MOTO_ERR_ARG;
  DevState h;
  CK(cudaMemcpyAsync(&h, c->st, sizeof(h), cudaMemcpyDeviceToHost, S(stream)));
  CK(cudaStreamSynchronize(S(stream)));
  if (basis_dev) *basis_dev = c->basis;
  if (ld) *ld = c->ld;
  if (nvec) *nvec = h.nT;
  if (reorth_steps) *reorth_steps = c->last_selective ? h.pad[4] : std::max(h.steps - 1, 0);
  return MOTO_OK;
}

int moto_set_wait_limit(moto_ctx* c, int polls) {
  if (!c || polls < 0) return MOTO_ERR_ARG;
  c->wait_polls = polls;
  c->gen += 1;
  return MOTO_OK;
}

int moto_set_pairs(moto_ctx* c, const moto_pair* pairs, int n) {
  if (!c || n < 0 || n > MOTO_MAX_PAIRS || (n > 0 && !pairs)) return MOTO_ERR_ARG;
  c->gen += 1;
  int reach = 0;
  std::vector<double> rec((size_t)n * 6);
  for (int p = 0; p < n; ++p) {
    const moto_pair& a = pairs[p];
    if (a.d1 == 0 && a.d2 == 0) return MOTO_ERR_ARG;
    if (std::abs(a.d1) > MOTO_MAX_REACH || std::abs(a.d2) > MOTO_MAX_REACH) return MOTO_ERR_ARG;
    if (!std::isfinite(a.J) || !std::isfinite(a.D[0]) || !std::isfinite(a.D[1]) || !std::isfinite(a.D[2]))
      return MOTO_ERR_ARG;
    reach = std::max(reach, std::max(std::abs(a.d1), std::abs(a.d2)));
    // closure: the reversed pair with the same J and the opposite D
    int partners = 0;
    for (int q = 0; q < n; ++q) {
      const moto_pair& b = pairs[q];
      if (b.d1 == -a.d1 && b.d2 == -a.d2 && b.J == a.J && b.D[0] == -a.D[0] && b.D[1] == -a.D[1] &&
          b.D[2] == -a.D[2])
        ++partners;
    }
    int same = 0;
    for (int q = 0; q < n; ++q)
      if (pairs[q].d1 == a.d1 && pairs[q].d2 == a.d2) ++same;
    if (partners != 1 || same != 1) return MOTO_ERR_ARG;
    double* r = rec.data() + 6 * (size_t)p;
    r[0] = a.d1;
    r[1] = a.d2;
    r[2] = a.J;
    r[3] = a.D[0];
    r[4] = a.D[1];
    r[5] = a.D[2];
  }
  if (n > 0 && (c->md.L1 < 2 * reach + 1 || c->md.L2 < 2 * reach + 1)) return MOTO_ERR_ARG;
  if (n > 0 && cudaMemcpy(c->pairs, rec.data(), rec.size() * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess)
    return MOTO_ERR_CUDA;
  c->md.pairs = n > 0 ? c->pairs : nullptr;
  c->md.npairs = n;
  c->md.reach = reach;
  return MOTO_OK;
}

size_t moto_workspace_bytes(const moto_ctx* c) { return c ? c->bytes : 0; }

int moto_status(moto_ctx* c, void* stream) {
  if (!c) return MOTO_ERR_ARG;
  DevState h;
  CK(cudaMemcpyAsync(&h, c->st, sizeof(h), cudaMemcpyDeviceToHost, S(stream)));
  CK(cudaStreamSynchronize(S(stream)));
  if (h.status & kStatusNonfinite) return MOTO_ERR_NONFINITE;
  if (h.status & kStatusTimeout) return MOTO_ERR_TIMEOUT;
  if (h.status & (kStatusBreakdown | kStatusNotSPD)) return MOTO_ERR_NUMERIC;
  return MOTO_OK;
}

int moto_clear_status(moto_ctx* c, void* stream) {
  if (!c) return MOTO_ERR_ARG;
  state_kernel<<<wgrid(1), 32, 0, S(stream)>>>(c->st, 2, walker_ws());
  CK(cudaGetLastError());
  return MOTO_OK;
}

int moto_energy_grad(moto_ctx* c, const void* m, void* g, void* s, double* out, void* stream) {
  if (!c || !m) return MOTO_ERR_ARG;
  if (c->dtype == MOTO_F32)
    P_energy_grad<float>(c, c->md, (const float*)m, (float*)g, (float*)s, c->part, c->counter, out,
                              &c->st->status, false, S(stream));
  else
    P_energy_grad<double>(c, c->md, (const double*)m, (double*)g, (double*)s, c->part, c->counter, out,
                               &c->st->status, false, S(stream));
  CK(cudaGetLastError());
  return MOTO_OK;
}

int moto_energy(moto_ctx* c, const void* m, double* E, void* stream) {
  if (!c || !m || !E) return MOTO_ERR_ARG;
  double* tmp = c->dsm + kTmp;
  if (c->dtype == MOTO_F32)
    P_energy_grad<float>(c, c->md, (const float*)m, nullptr, nullptr, c->part, c->counter, tmp, &c->st->status,
                              true, S(stream));
  else
    P_energy_grad<double>(c, c->md, (const double*)m, nullptr, nullptr, c->part, c->counter, tmp,
                               &c->st->status, true, S(stream));
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(E, tmp, sizeof(double), cudaMemcpyDeviceToDevice, S(stream)));
  return MOTO_OK;
}

int moto_hvp(moto_ctx* c, const void* m, const void* s, const void* v, size_t ldv, void* hv, size_t ldhv, int nvec,
             void* stream) {
  if (!c || !m || !s || !v || !hv || nvec < 1) return MOTO_ERR_ARG;
  if ((nvec > 1) && (ldv < c->n3 || ldhv < c->n3)) return MOTO_ERR_ARG;
  if (c->dtype == MOTO_F32)
    P_hvp<float>(c, c->md, (const float*)m, (const float*)s, (const float*)v, ldv, (float*)hv, ldhv, nvec,
                      nullptr, 0, S(stream));
  else
    P_hvp<double>(c, c->md, (const double*)m, (const double*)s, (const double*)v, ldv, (double*)hv, ldhv, nvec,
                       nullptr, 0, S(stream));
  CK(cudaGetLastError());
  return MOTO_OK;
}

int moto_energy_euclid_grad(moto_ctx* c, const void* m, void* grad, double* out, void* stream) {
  if (!c || !m || !grad || !out) return MOTO_ERR_ARG;
  cudaStream_t st = S(stream);
  if (c->dtype == MOTO_F32) {
    PROF(kPkStencil, 6.0 * c->N * sizeof(float));
    launch_energy_grad<float>(c->md, (const float*)m, (float*)grad, nullptr, c->part, c->counter, out,
                              &c->st->status, true, st, true);
  } else {
    PROF(kPkStencil, 6.0 * c->N * sizeof(double));
    launch_energy_grad<double>(c->md, (const double*)m, (double*)grad, nullptr, c->part, c->counter, out,
                               &c->st->status, true, st, true);
  }
  CK(cudaGetLastError());
  return MOTO_OK;
}

int moto_euclid_hvp(moto_ctx* c, const void* v, size_t ldv, void* hv, size_t ldhv, int nvec, void* stream) {
  if (!c || !v || !hv || nvec < 1) return MOTO_ERR_ARG;
  if ((nvec > 1) && (ldv < c->n3 || ldhv < c->n3)) return MOTO_ERR_ARG;
  cudaStream_t st = S(stream);
  if (c->dtype == MOTO_F32) {
    PROF(kPkHvp, 6.0 * nvec * c->N * sizeof(float));
    launch_euclid_hvp<float>(c->md, (const float*)v, ldv, (float*)hv, ldhv, nvec, st);
  } else {
    PROF(kPkHvp, 6.0 * nvec * c->N * sizeof(double));
    launch_euclid_hvp<double>(c->md, (const double*)v, ldv, (double*)hv, ldhv, nvec, st);
  }
  CK(cudaGetLastError());
  return MOTO_OK;
}

int moto_topo_charge(moto_ctx* c, const void* m, double* Q, void* stream) {
  if (!c || !m || !Q) return MOTO_ERR_ARG;
  if (c->dtype == MOTO_F32)
    launch_topo<float>(c->md, (const float*)m, c->part, c->counter, Q, S(stream));
  else
    launch_topo<double>(c->md, (const double*)m, c->part, c->counter, Q, S(stream));
  CK(cudaGetLastError());
  return MOTO_OK;
}

}  // extern "C"

// ============================================================================
// inner layer, outer layer
// ============================================================================
namespace {

__global__ void store_iters_kernel(const DevState* st, double* out, size_t ws) {
  st = wofs(st, ws);
  out = wofs(out, ws);
  if (threadIdx.x == 0) out[0] = (double)st->pad[1];
}

template <typename T>
void lowest_modes_impl(moto_ctx* c, const T* m, const T* s, const moto_params* p, const T* v0, size_t ld0, T* V,
                       size_t ldv, int nout, double* lam, cudaStream_t st) {
  if (p->solver == MOTO_SOLVER_LANCZOS) {
    block_lanczos<T>(c, m, s, v0, ld0, p->block, p->krylov_steps, V, ldv, nout, lam, st,
                     p->reorth == MOTO_REORTH_SELECTIVE);
  } else {
    lobpcg<T>(c, m, s, v0, ld0, p->k, p->max_iter, p->tol, V, ldv, lam, st);
  }
}

// One outer step.  ascent: reflected force and min-mode solve; otherwise plain
// descent on g.  update == false evaluates the stopping test only.
// trace_rows > 0: out6 is a trace of that many rows, the step's record goes
// to the row of the steps taken so far (read on the device).
template <typename T>
void opt_step(moto_ctx* c, T* m, const moto_params* p, T* V, double* out6, int* status, bool ascent, bool update,
              cudaStream_t st, int trace_rows = 0) {
  const int N = c->N;
  const size_t ld = c->ld, n3 = c->n3;
  T* g = static_cast<T*>(c->g);
  T* s = static_cast<T*>(c->s);
  const int R = p->lbfgs_mem + 1, nb = 2 * R + 1;
  T* ring = static_cast<T*>(c->ring);
  // ring fields: the 2R pair slots, then G, the staged candidate pair (so
  // that G, s, y are three equally strided fields), G_prev and d
  T* Gcur = ring + (size_t)(2 * R) * ld;
  T* stage = Gcur + ld;
  T* Gprev = stage + 2 * ld;
  T* d = Gprev + ld;
  double* D = c->dsm;
  int* gate = &c->st->gate;
  const int md = kGateDone;
  P_energy_grad<T>(c, c->md, m, g, s, c->part, c->counter, D + kEG, &c->st->status, false, st);
  double* lam = D + kTheta;
  if (ascent) {
    const int nv = std::max(p->k, p->solver == MOTO_SOLVER_LANCZOS ? p->block : p->k);
    lowest_modes_impl<T>(c, m, s, p, V, n3, V, n3, nv, lam, st);
    // G = -F_mmf = g - 2 V (V^T g) over v1 or the k lowest Ritz vectors
    const int nr = p->subspace ? p->k : 1;
    P_gram<T>(c, g, ld, 1, V, n3, nr, n3, D + kMmfDots, c->part, c->counter, gate, md, st);
    P_mmf_force<T>(c, g, V, n3, nr, D + kMmfDots, Gcur, N, c->part, c->counter, D + kFmax, gate, md, st);
  } else {
    P_mmf_force<T>(c, g, nullptr, n3, 0, D + kMmfDots, Gcur, N, c->part, c->counter, D + kFmax, gate, md, st);
  }
  P_saddle_test(c, D + kEG, D + kFmax, lam, D + kMmfDots, p->tau_F, p->tau_lambda, out6, status, c->st,
                ascent ? 1 : 0, update ? 0 : 1, trace_rows, st);
  if (!update) return;
  if (p->optimizer == MOTO_OPT_CG) {
    // nonlinear CG: the pair s = P d_prev, y = G - P G_prev (staging fields),
    // one Gram of [G, s, y], beta and the spectral step, then the
    // direction, the restart test and the capped step; p lives in the last
    // ring field (the pair kernel writes ring slot 0 only while CG runs)
    T* pdir = ring + (size_t)(2 * R - 1) * ld;
    P_lbfgs_pair<T>(c, m, d, Gprev, Gcur, ring, ld, stage, c->st, N, gate, md, st);
    P_gram<T>(c, Gcur, ld, 3, Gcur, ld, 3, n3, D + kCg, c->part, c->counter, gate, md, st);
    P_cg_coeffs(c, D + kCg, p->gamma0, c->st, st);
    P_cg_direction<T>(c, m, Gcur, pdir, N, D + kCg, p->theta_max, c->part, c->counter, c->st, gate, md, st);
    P_cg_retract<T>(c, m, Gcur, pdir, d, c->st, N, gate, md, st);
    copy_walkers(Gprev, Gcur, n3 * sizeof(T), st);
    return;
  }
  P_lbfgs_pair<T>(c, m, d, Gprev, Gcur, ring, ld, stage, c->st, N, gate, md, st);
  P_gram<T>(c, ring, ld, nb, Gcur, ld, 3, n3, D + kLbNew, c->part, c->counter, gate, md, st);
  P_lbfgs_solve(c, D + kLbM, p->lbfgs_mem, D + kLbNew, p->gamma0, D + kLbCoef, c->st, st);
  P_lbfgs_direction<T>(c, ring, ld, nb, D + kLbCoef, m, d, N, p->theta_max, c->part, c->counter, c->st, gate, md,
                            st);
  P_retract<T>(c, m, d, c->st, N, gate, md, st);
  copy_walkers(Gprev, Gcur, n3 * sizeof(T), st);
}

int read_state(moto_ctx* c, DevState* h, cudaStream_t st) {
  if (cudaMemcpyAsync(h, c->st, sizeof(DevState), cudaMemcpyDeviceToHost, st) != cudaSuccess) return MOTO_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return MOTO_ERR_CUDA;
  return MOTO_OK;
}

int status_code(const DevState& h) {
  if (h.status & kStatusNonfinite) return MOTO_ERR_NONFINITE;
  if (h.status & kStatusTimeout) return MOTO_ERR_TIMEOUT;
  if (h.status & (kStatusBreakdown | kStatusNotSPD)) return MOTO_ERR_NUMERIC;
  return MOTO_OK;
}

bool same_params(const moto_params& a, const moto_params& b) {
  return a.k == b.k && a.solver == b.solver && a.block == b.block && a.krylov_steps == b.krylov_steps &&
         a.max_iter == b.max_iter && a.tol == b.tol && a.lbfgs_mem == b.lbfgs_mem && a.theta_max == b.theta_max &&
         a.gamma0 == b.gamma0 && a.tau_F == b.tau_F && a.eta_theta == b.eta_theta && a.max_steps == b.max_steps &&
         a.descent_max_steps == b.descent_max_steps && a.optimizer == b.optimizer && a.subspace == b.subspace &&
         a.descent == b.descent && a.llg_alpha == b.llg_alpha && a.llg_dt == b.llg_dt && a.llg_time == b.llg_time &&
         a.reorth == b.reorth && a.tau_lambda == b.tau_lambda;
}

// Whether the outer step can be replayed as a captured CUDA graph: every
// decision of a descent step and of a block Lanczos ascent step is taken on
// the device (gate bits), while LOBPCG leaves its iteration early from the
// host and the launch profiler records events around each launch.
// MOTO_GRAPHS=0 in the environment launches every step's kernels one by one
// instead.
bool step_graphable(const moto_ctx* c, const moto_params* p, bool ascent) {
  if ((ascent && p->solver != MOTO_SOLVER_LANCZOS) || c->prof_ev) return false;
  const char* env = getenv("MOTO_GRAPHS");
  return !(env && strcmp(env, "0") == 0);
}

// The outer loop of one walker: steps 0 .. max_steps - 1 update, the last
// evaluates the stopping test only; the host reads the state word every
// check_every steps.  Step 0 runs uncaptured (it also sets the kernels'
// one-time attributes); when the step is graphable, the update step is then
// captured once on a private stream and replayed, the records going to the
// trace row of the device's step count.
template <typename T>
int run_opt(moto_ctx* c, T* m, const moto_params* p, T* V, double* trace, int check_every, int max_steps,
            bool ascent, int* steps_out, cudaStream_t st) {
  if (check_every < 1) check_every = 1;
  state_kernel<<<wgrid(1), 32, 0, st>>>(c->st, 1, walker_ws());
  DevState h;
  memset(&h, 0, sizeof(h));
  double* o = trace ? trace : c->dsm + kTmp;
  const int rows = trace ? max_steps + 1 : 0;
  cudaStream_t run = st;
  cudaStream_t cs = nullptr;
  cudaEvent_t ev = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  if (max_steps > 1 && step_graphable(c, p, ascent) && cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) == cudaSuccess) {
    if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) == cudaSuccess && cudaEventRecord(ev, st) == cudaSuccess &&
        cudaStreamWaitEvent(cs, ev, 0) == cudaSuccess)
      run = cs;
  }
  int rc = MOTO_OK;
  for (int t = 0; t <= max_steps; ++t) {
    const bool update = t < max_steps;
    if (update && t == 1 && run == cs) {
      // capture failures fall back to plain launches
      if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
        opt_step<T>(c, m, p, V, o, nullptr, ascent, true, cs, rows);
        const cudaError_t ce = cudaStreamEndCapture(cs, &graph);
        if (ce != cudaSuccess || cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) {
          if (graph) cudaGraphDestroy(graph);
          graph = nullptr;
          exec = nullptr;
        }
      }
      cudaGetLastError();
    }
    if (update && exec) {
      const cudaError_t le = cudaGraphLaunch(exec, cs);
      if (le != cudaSuccess) {
        rc = cuda_fail(le, "cudaGraphLaunch", __LINE__);
        break;
      }
    } else {
      opt_step<T>(c, m, p, V, o, nullptr, ascent, update, run, rows);
      const cudaError_t le = cudaGetLastError();
      if (le != cudaSuccess) {
        rc = cuda_fail(le, "a launch of the outer step", __LINE__);
        break;
      }
    }
    if ((t + 1) % check_every == 0 || t == max_steps) {
      rc = read_state(c, &h, run);
      if (rc) break;
      if (h.converged || status_code(h)) break;
    }
  }
  if (exec) cudaGraphExecDestroy(exec);
  if (graph) cudaGraphDestroy(graph);
  if (cs) {
    if (ev && cudaEventRecord(ev, cs) == cudaSuccess) cudaStreamWaitEvent(st, ev, 0);
    cudaStreamDestroy(cs);
  }
  if (ev) cudaEventDestroy(ev);
  if (rc) return rc;
  if (steps_out) *steps_out = h.pad[1];
  int sc = status_code(h);
  if (sc) return sc;
  return h.converged ? MOTO_OK : MOTO_NOT_CONVERGED;
}

// Damped spin dynamics (two-sided descent with params.descent = LLG): Heun
// steps m -> m_pred (gradient at m) -> m (gradients at m and m_pred) until
// max_i |g_i| <= tau_F or llg_time; the stopping test runs on the device
// after the gradient at m, the host reads it every check_every steps.
template <typename T>
int run_llg(moto_ctx* c, T* m, const moto_params* p, int check_every, int* steps_out, cudaStream_t st) {
  const size_t ld = c->ld;
  const int N = c->N;
  T* g0 = static_cast<T*>(c->g);
  T* ring = static_cast<T*>(c->ring);
  T* mp = ring;  // predictor spins and their gradient: ring fields 0, 1
  T* g1 = ring + ld;
  double* D = c->dsm;
  int* gate = &c->st->gate;
  const long nmax = (long)std::ceil(p->llg_time / p->llg_dt - 1e-9);
  state_kernel<<<wgrid(1), 32, 0, st>>>(c->st, 1, walker_ws());
  DevState h;
  memset(&h, 0, sizeof(h));
  // one Heun step (the last evaluates the stopping test only); like the
  // optimiser's loop, step 0 runs launch by launch and the update step is
  // then captured on a private stream and replayed
  auto heun = [&](bool last, cudaStream_t s) {
    P_energy_grad<T>(c, c->md, m, g0, nullptr, c->part, c->counter, D + kEG, &c->st->status, false, s);
    P_saddle_test(c, D + kEG, D + kFmax, D + kTheta, D + kMmfDots, p->tau_F, p->tau_lambda, D + kTmp, nullptr,
                  c->st, 0, last ? 1 : 0, 0, s);
    if (!last) {
      P_llg_predict<T>(c, m, g0, mp, p->llg_alpha, p->llg_dt, N, gate, kGateDone, s);
      P_energy_grad<T>(c, c->md, mp, g1, nullptr, c->part, c->counter, D + kTmp + 2, &c->st->status, false, s);
      P_llg_correct<T>(c, m, g0, mp, g1, p->llg_alpha, p->llg_dt, N, gate, kGateDone, s);
    }
  };
  cudaStream_t run = st, cs = nullptr;
  cudaEvent_t ev = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  if (nmax > 1 && !c->prof_ev && step_graphable(c, p, false) &&
      cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) == cudaSuccess) {
    if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) == cudaSuccess && cudaEventRecord(ev, st) == cudaSuccess &&
        cudaStreamWaitEvent(cs, ev, 0) == cudaSuccess)
      run = cs;
  }
  int rc = MOTO_OK;
  for (long t = 0; t <= nmax; ++t) {
    const bool last = t == nmax;
    if (!last && t == 1 && run == cs) {
      if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
        heun(false, cs);
        if (cudaStreamEndCapture(cs, &graph) != cudaSuccess || cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) {
          if (graph) cudaGraphDestroy(graph);
          graph = nullptr;
          exec = nullptr;
        }
      }
      cudaGetLastError();  // a failed capture falls back to plain launches
    }
    if (!last && exec) {
      if (cudaGraphLaunch(exec, cs) != cudaSuccess) {
        rc = MOTO_ERR_CUDA;
        break;
      }
    } else {
      heun(last, run);
    }
    if (cudaGetLastError() != cudaSuccess) {
      rc = MOTO_ERR_CUDA;
      break;
    }
    if ((t + 1) % check_every == 0 || last) {
      rc = read_state(c, &h, run);
      if (rc) break;
      if (h.converged || status_code(h)) break;
    }
  }
  if (exec) cudaGraphExecDestroy(exec);
  if (graph) cudaGraphDestroy(graph);
  if (cs) {
    if (ev && cudaEventRecord(ev, cs) == cudaSuccess) cudaStreamWaitEvent(st, ev, 0);
    cudaStreamDestroy(cs);
  }
  if (ev) cudaEventDestroy(ev);
  if (rc) return rc;
  if (steps_out) *steps_out = h.pad[1];
  int sc = status_code(h);
  if (sc) return sc;
  return h.converged ? MOTO_OK : MOTO_NOT_CONVERGED;
}

}  // namespace

extern "C" {

int moto_lowest_modes(moto_ctx* c, const void* m, const void* s, const moto_params* p, const void* v0, void* V,
                      double* lam, int* info, void* stream) {
  if (!c || !m || !p || !v0 || !V || !lam) return MOTO_ERR_ARG;
  int rc = check_params(p);
  if (rc) return rc;
  cudaStream_t st = S(stream);
  state_kernel<<<wgrid(1), 32, 0, st>>>(c->st, 4, walker_ws());
  if (c->dtype == MOTO_F32) {
    const float* sp = (const float*)s;
    if (!sp) {
      P_energy_grad<float>(c, c->md, (const float*)m, (float*)c->g, (float*)c->s, c->part, c->counter,
                                c->dsm + kEG, &c->st->status, false, st);
      sp = (const float*)c->s;
    }
    lowest_modes_impl<float>(c, (const float*)m, sp, p, (const float*)v0, c->n3, (float*)V, c->n3, p->k, lam, st);
  } else {
    const double* sp = (const double*)s;
    if (!sp) {
      P_energy_grad<double>(c, c->md, (const double*)m, (double*)c->g, (double*)c->s, c->part, c->counter,
                                 c->dsm + kEG, &c->st->status, false, st);
      sp = (const double*)c->s;
    }
    lowest_modes_impl<double>(c, (const double*)m, sp, p, (const double*)v0, c->n3, (double*)V, c->n3, p->k, lam,
                              st);
  }
  if (info) info_kernel<<<wgrid(1), 32, 0, st>>>(c->st, info, walker_ws());
  CK(cudaGetLastError());
  return MOTO_OK;
}

int moto_lbfgs_reset(moto_ctx* c, void* stream) {
  if (!c) return MOTO_ERR_ARG;
  state_kernel<<<wgrid(1), 32, 0, S(stream)>>>(c->st, 1, walker_ws());
  CK(cudaGetLastError());
  return MOTO_OK;
}

int moto_mmf_step(moto_ctx* c, void* m, const moto_params* p, void* V, double* out, int* status, void* stream) {
  if (!c || !m || !p || !V) return MOTO_ERR_ARG;
  int rc = check_params(p);
  if (rc) return rc;
  if (p->lbfgs_mem != c->p.lbfgs_mem) return MOTO_ERR_ARG;
  cudaStream_t st = S(stream);
  // the same arguments as the last call: the second such call captures the
  // step once, later ones replay it (the step's decisions are all taken on
  // the device); anything else launches the step kernel by kernel
  const bool same = c->step_seen > 0 && c->step_m == m && c->step_V == V && c->step_out == out &&
                    c->step_status == status && c->step_gen == c->gen && same_params(c->step_p, *p);
  if (!same) {
    if (c->step_exec) cudaGraphExecDestroy(c->step_exec);
    c->step_exec = nullptr;
    c->step_seen = 0;
    c->step_m = m;
    c->step_V = V;
    c->step_out = out;
    c->step_status = status;
    c->step_p = *p;
    c->step_gen = c->gen;
  }
  c->step_seen += 1;
  if (c->step_seen >= 2 && !c->step_exec && step_graphable(c, p, true)) {
    if (!c->step_stream) cudaStreamCreateWithFlags(&c->step_stream, cudaStreamNonBlocking);
    cudaGraph_t graph = nullptr;
    if (c->step_stream && cudaStreamBeginCapture(c->step_stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
      if (c->dtype == MOTO_F32)
        opt_step<float>(c, (float*)m, p, (float*)V, out, status, true, true, c->step_stream);
      else
        opt_step<double>(c, (double*)m, p, (double*)V, out, status, true, true, c->step_stream);
      if (cudaStreamEndCapture(c->step_stream, &graph) != cudaSuccess ||
          cudaGraphInstantiate(&c->step_exec, graph, 0) != cudaSuccess)
        c->step_exec = nullptr;
      if (graph) cudaGraphDestroy(graph);
    }
    cudaGetLastError();  // a failed capture falls back to plain launches
  }
  if (c->step_exec && !c->prof_ev) {
    CK(cudaGraphLaunch(c->step_exec, st));
    return MOTO_OK;
  }
  if (c->dtype == MOTO_F32)
    opt_step<float>(c, (float*)m, p, (float*)V, out, status, true, true, st);
  else
    opt_step<double>(c, (double*)m, p, (double*)V, out, status, true, true, st);
  CK(cudaGetLastError());
  return MOTO_OK;
}

int moto_ascend(moto_ctx* c, void* m, const moto_params* p, void* V, double* trace, int check_every,
                int* steps_out, void* stream) {
  if (!c || !m || !p || !V) return MOTO_ERR_ARG;
  int rc = check_params(p);
  if (rc) return rc;
  if (p->lbfgs_mem != c->p.lbfgs_mem) return MOTO_ERR_ARG;
  if (c->dtype == MOTO_F32)
    return run_opt<float>(c, (float*)m, p, (float*)V, trace, check_every, p->max_steps, true, steps_out, S(stream));
  return run_opt<double>(c, (double*)m, p, (double*)V, trace, check_every, p->max_steps, true, steps_out, S(stream));
}

int moto_descend(moto_ctx* c, const void* m_saddle, const void* v1, const moto_params* p, void* m_plus,
                 void* m_minus, double* out, void* stream) {
  if (!c || !m_saddle || !v1 || !p || !m_plus || !m_minus || !out) return MOTO_ERR_ARG;
  int rc = check_params(p);
  if (rc) return rc;
  if (p->lbfgs_mem != c->p.lbfgs_mem) return MOTO_ERR_ARG;
  cudaStream_t st = S(stream);
  int result = MOTO_OK;
  for (int side = 0; side < 2; ++side) {
    void* mo = side == 0 ? m_plus : m_minus;
    const double sign = side == 0 ? 1.0 : -1.0;
    int steps = 0;
    if (c->dtype == MOTO_F32) {
      launch_descent_seed<float>((const float*)m_saddle, (const float*)v1, p->eta_theta, sign, (float*)mo, c->N,
                                 c->part, c->counter, c->dsm + kTmp, st);
      rc = p->descent == MOTO_DESCENT_LLG
               ? run_llg<float>(c, (float*)mo, p, 25, &steps, st)
               : run_opt<float>(c, (float*)mo, p, nullptr, nullptr, 25, p->descent_max_steps, false, &steps, st);
    } else {
      launch_descent_seed<double>((const double*)m_saddle, (const double*)v1, p->eta_theta, sign, (double*)mo,
                                  c->N, c->part, c->counter, c->dsm + kTmp, st);
      rc = p->descent == MOTO_DESCENT_LLG
               ? run_llg<double>(c, (double*)mo, p, 25, &steps, st)
               : run_opt<double>(c, (double*)mo, p, nullptr, nullptr, 25, p->descent_max_steps, false, &steps, st);
    }
    if (rc < 0) return rc;
    if (rc == MOTO_NOT_CONVERGED) result = MOTO_NOT_CONVERGED;
    int e = moto_energy(c, mo, out + 2 * side, stream);
    if (e) return e;
    e = moto_topo_charge(c, mo, out + 2 * side + 1, stream);
    if (e) return e;
    store_iters_kernel<<<wgrid(1), 32, 0, st>>>(c->st, out + 4 + side, walker_ws());
  }
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(st));
  return result;
}

}  // extern "C"

// ============================================================================
// launch profiler
// ============================================================================
extern "C" {

int moto_profile_begin(moto_ctx* c, int capacity) {
  if (!c || capacity < 1) return MOTO_ERR_ARG;
  if (c->prof_ev) return MOTO_ERR_ARG;
  c->prof_ev = new cudaEvent_t[2 * (size_t)capacity];
  c->prof_kind = new int[capacity];
  c->prof_bytes = new double[capacity];
  c->prof_cond = new int[capacity];
  c->prof_cond_cur = -1;
  for (int i = 0; i < 2 * capacity; ++i) {
    if (cudaEventCreate(&c->prof_ev[i]) != cudaSuccess) {
      for (int j = 0; j < i; ++j) cudaEventDestroy(c->prof_ev[j]);
      delete[] c->prof_ev;
      delete[] c->prof_kind;
      delete[] c->prof_bytes;
      delete[] c->prof_cond;
      c->prof_ev = nullptr;
      return MOTO_ERR_CUDA;
    }
  }
  c->prof_cap = capacity;
  c->prof_n = 0;
  c->prof_on = 1;
  return MOTO_OK;
}

int moto_profile_end(moto_ctx* c, int nkinds, int* launches, double* ms, double* bytes) {
  if (!c || !c->prof_ev) return MOTO_ERR_ARG;
  c->prof_on = 0;
  int rc = MOTO_OK;
  if (c->prof_n > 0 && cudaEventSynchronize(c->prof_ev[2 * c->prof_n - 1]) != cudaSuccess) rc = MOTO_ERR_CUDA;
  for (int k = 0; k < nkinds; ++k) {
    if (launches) launches[k] = 0;
    if (ms) ms[k] = 0.0;
    if (bytes) bytes[k] = 0.0;
  }
  // conditional launches (the full pass of a selective Lanczos step) moved
  // their bytes only if the step took the pass: the device log of the last
  // solve says which did
  double rlog[MOTO_MAX_BASIS];
  bool have_log = false;
  for (int i = 0; i < c->prof_n; ++i)
    if (c->prof_cond[i] >= 0) have_log = true;
  if (rc == MOTO_OK && have_log &&
      cudaMemcpy(rlog, c->dsm + kRlog, sizeof(rlog), cudaMemcpyDeviceToHost) != cudaSuccess)
    rc = MOTO_ERR_CUDA;
  for (int i = 0; rc == MOTO_OK && i < c->prof_n; ++i) {
    if (c->prof_cond[i] >= 0 && c->prof_cond[i] < MOTO_MAX_BASIS && rlog[c->prof_cond[i]] == 0.0)
      c->prof_bytes[i] = 0.0;
    float t = 0.f;
    if (cudaEventElapsedTime(&t, c->prof_ev[2 * i], c->prof_ev[2 * i + 1]) != cudaSuccess) {
      rc = MOTO_ERR_CUDA;
      break;
    }
    const int k = c->prof_kind[i];
    if (k < nkinds) {
      if (launches) launches[k] += 1;
      if (ms) ms[k] += t;
      if (bytes) bytes[k] += c->prof_bytes[i];
    }
  }
  for (int i = 0; i < 2 * c->prof_cap; ++i) cudaEventDestroy(c->prof_ev[i]);
  delete[] c->prof_ev;
  delete[] c->prof_kind;
  delete[] c->prof_bytes;
  delete[] c->prof_cond;
  c->prof_ev = nullptr;
  c->prof_cap = c->prof_n = 0;
  return rc;
}

}  // extern "C"

// ============================================================================
// Explorer front-end
// ============================================================================
extern "C" int moto_perturb(moto_ctx* c, const void* x0, const unsigned char* mask, const void* delta,
                            size_t ld_delta, int count, void* out, size_t ld_out, void* stream) {
  if (!c || !x0 || !delta || !out || count < 0) return MOTO_ERR_ARG;
  if (count == 0) return MOTO_OK;
  if ((count > 1 && (ld_delta < c->n3 || ld_out < c->n3)) || count > 65535) return MOTO_ERR_ARG;
  cudaStream_t st = S(stream);
  if (c->dtype == MOTO_F32)
    launch_perturb<float>((const float*)x0, mask, (const float*)delta, ld_delta, count, (float*)out, ld_out, c->N,
                          st);
  else
    launch_perturb<double>((const double*)x0, mask, (const double*)delta, ld_delta, count, (double*)out, ld_out,
                           c->N, st);
  CK(cudaGetLastError());
  return MOTO_OK;
}

extern "C" int moto_pairwise_l1(moto_ctx* c, const void* X, size_t ldx, int count, double* D, void* stream) {
  if (!c || !X || !D || count < 2 || count > MOTO_MAX_POP || ldx < c->n3) return MOTO_ERR_ARG;
  cudaStream_t st = S(stream);
  bool ok;
  if (c->dtype == MOTO_F32)
    ok = launch_pairwise_l1<float>((const float*)X, ldx, count, c->n3, c->part, c->part_len, c->counter, D, st);
  else
    ok = launch_pairwise_l1<double>((const double*)X, ldx, count, c->n3, c->part, c->part_len, c->counter, D, st);
  if (!ok) return MOTO_ERR_ARG;
  CK(cudaGetLastError());
  return MOTO_OK;
}

// ============================================================================
// Gram utility
// ============================================================================
extern "C" int moto_gram(moto_ctx* c, const void* X, size_t ldx, int nx, const void* Y, size_t ldy, int ny,
                         double* out, void* stream) {
  if (!c || !X || !Y || !out || nx < 1 || nx > MOTO_MAX_BASIS || ny < 1 || ny > MOTO_MAX_K) return MOTO_ERR_ARG;
  if ((nx > 1 && ldx < c->n3) || (ny > 1 && ldy < c->n3)) return MOTO_ERR_ARG;
  cudaStream_t st = S(stream);
  if (c->dtype == MOTO_F32)
    P_gram<float>(c, (const float*)X, ldx, nx, (const float*)Y, ldy, ny, c->n3, out, c->part, c->counter, nullptr,
                  0, st);
  else
    P_gram<double>(c, (const double*)X, ldx, nx, (const double*)Y, ldy, ny, c->n3, out, c->part, c->counter,
                   nullptr, 0, st);
  CK(cudaGetLastError());
  return MOTO_OK;
}

// ============================================================================
// Batched walkers.  The walkers are grouped by lattice size; a group is one
// context whose scratch, spins and modes lie in equally sized slices of one
// allocation (create_ctx with nw walkers), and every kernel of its outer step
// runs once for all of its walkers (the walker is blockIdx.z, see
// WalkerScope).  Walkers whose step met its stopping test set their done gate
// on the device; their blocks of later launches return at once, so the
// captured step never changes.  One outer step of every group is captured
// into a CUDA graph, the groups fanned out over n_streams streams, and the
// graph is replayed until every walker has stopped; every check_every replays
// one packed copy of all walkers' [converged, status, steps] words reaches the
// host.  Parameters whose kernels have no walker dimension (LOBPCG, nonlinear
// CG) run every walker as a group of one.
// ============================================================================
namespace {

__global__ void batch_flags_kernel(DevState* const* sts, int n, int* flags) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const DevState* s = sts[i];
    flags[3 * i] = s->converged;
    flags[3 * i + 1] = s->status;
    flags[3 * i + 2] = s->pad[1];
  }
}

__global__ void batch_reset_kernel(DevState* const* sts, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    DevState* st = sts[i];
    st->gate = 0;
    st->pad[1] = 0;
    st->lb_head = 0;
    st->lb_count = 0;
    st->lb_have_prev = 0;
    st->converged = 0;
    st->iters = 0;
  }
}

int status_of(int flags_status) {
  DevState h;
  memset(&h, 0, sizeof(h));
  h.status = flags_status;
  return status_code(h);
}

bool batchable(const moto_params& p) {
  return p.solver == MOTO_SOLVER_LANCZOS && p.optimizer == MOTO_OPT_LBFGS && p.descent == MOTO_DESCENT_OPT;
}

}  // namespace

struct BatchGroup {
  moto_ctx* c = nullptr;  // nw walkers in slices of one allocation
  std::vector<int> idx;   // the batch's walker index of each slice
  int stream = 0;
};

struct moto_batch {
  int n = 0, dtype = 0, nstreams = 1;
  moto_params p;
  std::vector<BatchGroup> groups;
  std::vector<moto_walker> w;  // the caller's walkers
  DevState** sts_dev = nullptr;  // device array of the walkers' state words
  int* flags_dev = nullptr;
  int* flags_host = nullptr;  // pinned
  cudaStream_t master = nullptr;
  cudaStream_t* streams = nullptr;
  cudaEvent_t fork = nullptr;
  cudaEvent_t* join = nullptr;
};

namespace {

enum BatchSlot { kSlotM = 0, kSlotMP = 1, kSlotMM = 2 };

void* slot_of(const moto_ctx* c, int slot) {
  return slot == kSlotM ? c->mslot : (slot == kSlotMP ? c->mpslot : c->mmslot);
}
// address of a walker's copy of a slice pointer
template <typename P>
P* at_walker(const moto_ctx* c, P* p, int z) {
  return reinterpret_cast<P*>(reinterpret_cast<char*>(p) + (size_t)z * c->wstride);
}

void batch_free(moto_batch* b) {
  if (!b) return;
  for (auto& g : b->groups) moto_destroy(g.c);
  if (b->streams)
    for (int k = 0; k < b->nstreams; ++k)
      if (b->streams[k]) cudaStreamDestroy(b->streams[k]);
  if (b->join)
    for (int k = 0; k < b->nstreams; ++k)
      if (b->join[k]) cudaEventDestroy(b->join[k]);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->master) cudaStreamDestroy(b->master);
  if (b->sts_dev) cudaFree(b->sts_dev);
  if (b->flags_dev) cudaFree(b->flags_dev);
  if (b->flags_host) cudaFreeHost(b->flags_host);
  delete[] b->streams;
  delete[] b->join;
  delete b;
}

// Records one outer step of every group (group g on stream g % nstreams) and
// the flag gather, forked from and joined into the master stream.  The spins
// stepped are the groups' slot `slot` (ascent: the walkers' spins; descent:
// the copies of one side); records go to each walker's dsm + kTmp.
template <typename T>
int batch_record_step(moto_batch* b, bool ascent, int slot, bool update) {
  CK(cudaEventRecord(b->fork, b->master));
  for (int k = 0; k < b->nstreams; ++k) CK(cudaStreamWaitEvent(b->streams[k], b->fork, 0));
  for (auto& g : b->groups) {
    WalkerScope scope(g.c);
    opt_step<T>(g.c, static_cast<T*>(slot_of(g.c, slot)), &b->p, ascent ? static_cast<T*>(g.c->Vslot) : nullptr,
                g.c->dsm + kTmp, nullptr, ascent, update, b->streams[g.stream]);
  }
  for (int k = 0; k < b->nstreams; ++k) {
    CK(cudaEventRecord(b->join[k], b->streams[k]));
    CK(cudaStreamWaitEvent(b->master, b->join[k], 0));
  }
  batch_flags_kernel<<<(b->n + 127) / 128, 128, 0, b->master>>>(b->sts_dev, b->n, b->flags_dev);
  CK(cudaGetLastError());
  return MOTO_OK;
}

// Runs the captured step until every walker stopped or max_steps replays;
// then one evaluation of the stopping test at the final iterate of the
// walkers still running (as the one-walker loop does).
template <typename T>
int batch_run(moto_batch* b, bool ascent, int slot, int max_steps, int check_every, int* status_host,
              int* steps_host) {
  if (check_every < 1) check_every = 1;
  batch_reset_kernel<<<(b->n + 127) / 128, 128, 0, b->master>>>(b->sts_dev, b->n);
  CK(cudaGetLastError());
  int done = (max_steps == 0);
  int t = 0;
  if (!done) {
    // first step uncaptured: it also sets the kernels' one-time attributes
    int rc = batch_record_step<T>(b, ascent, slot, true);
    if (rc) return rc;
    t = 1;
  }
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  if (!done && t < max_steps) {
    CK(cudaStreamBeginCapture(b->master, cudaStreamCaptureModeThreadLocal));
    int rc = batch_record_step<T>(b, ascent, slot, true);
    cudaError_t ce = cudaStreamEndCapture(b->master, &graph);
    if (rc || ce != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      return rc ? rc : cuda_fail(ce, "cudaStreamEndCapture", __LINE__);
    }
    ce = cudaGraphInstantiate(&exec, graph, 0);
    if (ce != cudaSuccess) {
      cudaGraphDestroy(graph);
      return cuda_fail(ce, "cudaGraphInstantiate", __LINE__);
    }
  }
  int rc = MOTO_OK;
  while (!done) {
    if (t % check_every == 0 || t >= max_steps) {
      if (cudaMemcpyAsync(b->flags_host, b->flags_dev, 3 * sizeof(int) * b->n, cudaMemcpyDeviceToHost, b->master) !=
              cudaSuccess ||
          cudaStreamSynchronize(b->master) != cudaSuccess) {
        rc = MOTO_ERR_CUDA;
        break;
      }
      bool all = true;
      for (int i = 0; i < b->n; ++i)
        if (!b->flags_host[3 * i] && !status_of(b->flags_host[3 * i + 1])) all = false;
      if (all || t >= max_steps) break;
    }
    const cudaError_t le = cudaGraphLaunch(exec, b->master);
    if (le != cudaSuccess) {
      rc = cuda_fail(le, "cudaGraphLaunch", __LINE__);
      break;
    }
    ++t;
  }
  if (exec) cudaGraphExecDestroy(exec);
  if (graph) cudaGraphDestroy(graph);
  if (rc) return rc;
  // stopping test at the final iterate (no update) for walkers still running
  rc = batch_record_step<T>(b, ascent, slot, false);
  if (rc) return rc;
  CK(cudaMemcpyAsync(b->flags_host, b->flags_dev, 3 * sizeof(int) * b->n, cudaMemcpyDeviceToHost, b->master));
  CK(cudaStreamSynchronize(b->master));
  int result = MOTO_OK;
  for (int i = 0; i < b->n; ++i) {
    const int sc = status_of(b->flags_host[3 * i + 1]);
    const int code = sc ? sc : (b->flags_host[3 * i] ? MOTO_OK : MOTO_NOT_CONVERGED);
    if (status_host) status_host[i] = code;
    if (steps_host) steps_host[i] = b->flags_host[3 * i + 2];
    if (code < 0 && result >= 0) result = code;
    if (code == MOTO_NOT_CONVERGED && result == MOTO_OK) result = MOTO_NOT_CONVERGED;
  }
  return result;
}

// caller's spins and modes into the slices, or back out
int batch_copy_walkers(moto_batch* b, bool in) {
  for (auto& g : b->groups) {
    const size_t fb = g.c->n3 * g.c->esize;
    const size_t vbytes = fb * (size_t)std::max(b->p.k, b->p.block);
    for (size_t z = 0; z < g.idx.size(); ++z) {
      const moto_walker& w = b->w[g.idx[z]];
      void* ms = at_walker(g.c, g.c->mslot, (int)z);
      void* vs = at_walker(g.c, g.c->Vslot, (int)z);
      if (in) {
        CK(cudaMemcpyAsync(ms, w.m_dev, fb, cudaMemcpyDeviceToDevice, b->master));
        CK(cudaMemcpyAsync(vs, w.V_dev, vbytes, cudaMemcpyDeviceToDevice, b->master));
      } else {
        CK(cudaMemcpyAsync(w.m_dev, ms, fb, cudaMemcpyDeviceToDevice, b->master));
        CK(cudaMemcpyAsync(w.V_dev, vs, vbytes, cudaMemcpyDeviceToDevice, b->master));
      }
    }
  }
  return MOTO_OK;
}

}  // namespace

extern "C" {

int moto_batch_create(const moto_model* model, int dtype, const moto_params* params, const moto_walker* walkers,
                      int n_walkers, int n_streams, moto_batch** out) {
  if (!model || !params || !walkers || !out || n_walkers < 1 || n_streams < 1) return MOTO_ERR_ARG;
  if (params->descent != MOTO_DESCENT_OPT) return MOTO_ERR_ARG;  // batches descend with the optimiser
  for (int i = 0; i < n_walkers; ++i)
    if (!walkers[i].m_dev || !walkers[i].V_dev) return MOTO_ERR_ARG;
  *out = nullptr;
  moto_batch* b = new moto_batch();
  b->n = n_walkers;
  b->dtype = dtype;
  b->p = *params;
  b->w.assign(walkers, walkers + n_walkers);
  // groups: walkers of equal lattices together (in the order they come)
  const bool together = batchable(*params);
  std::vector<std::pair<std::pair<int, int>, std::vector<int>>> sets;
  for (int i = 0; i < n_walkers; ++i) {
    const std::pair<int, int> key(walkers[i].L1, walkers[i].L2);
    bool placed = false;
    if (together)
      for (auto& e : sets)
        if (e.first == key) {
          e.second.push_back(i);
          placed = true;
          break;
        }
    if (!placed) sets.push_back({key, std::vector<int>{i}});
  }
  b->nstreams = std::max(1, std::min(n_streams, (int)sets.size()));
  b->streams = new cudaStream_t[b->nstreams]();
  b->join = new cudaEvent_t[b->nstreams]();
  std::vector<DevState*> sts(n_walkers, nullptr);
  int rc = MOTO_OK;
  for (size_t gi = 0; gi < sets.size() && !rc; ++gi) {
    moto_model mw = *model;
    mw.L1 = sets[gi].first.first;
    mw.L2 = sets[gi].first.second;
    BatchGroup g;
    g.idx = sets[gi].second;
    g.stream = (int)(gi % b->nstreams);
    rc = create_ctx(&mw, dtype, params, (int)g.idx.size(), &g.c);
    if (!rc) {
      for (size_t z = 0; z < g.idx.size(); ++z) sts[g.idx[z]] = at_walker(g.c, g.c->st, (int)z);
      b->groups.push_back(std::move(g));
    }
  }
  if (!rc) {
    bool ok = cudaStreamCreateWithFlags(&b->master, cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) == cudaSuccess;
    for (int k = 0; ok && k < b->nstreams; ++k)
      ok = cudaStreamCreateWithFlags(&b->streams[k], cudaStreamNonBlocking) == cudaSuccess &&
           cudaEventCreateWithFlags(&b->join[k], cudaEventDisableTiming) == cudaSuccess;
    ok = ok && cudaMalloc(&b->sts_dev, sizeof(DevState*) * n_walkers) == cudaSuccess &&
         cudaMalloc(&b->flags_dev, 3 * sizeof(int) * n_walkers) == cudaSuccess &&
         cudaMallocHost(&b->flags_host, 3 * sizeof(int) * n_walkers) == cudaSuccess &&
         cudaMemcpy(b->sts_dev, sts.data(), sizeof(DevState*) * n_walkers, cudaMemcpyHostToDevice) == cudaSuccess;
    if (!ok) rc = MOTO_ERR_NOMEM;
  }
  if (rc) {
    batch_free(b);
    return rc;
  }
  *out = b;
  return MOTO_OK;
}

void moto_batch_destroy(moto_batch* b) {
  if (!b) return;
  cudaDeviceSynchronize();
  batch_free(b);
}

int moto_batch_ascend(moto_batch* b, int check_every, double* rec_dev, int* status_host, int* steps_host,
                      void* stream) {
  if (!b || !rec_dev) return MOTO_ERR_ARG;
  CK(cudaStreamSynchronize(S(stream)));
  int rc = batch_copy_walkers(b, true);
  if (rc) return rc;
  const int result = b->dtype == MOTO_F32
                         ? batch_run<float>(b, true, kSlotM, b->p.max_steps, check_every, status_host, steps_host)
                         : batch_run<double>(b, true, kSlotM, b->p.max_steps, check_every, status_host, steps_host);
  if (result < 0) return result;
  // records of the last test, and the walkers back to the caller
  for (auto& g : b->groups)
    for (size_t z = 0; z < g.idx.size(); ++z)
      CK(cudaMemcpyAsync(rec_dev + 6 * (size_t)g.idx[z], at_walker(g.c, g.c->dsm, (int)z) + kTmp,
                         6 * sizeof(double), cudaMemcpyDeviceToDevice, b->master));
  rc = batch_copy_walkers(b, false);
  if (rc) return rc;
  CK(cudaStreamSynchronize(b->master));
  return result;
}

int moto_batch_descend(moto_batch* b, void* const* m_plus, void* const* m_minus, double* out_dev, int* status_host,
                       void* stream) {
  if (!b || !m_plus || !m_minus || !out_dev) return MOTO_ERR_ARG;
  for (int i = 0; i < b->n; ++i)
    if (!m_plus[i] || !m_minus[i]) return MOTO_ERR_ARG;
  CK(cudaStreamSynchronize(S(stream)));
  // the walkers' spins and first modes are the saddles and their v1
  int rc = batch_copy_walkers(b, true);
  if (rc) return rc;
  int result = MOTO_OK;
  std::vector<int> st_side(b->n);
  for (int side = 0; side < 2 && result >= 0; ++side) {
    const double sign = side == 0 ? 1.0 : -1.0;
    const int slot = side == 0 ? kSlotMP : kSlotMM;
    for (auto& g : b->groups) {
      WalkerScope scope(g.c);
      moto_ctx* c = g.c;
      if (b->dtype == MOTO_F32)
        launch_descent_seed<float>((const float*)c->mslot, (const float*)c->Vslot, b->p.eta_theta, sign,
                                   (float*)slot_of(c, slot), c->N, c->part, c->counter, c->dsm + kTmp, b->master);
      else
        launch_descent_seed<double>((const double*)c->mslot, (const double*)c->Vslot, b->p.eta_theta, sign,
                                    (double*)slot_of(c, slot), c->N, c->part, c->counter, c->dsm + kTmp,
                                    b->master);
    }
    CK(cudaGetLastError());
    rc = b->dtype == MOTO_F32 ? batch_run<float>(b, false, slot, b->p.descent_max_steps, 25, st_side.data(), nullptr)
                              : batch_run<double>(b, false, slot, b->p.descent_max_steps, 25, st_side.data(), nullptr);
    if (rc < 0) {
      result = rc;
      break;
    }
    // FP64-arithmetic energy, charge and steps of each minimum (a walker's
    // dsm + kBout: [E+, Q+, E-, Q-, steps+, steps-])
    for (auto& g : b->groups) {
      WalkerScope scope(g.c);
      moto_ctx* c = g.c;
      double* o = c->dsm + kBout;
      if (b->dtype == MOTO_F32) {
        launch_energy_grad<float>(c->md, (const float*)slot_of(c, slot), nullptr, nullptr, c->part, c->counter,
                                  o + 2 * side, &c->st->status, true, b->master);
        launch_topo<float>(c->md, (const float*)slot_of(c, slot), c->part, c->counter, o + 2 * side + 1, b->master);
      } else {
        launch_energy_grad<double>(c->md, (const double*)slot_of(c, slot), nullptr, nullptr, c->part, c->counter,
                                   o + 2 * side, &c->st->status, true, b->master);
        launch_topo<double>(c->md, (const double*)slot_of(c, slot), c->part, c->counter, o + 2 * side + 1,
                            b->master);
      }
      store_iters_kernel<<<wgrid(1), 32, 0, b->master>>>(c->st, o + 4 + side, walker_ws());
    }
    CK(cudaGetLastError());
    for (int i = 0; i < b->n; ++i) {
      if (status_host) {
        const int prev = side == 0 ? MOTO_OK : status_host[i];
        int code = st_side[i];
        if (prev < 0 || (prev == MOTO_NOT_CONVERGED && code == MOTO_OK)) code = prev;
        status_host[i] = code;
      }
    }
    if (rc == MOTO_NOT_CONVERGED && result == MOTO_OK) result = MOTO_NOT_CONVERGED;
  }
  if (result >= 0) {
    for (auto& g : b->groups) {
      const size_t fb = g.c->n3 * g.c->esize;
      for (size_t z = 0; z < g.idx.size(); ++z) {
        const int i = g.idx[z];
        CK(cudaMemcpyAsync(out_dev + 6 * (size_t)i, at_walker(g.c, g.c->dsm, (int)z) + kBout, 6 * sizeof(double),
                           cudaMemcpyDeviceToDevice, b->master));
        CK(cudaMemcpyAsync(m_plus[i], at_walker(g.c, g.c->mpslot, (int)z), fb, cudaMemcpyDeviceToDevice, b->master));
        CK(cudaMemcpyAsync(m_minus[i], at_walker(g.c, g.c->mmslot, (int)z), fb, cudaMemcpyDeviceToDevice,
                           b->master));
      }
    }
  }
  if (cudaStreamSynchronize(b->master) != cudaSuccess) return MOTO_ERR_CUDA;
  return result;
}

}  // extern "C"
