/*
 * moto.h -- C ABI of the GB300 (sm_103a) minimum-mode kernel for atomistic
 * spin systems on a periodic 2D triangular lattice (arXiv 2509.26269, "MOTO":
 * bilayer minimum-mode following with HVP-driven Krylov eigensolvers).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Layout.  A spin field or a tangent vector field is a contiguous device array
 *   of 3*N elements, N = L1*L2, component-major (structure of arrays):
 *   x[c*N + i2*L1 + i1] is component c (0 = x, 1 = y, 2 = z) of site (i1, i2),
 *   the site at i1*a1 + i2*a2 with a1 = (1, 0), a2 = (1/2, sqrt(3)/2).  The
 *   element type is float (MOTO_F32) or double (MOTO_F64), fixed when the
 *   context is created.  Scalars produced on the device (energies, eigenvalues,
 *   forces) are always double.  Base addresses must be 16-byte aligned.
 * Ownership.  Every pointer argument is caller-owned memory; the library never
 *   frees or retains it past the call's stream work.  "dev" pointers are device
 *   memory, all others host memory.  The context owns its scratch (Krylov
 *   basis, L-BFGS history, reduction partials), sized once in moto_create; no
 *   other call allocates device memory.
 * Streams.  Calls enqueue work on the given stream (a cudaStream_t passed as
 *   void*; NULL = legacy default stream) and return without synchronising,
 *   except where stated (moto_ascend, moto_descend read a status word back).
 *   A context is not thread-safe and must not be used on two streams at once.
 * Errors.  Every call returns an int: MOTO_OK (0), a positive informational
 *   code, or a negative error.  Argument errors are detected on the host before
 *   any launch.  Errors detected on the device (non-finite values, a Krylov
 *   breakdown, a timeout of a bounded wait) are written to the context's
 *   device status word and returned by moto_status(); they never trap.
 *   MOTO_ERR_CUDA names no cause; with the environment variable MOTO_DEBUG
 *   set, the failing CUDA call and its error string are printed to stderr.
 * Units.  Energies and model parameters in meV, forces (torques) in meV/rad,
 *   eigenvalues in meV (per rad^2), angles in rad.
 */
#ifndef MOTO_H
#define MOTO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct moto_ctx moto_ctx;

enum {
  MOTO_F32 = 0,
  MOTO_F64 = 1
};

enum {
  MOTO_OK = 0,
  MOTO_NOT_CONVERGED = 1,   /* an iteration hit its cap; results are the last iterate */
  MOTO_ERR_ARG = -1,        /* invalid argument (checked on the host) */
  MOTO_ERR_CUDA = -2,       /* a CUDA runtime call failed */
  MOTO_ERR_NUMERIC = -3,    /* Krylov breakdown or a non-SPD small Gram matrix */
  MOTO_ERR_NONFINITE = -4,  /* NaN/Inf met on the device */
  MOTO_ERR_TIMEOUT = -5,    /* a bounded device-side wait gave up */
  MOTO_ERR_NOMEM = -6       /* moto_create could not allocate its scratch */
};

enum {
  MOTO_SOLVER_LANCZOS = 0,  /* block Lanczos, block size params.block (1 = Lanczos) */
  MOTO_SOLVER_LOBPCG = 1
};

/* Relaxation of the two-sided descent (Supplementary Note 1 (iii): "a
 * deterministic optimizer (e.g., L-BFGS/CG) or dynamic simulator"). */
enum {
  MOTO_DESCENT_OPT = 0,  /* the outer optimiser (params.optimizer) on g */
  MOTO_DESCENT_LLG = 1   /* damped spin dynamics (Landau-Lifshitz-Gilbert, Heun) */
};

/* Reorthogonalisation of block Lanczos.  FULL: every new block is
 * orthogonalised against the whole basis (the three-term local pass, then one
 * pass against every block).  SELECTIVE: the local pass only, while a block
 * form of Simon's estimate of the loss of orthogonality (the omega
 * recurrence; Simon 1984) stays below sqrt(eps) of the field precision; when
 * it crosses, the new block and the next one get the full pass (partial
 * reorthogonalisation: the basis stays semi-orthogonal, which keeps the Ritz
 * values as accurate as with full reorthogonalisation). */
enum {
  MOTO_REORTH_FULL = 0,
  MOTO_REORTH_SELECTIVE = 1
};

/* Outer-layer optimiser (Results, "Bilayer MMF": "LBFGS or CG"). */
enum {
  MOTO_OPT_LBFGS = 0,  /* tangent-space L-BFGS two-loop, step cap theta_max, no line search */
  MOTO_OPT_CG = 1      /* nonlinear CG, Polak-Ribiere+ with restarts, spectral step
                          s.y / y.y of the last step (gamma0 without one), step cap */
};

#define MOTO_MAX_K 8        /* modes per solve */
#define MOTO_MAX_BASIS 96   /* Krylov basis vectors (block * steps) */
#define MOTO_MAX_MEM 8      /* L-BFGS pairs */
#define MOTO_MAX_POP 64     /* candidates of one pairwise-distance call */
#define MOTO_MAX_PAIRS 512  /* ordered pairs of a pair-list Hamiltonian */
#define MOTO_MAX_REACH 12   /* largest |d1|, |d2| of a pair offset */

/* Spin Hamiltonian of Eq. param-hamiltonian (Methods, "Spin Hamiltonian and
 * manifold gradient"), read with ordered-pair sums (each bond counted twice):
 *   E = - sum_i sum_s J[s] sum_{d in shell s} m_i . m_{i+d}
 *       - D sum_i sum_{d in shell 1} (z x d_hat) . (m_i x m_{i+d})
 *       - muB sum_i m_iz - K sum_i m_iz^2
 * Shells (index-space offsets): 1: +-(1,0), +-(0,1), +-(-1,1);
 * 2: +-(1,1), +-(-1,2), +-(-2,1); 3: +-(2,0), +-(0,2), +-(-2,2). */
typedef struct {
  int L1, L2;        /* lattice sides, each >= 5 */
  int n_shells;      /* 1..3 exchange shells */
  double J[3];       /* exchange per shell, meV */
  double D;          /* Neel DMI on shell 1, meV */
  double K;          /* uniaxial anisotropy along z, meV */
  double muB;        /* Zeeman energy mu*B along +z, meV */
} moto_model;

/* Parameters of the inner (eigensolver) and outer (ascent, descent) layers.
 * moto_default_params fills the values used throughout the tests. */
typedef struct {
  int k;              /* eigenpairs wanted, 1..MOTO_MAX_K                       (1) */
  int solver;         /* MOTO_SOLVER_*                                         (LANCZOS) */
  int block;          /* block size of block Lanczos, k..MOTO_MAX_K            (1) */
  int krylov_steps;   /* Lanczos steps (block steps); block*steps <= MAX_BASIS (60) */
  int max_iter;       /* LOBPCG iteration cap                                  (200) */
  double tol;         /* LOBPCG: stop when all |H x - theta x| <= tol*|theta|max (1e-6) */
  int lbfgs_mem;      /* L-BFGS pairs, 1..MOTO_MAX_MEM                         (5) */
  double theta_max;   /* largest per-spin rotation of one step, rad             (0.2) */
  double gamma0;      /* steepest-descent scale without history, rad^2/meV      (0.02) */
  double tau_F;       /* force tolerance, meV/rad                               (1e-3) */
  double eta_theta;   /* largest per-spin rotation of a descent seed, rad       (0.1) */
  int max_steps;      /* ascent step cap                                       (300) */
  int descent_max_steps; /* descent step cap per side                          (5000) */
  int optimizer;      /* MOTO_OPT_*, used by ascent and descent                (LBFGS) */
  int subspace;       /* 1: reflect the force in all k Ritz vectors,
                         F_mmf = F - 2 V (V^T F) (the paper's subspace variant
                         for k > 1, P_min = V V^T); 0: in v1 only              (0) */
  int descent;        /* MOTO_DESCENT_*                                        (OPT) */
  double llg_alpha;   /* Gilbert damping of the LLG descent                    (1.0) */
  double llg_dt;      /* LLG time step, hbar/meV (0.6582 ps)                   (0.01) */
  double llg_time;    /* LLG duration per side, hbar/meV            (75.96 = 50 ps) */
  int reorth;         /* MOTO_REORTH_*, block Lanczos reorthogonalisation       (FULL) */
  double tau_lambda;  /* curvature threshold of the saddle test: lambda_1 < -tau_lambda
                         and lambda_2 > -tau_lambda (0: the printed test
                         lambda_1 < 0 < lambda_2), meV                        (0) */
} moto_params;

/* One ordered pair (i, i + d) of a pair-list Hamiltonian, d = d1 a1 + d2 a2
 * in index space. */
typedef struct {
  int d1, d2;
  double J;      /* exchange, meV */
  double D[3];   /* DMI vector (x, y, z), meV */
} moto_pair;

/* Fills *p with the defaults listed above. */
void moto_default_params(moto_params* p);

/* Creates a context for one lattice: validates the model (L1, L2 >= 5,
 * 1 <= n_shells <= 3) and params (k, block, steps, mem limits), then
 * allocates the scratch every later call uses.  dtype is MOTO_F32 or
 * MOTO_F64.  On success *out receives the context.  Must be called with the
 * target device current. */
int moto_create(const moto_model* model, int dtype, const moto_params* params, moto_ctx** out);

/* Replaces the context's exchange shells and Neel DMI by a general pair list
 * (an extension for many-shell parameterisations with full DMI vectors, such
 * as the paper's Pd/Fe/Ir(111) tables; K and muB of the model stay):
 *   E = - sum_i sum_p [ J_p m_i . m_{i+d_p} + D_p . (m_i x m_{i+d_p}) ]
 *       - muB sum_i m_iz - K sum_i m_iz^2.
 * The list must be closed under d -> -d with J_{-d} = J_d and D_{-d} = -D_d
 * (every bond counted twice, as in Eq. param-hamiltonian; checked exactly),
 * have no d = 0, at most MOTO_MAX_PAIRS entries, |d1|, |d2| <= MOTO_MAX_REACH
 * and L1, L2 >= 2 max(|d1|, |d2|) + 1.  Every later energy, gradient, HVP and
 * solver call of the context uses it; n_pairs = 0 restores the shell model.
 * Copies the list (synchronously); returns MOTO_ERR_ARG when a rule fails. */
int moto_set_pairs(moto_ctx* ctx, const moto_pair* pairs, int n_pairs);

/* Releases the context and its scratch (synchronises the device first). */
void moto_destroy(moto_ctx* ctx);

/* Energy and Riemannian gradient (Methods, "Gradient, HVP, and Hessian via
 * the autograd engine": F = -grad E understood as tangent-projected).
 * m_dev: unit spins (3N).  Writes, each optional (NULL to skip):
 *   g_dev  (3N): g_i = grad_i E - s_i m_i, the Riemannian gradient (F = -g);
 *   s_dev  (N):  s_i = m_i . grad_i E (needed by moto_hvp);
 *   out_dev (2 doubles): [E, max_i |g_i|].
 * E here is summed in double from per-site shares computed in the context
 * precision; moto_energy gives the FP64-arithmetic energy. */
int moto_energy_grad(moto_ctx* ctx, const void* m_dev, void* g_dev, void* s_dev,
                     double* out_dev, void* stream);

/* E(m) of Eq. param-hamiltonian evaluated in double arithmetic whatever the
 * context precision (final saddle and minimum energies).  E_dev: 1 double. */
int moto_energy(moto_ctx* ctx, const void* m_dev, double* E_dev, void* stream);

/* Tangent Hessian-vector products (Methods, "HVP operator mode"):
 *   (H v)_i = P_i [ (hess E v)_i - s_i v_i ],   P_i = I - m_i m_i^T,
 * for nvec tangent vectors v_j stored at v_dev + j*ldv (element stride ldv >=
 * 3N), results at hv_dev + j*ldhv.  s_dev from moto_energy_grad at the same m.
 * For tangent v this is the Riemannian Hessian on the product of spheres. */
int moto_hvp(moto_ctx* ctx, const void* m_dev, const void* s_dev, const void* v_dev,
             size_t ldv, void* hv_dev, size_t ldhv, int nvec, void* stream);

/* Energy and Euclidean gradient, the reverse-mode derivative an autodiff
 * engine takes of E (Methods, "Gradient, HVP, and Hessian via the autograd
 * engine"; the backward of torch.autograd.Function MotoEnergy):
 *   grad_dev (3N): grad_i E = h_i(m) - muB z - 2 K m_iz z (no projection);
 *   out_dev (2 doubles): [E, max_i |grad_i E|],
 * both evaluated in double arithmetic whatever the context precision (grad
 * stored in it).  m_dev need not be unit length here: E is the polynomial of
 * Eq. param-hamiltonian.  All pointers required. */
int moto_energy_euclid_grad(moto_ctx* ctx, const void* m_dev, void* grad_dev, double* out_dev, void* stream);

/* Euclidean Hessian-vector products (hess E v_j) for nvec vectors (Methods,
 * "HVP operator mode": the double backward of E).  E is quadratic in m, so
 * hess E is the same at every m and no state is read:
 *   (hess E v)_i = h_i(v) - 2 K v_iz z.
 * Layout and strides as for moto_hvp; v need not be tangent. */
int moto_euclid_hvp(moto_ctx* ctx, const void* v_dev, size_t ldv, void* hv_dev, size_t ldhv, int nvec,
                    void* stream);

/* Inner layer of the bilayer MMF kernel (Results, "Bilayer MMF"): the k
 * smallest eigenpairs of the tangent Hessian at m by HVP-driven block
 * Lanczos or LOBPCG (params->solver).
 *   v0_dev:  start vectors, params->block (Lanczos) or params->k (LOBPCG)
 *            fields of 3N elements, consecutive; projected on the tangent
 *            planes before use.
 *   V_dev:   out, k Ritz vectors (3N each, consecutive), tangent, unit norm,
 *            entry of largest magnitude positive (lowest index on ties).
 *   lam_dev: out, MOTO_MAX_BASIS doubles: the lowest Ritz values ascending
 *            (block Lanczos: the lowest min(16, basis size); LOBPCG: k);
 *            the other entries are set to +inf.
 *   info_dev: out, 2 ints: [iterations or steps done, device status].
 * s_dev may be NULL, in which case it is recomputed from m. */
int moto_lowest_modes(moto_ctx* ctx, const void* m_dev, const void* s_dev,
                      const moto_params* params, const void* v0_dev, void* V_dev,
                      double* lam_dev, int* info_dev, void* stream);

/* Topological charge Q = -(1/4pi) sum over the 2N elementary triangles of the
 * Berg-Luescher solid angle (up triangles (i, i+a1, i+a2), down triangles
 * (i+a1, i+a1+a2, i+a2)).  Q_dev: 1 double. */
int moto_topo_charge(moto_ctx* ctx, const void* m_dev, double* Q_dev, void* stream);

/* Masked perturbations of a reference configuration (Results,
 * "Multi-objective initial-configuration explorer": x = x0 + P_Omega delta,
 * followed by the spin-tangent retraction):
 *   out_j = R_x0(P_Omega P_x0 delta_j),  j < count,
 * i.e. on every active site the tangent part of delta_j at x0 rotates the spin
 * (Rodrigues), and inactive sites keep x0 exactly.
 *   x0_dev: unit spins (3N);  mask_dev: N bytes, nonzero = active (NULL: all);
 *   delta_dev: count fields at element stride ld_delta (>= 3N when count > 1),
 *   the caller's random draws;  out_dev: count fields at stride ld_out.
 * count <= 65535.  Enqueues only. */
int moto_perturb(moto_ctx* ctx, const void* x0_dev, const unsigned char* mask_dev, const void* delta_dev,
                 size_t ld_delta, int count, void* out_dev, size_t ld_out, void* stream);

/* Pairwise L1 distances of a population (the explorer's diversity objective;
 * the population figures of Fig. 2e-f are its pair sum and its smallest
 * off-diagonal entry):
 *   D[a*count + b] = sum over the 3N elements e of |X_a[e] - X_b[e]|,
 * 2 <= count <= MOTO_MAX_POP fields of X_dev at stride ldx >= 3N;
 * D_dev: count x count doubles (symmetric, zero diagonal).  Sums in FP64 in a
 * fixed order (FP32 fields: FP32 partial sums over a few hundred elements).
 * Uses the context's reduction scratch: calls on one context must not overlap
 * on the device.  Enqueues only. */
int moto_pairwise_l1(moto_ctx* ctx, const void* X_dev, size_t ldx, int count, double* D_dev, void* stream);

/* Skinny Gram product out[r * ny + c] = X_r . Y_c over the 3N elements of
 * nx <= MOTO_MAX_BASIS fields X_r (at X_dev + r * ldx) and ny <= MOTO_MAX_K
 * fields Y_c (at Y_dev + c * ldy), accumulated as the Krylov solvers do it
 * (FP32 products and short FP32 runs, then fixed-order sums in two-float
 * FP32 arithmetic, about 44 significant bits; all FP64 in an FP64 context).  out_dev: nx * ny doubles, row-major.  The building block of the
 * reorthogonalisation and Rayleigh-Ritz steps, exposed for checks of
 * orthogonality and for tests. */
int moto_gram(moto_ctx* ctx, const void* X_dev, size_t ldx, int nx, const void* Y_dev, size_t ldy,
              int ny, double* out_dev, void* stream);

/* Clears the L-BFGS history of the context (start of an ascent or descent). */
int moto_lbfgs_reset(moto_ctx* ctx, void* stream);

/* One step of the outer layer (Results, "Bilayer MMF"; Algorithm 1 of
 * Supplementary Note 1): g at m, the k lowest modes warm-started from V_dev,
 * F_mmf = F - 2 (F . v1) v1 with F = -g, the saddle test
 * max_i |F_mmf,i| <= tau_F and lambda_1 < 0 < lambda_2, and unless the test
 * passed, an L-BFGS step on -F_mmf capped at theta_max per spin and applied
 * by a per-spin Rodrigues rotation.
 *   m_dev:   in/out spins.  V_dev: in/out modes (k fields), also the start
 *            of the inner solve (the first block column when block > k is
 *            filled from v0 of the context's last solve).
 *   out_dev: out, 6 doubles [E, max|F_mmf,i|, lambda_1, lambda_2, max|g_i|, F.v1]
 *            at the m the step started from.
 *   status_dev: out, 1 int: 1 if the saddle test passed (m unchanged), else 0.
 * The L-BFGS history persists in the context between calls.  Called again
 * with the same pointers and parameter values (block Lanczos solver, no
 * launch profile recording), the step is captured once as a CUDA graph and
 * later calls replay it on `stream`; the results are bit-identical to the
 * kernel-by-kernel launches (MOTO_GRAPHS=0 in the environment).  Changing a
 * variant, the wait limit or the pair list discards the captured step. */
int moto_mmf_step(moto_ctx* ctx, void* m_dev, const moto_params* params, void* V_dev,
                  double* out_dev, int* status_dev, void* stream);

/* Runs moto_mmf_step until the saddle test passes or params->max_steps steps
 * were taken, reading the status word back every `check_every` steps
 * (synchronises the stream).  trace_dev (optional, 6 doubles per step,
 * max_steps+1 rows) receives each step's out vector.  *steps_out: steps
 * taken.  Returns MOTO_OK at a saddle, MOTO_NOT_CONVERGED at the cap.
 * With the block Lanczos solver (and no launch profile recording) the first
 * step runs launch by launch and the update step is then captured once as a
 * CUDA graph on a private stream, joined back to `stream`, and replayed; the
 * trace row of each replay is picked on the device from the steps taken.
 * moto_descend does the same for its steps.  Results are bit-identical to
 * launching every kernel (MOTO_GRAPHS=0 in the environment). */
int moto_ascend(moto_ctx* ctx, void* m_dev, const moto_params* params, void* V_dev,
                double* trace_dev, int check_every, int* steps_out, void* stream);

/* Two-sided descent (Results, "Deterministic bidirectional saddle descent";
 * Algorithm 1): seeds m_saddle +- eta v1 with eta = eta_theta / max_i |v1_i|
 * (retracted), each relaxed by the outer optimiser (params.optimizer) on g,
 * or with params.descent = MOTO_DESCENT_LLG by damped spin dynamics
 *   dm_i/dt = (m_i x g_i - alpha g_i) / (1 + alpha^2)
 * (Landau-Lifshitz-Gilbert with h = -grad E, time in hbar/meV; Heun with
 * renormalisation, step llg_dt, at most llg_time; Supplementary Note 2: alpha
 * = 1 for 50 ps, its T = 1e-6 taken as zero), until max_i |g_i| <= tau_F or
 * descent_max_steps (optimiser) / llg_time (LLG).  Writes m_plus_dev,
 * m_minus_dev (3N each) and
 * out_dev (6 doubles): [E+, Q+, E-, Q-, steps+, steps-] with E in double
 * arithmetic.  Synchronises the stream.  Returns MOTO_OK if both sides
 * converged, MOTO_NOT_CONVERGED otherwise. */
int moto_descend(moto_ctx* ctx, const void* m_saddle_dev, const void* v1_dev,
                 const moto_params* params, void* m_plus_dev, void* m_minus_dev,
                 double* out_dev, void* stream);

/* ------------------------------------------------------------------------
 * Batched walkers.  The paper runs the bilayer MMF kernel on many perturbed
 * starting points (Alg. 1, one walker per explorer proposal); the batch
 * advances n independent walkers together on one GPU.  Each walker has its
 * own lattice size (the model strengths are shared) and its own context
 * (workspace sized at creation); one outer step of all walkers is captured
 * once into a CUDA graph, fanned out over n_streams streams, and replayed
 * until every walker has stopped.  Walkers never exchange data.
 * ------------------------------------------------------------------------ */
typedef struct moto_batch moto_batch;
typedef struct {
  int L1, L2;   /* lattice of this walker (L >= 5) */
  void* m_dev;  /* 3N unit spins, caller-owned, updated in place */
  void* V_dev;  /* max(k, block) x 3N mode block: start block in, modes out */
} moto_walker;

/* Creates one context per walker (MOTO_ERR_NOMEM if any allocation fails;
 * nothing is kept then).  model->L1/L2 are ignored; walkers[i].L1/L2 are
 * used.  Buffers stay bound to the batch until moto_batch_destroy. */
int moto_batch_create(const moto_model* model, int dtype, const moto_params* params, const moto_walker* walkers,
                      int n_walkers, int n_streams, moto_batch** out);
void moto_batch_destroy(moto_batch* batch);

/* MMF ascent of every walker (as moto_ascend, params->max_steps outer steps
 * at most, the stopping test read every check_every steps).  rec_dev (n x 6
 * doubles, device): per walker [E, max_i|F_mmf,i|, lambda_1, lambda_2,
 * max_i|g_i|, g.v1] at its last test.  status_host / steps_host (n ints,
 * host, optional): MOTO_OK at a saddle, MOTO_NOT_CONVERGED at the cap, or
 * the walker's error; outer steps taken.  Synchronous.  Returns the worst
 * walker code. */
int moto_batch_ascend(moto_batch* batch, int check_every, double* rec_dev, int* status_host, int* steps_host,
                      void* stream);

/* Two-sided descent (as moto_descend, with the outer optimiser; a batch
 * created with params.descent = MOTO_DESCENT_LLG is refused with
 * MOTO_ERR_ARG) from every walker's current spins and
 * first mode: m_plus[i], m_minus[i] (3N each, device) receive the two
 * minima; out_dev (n x 6 doubles): [E+, Q+, E-, Q-, steps+, steps-]. */
int moto_batch_descend(moto_batch* batch, void* const* m_plus, void* const* m_minus, double* out_dev,
                       int* status_host, void* stream);

/* Device status word of the context (synchronises the stream): MOTO_OK or
 * the first device-detected error since the last moto_clear_status. */
int moto_status(moto_ctx* ctx, void* stream);
/* Clears the context's device status word (enqueued on the stream). */
int moto_clear_status(moto_ctx* ctx, void* stream);

/* Diagnostics of the last block Lanczos solve of the context (synchronises
 * the stream): *basis_dev receives the device address of its Krylov basis
 * (*nvec fields at element stride *ld, read-only, valid until the next solver
 * call of the context), *reorth_steps the number of steps that ran the full
 * pass against the basis (all of them with MOTO_REORTH_FULL, those the
 * orthogonality estimate asked for with MOTO_REORTH_SELECTIVE).  Each output
 * pointer is optional.  With moto_gram this measures Q^T Q - I. */
int moto_krylov_basis(moto_ctx* ctx, const void** basis_dev, size_t* ld, int* nvec, int* reorth_steps,
                      void* stream);

/* HVP autotuner.  The strip HVP kernel exists in several variants (strip
 * length, warps per block, spins held in registers, FP32 pair arithmetic as
 * packed f32x2 or scalar instructions) that give bit-identical results and
 * differ only in speed.  moto_create times each variant once on
 * its own scratch (vectors per call: params.block for block Lanczos,
 * params.k for LOBPCG) and records the fastest for (L1, L2, precision,
 * vectors) process-wide; later contexts of the same lattice reuse the record.
 * With MOTO_AUTOTUNE=0 in the environment variant 0 is recorded untimed.
 * moto_hvp_tuning returns the number of variants and writes the variant in
 * use (*variant, optional) and, when this context ran the timing, the
 * measured milliseconds per launch of each variant (ms[0 .. cap), optional;
 * zeros otherwise).  moto_set_hvp_variant forces a variant for every later
 * HVP of the context (-1 returns to the tuned one; MOTO_ERR_ARG when out of
 * range); the pair-list model has its own kernel and ignores it. */
int moto_hvp_tuning(const moto_ctx* ctx, int* variant, float* ms, int cap);
int moto_set_hvp_variant(moto_ctx* ctx, int variant);
/* The same for the energy / gradient stencil of moto_energy_grad and the
 * solvers (variants: staged tiles and blocks an SM, FP32 pair arithmetic
 * packed or scalar; g and s are bit-identical across them, the energy's sum
 * follows each variant's grid), timed by moto_create and recorded for (L1,
 * L2, precision).  moto_topo_charge uses the recorded variant's layout.  The
 * pair-list model and the FP64-arithmetic energy use their own kernels. */
int moto_stencil_tuning(const moto_ctx* ctx, int* variant, float* ms, int cap);
int moto_set_stencil_variant(moto_ctx* ctx, int variant);

/* Failure-detection control (host side only).  Every wait inside the
 * library's kernels is bounded: a consumer warp of the streaming
 * reorthogonalisation kernel that waits for a stage of tensor copies gives up
 * after about 2^22 blocking polls, drains the copies it has in flight, sets
 * MOTO_ERR_TIMEOUT in the context's status word and lets the launch finish.
 * polls > 0 replaces that bound by `polls` non-blocking tests for every later
 * solver call of the context, so that a test can make the waits give up and
 * check the reported status without a real stall; 0 restores the default.
 * The copies in flight are always drained with the full bound.  Results of a
 * solve whose waits gave up are meaningless; clear the status (and restore
 * the default) before relying on later calls.  Returns MOTO_ERR_ARG for
 * polls < 0. */
int moto_set_wait_limit(moto_ctx* ctx, int polls);

/* Human-readable text of a return code (static storage). */
const char* moto_status_string(int code);

/* Launch profiler (tracing).  moto_profile_begin starts recording a CUDA
 * event pair around each of the next `capacity` launches that the context's
 * solver sequences enqueue, tagged with a kernel class
 *   0 HVP, 1 Gram (skinny X^T Y), 2 field combination, 3 energy/gradient
 *   stencil, 4 single-block FP64 steps, 5 other field kernels, 6 the
 *   projected-matrix eigensolver, 7 block Lanczos local pass + Gram against
 *   the basis (read-only sweep), 8 block Lanczos full update + Cholesky Gram,
 *   9 second Cholesky QR Gram
 * and the algorithmic bytes of the launch (every field read or written once;
 * a launch of the full pass of a selective Lanczos step counts its bytes only
 * if the step took the pass, as the device's log of the last solve records).
 * moto_profile_end synchronises, writes per class (nkinds entries each,
 * NULL to skip) the number of launches, the summed event time in ms and the
 * summed algorithmic bytes, and releases the events.  Launches beyond
 * `capacity` are not recorded.  Not for use during stream capture. */
int moto_profile_begin(moto_ctx* ctx, int capacity);
int moto_profile_end(moto_ctx* ctx, int nkinds, int* launches, double* ms, double* bytes);

/* Allocation-free energy and Riemannian gradient (the paper has no
 * counterpart; it exists for callers that cannot allocate device memory).
 * Creating a moto_ctx allocates scratch, which some callers cannot do: a host
 * framework that owns all device memory and hands a library only the buffers
 * of each call, or a caller that must not risk the device-wide
 * synchronisation cudaMalloc / cudaFree may imply.  This call computes the
 * same outputs as moto_energy_grad (g_dev, s_dev, out_dev = [E, max_i |g_i|];
 * each optional) for the model and dtype given here, without a context.
 * Its only scratch is a fixed device array inside the library (512 KB + 256 B,
 * held by every GPU that loads the library until the process exits); it
 * holds the partial sums of at most 32768 tiles of 32 x 32 sites, so
 * ceil(L1/32) * ceil(L2/32) > 32768 (and, as for moto_create, L1 * L2 > 2^30)
 * is rejected with MOTO_ERR_ARG before any CUDA call.  The first call on a
 * device looks the array up with that device current and keeps its address
 * for the life of the process; make that first call outside any stream
 * capture, and do not use this call after a cudaDeviceReset of that device
 * (the library's module, and with it the array, may then move).  Every call
 * shares the array and keeps the last call's contents, so calls that overlap
 * on the GPU (several streams or devices' threads at once) race; serialise
 * them.  If a CUDA error from earlier work is pending on the calling thread,
 * the call launches nothing and returns MOTO_ERR_CUDA (the error stays
 * pending).  Non-finite inputs are not reported by this variant.  Calls no
 * cudaMalloc or cudaFree. */
int moto_energy_grad_noalloc(const moto_model* model, int dtype, const void* m_dev, void* g_dev,
                             void* s_dev, double* out_dev, void* stream);

/* Bytes of device scratch owned by the context. */
size_t moto_workspace_bytes(const moto_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* MOTO_H */
