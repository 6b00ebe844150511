"""Reflected-force ascent, saddle test and two-sided descent (oracle, FP64).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Follows the outer layer of the bilayer MMF kernel (Results, "Bilayer MMF":
F_mmf = F - 2 (F^T v_min) v_min, climbed with a GPU L-BFGS; Algorithm 1 of
Supplementary Note 1: MinMode -> F -> F_mmf -> retraction until
|F_mmf| <= tau_F and lambda_1 < 0 < lambda_2; then x_saddle +- eta v_min relaxed
downhill).  Readings where the paper gives no rule:

* [R6] Optimiser: L-BFGS two-loop recursion (Nocedal & Wright, Numerical
  Optimization, Alg. 7.4) on the "gradient" G = -F_mmf (ascent) or G = g
  (descent), memory 5.  A new pair is formed at the current point from the
  last step and gradient, both projected on the current tangent planes
  (vector transport by projection, applied once when the pair is formed):
  s = P d_prev, y = G - P G_prev; it is kept only when s.y > 1e-12 |s||y|.
  The initial inverse Hessian is gamma I with gamma = s.y / y.y of the newest
  pair (gamma0 = 0.02 rad^2/meV without history).  If the direction is not a
  descent direction for G the history is cleared and d = -gamma0 G.  No line
  search (the reflected force is not a gradient field); instead the step is
  scaled so that the largest per-spin rotation is at most theta_max = 0.2 rad.
* [R7] Retraction: per-spin Rodrigues rotation (exponential map of S^2).
* [R8] |F_mmf| is read as max_i |F_mmf,i| (per-spin torque, meV/rad) with
  tau_F = 1e-3 meV/rad (1e-6 eV/rad); the index-1 signature uses the two lowest
  Ritz values of the inner solve.
* [R9] eta scales v1 so that the largest per-spin rotation of the seed is
  0.1 rad; "+" is the side along the sign-fixed v1 (R4); each side is relaxed by
  the same optimiser on G = g to max_i |F_i| <= tau_F (at most 5000 steps).
* [R15] Subspace variant (Results, "Bilayer MMF": for k > 1 the projector
  v v^T is replaced by P_min = V V^T): F_mmf = F - 2 V (V^T F) over the k
  orthonormal Ritz vectors; off by default (v1 only), the saddle test is
  unchanged.
* [R16] Nonlinear CG (the paper's alternative optimiser, Fig. 2g-h): the
  Polak-Ribiere+ direction p = -G + beta P p_prev with
  beta = max(0, G.(G - P G_prev) / |G_prev|^2) (Nocedal & Wright, eqs.
  5.44-5.45), transport by projection as for L-BFGS, a restart p = -G when p
  is not a descent direction for G.  No line search (R6): the step is
  alpha p with the spectral length alpha = s.y / y.y of the last step
  (s = P d_prev, y = G - P G_prev, kept when s.y > 1e-12 |s||y|, else gamma0;
  Barzilai & Borwein 1988, the same scale L-BFGS starts from), capped at
  theta_max per spin.  (A fixed alpha = gamma0 was tried first: on the
  32 x 32 workload it did not reach a saddle in 300 steps.)
* [R22] The saddle test's curvature threshold: Algorithm 1 takes thresholds
  (tau_F, tau_lambda) as inputs but prints the test as lambda_1 < 0 <
  lambda_2.  Read with tau_lambda: lambda_1 < -tau_lambda (one clearly
  negative curvature) and lambda_2 > -tau_lambda (no second one beyond the
  resolution of the curvatures, e.g. a soft translation mode of a texture on
  the periodic lattice); tau_lambda = 0 (the default) is the printed test.
* [R20] Dynamic certifier (Supplementary Note 1 (iii), "or dynamic simulator";
  Supplementary Note 2: atomistic spin dynamics, Gilbert damping alpha = 1,
  T = 1e-6, 50 ps): the Landau-Lifshitz-Gilbert equation in the
  Landau-Lifshitz form with the effective field h_i = -grad_i E in meV and
  time in units of hbar/meV (0.6582 ps):
      dm_i/dt = (m_i x g_i - alpha g_i) / (1 + alpha^2),
  g the Riemannian gradient (the tangent part of grad E; m x (m x h) = -h_t
  for unit m).  Heun predictor-corrector with renormalisation after each
  stage, step dt = 0.01 hbar/meV, at most 50 ps = 75.96 hbar/meV, stopped
  early when max_i |g_i| <= tau_F.  T = 1e-6 of the paper is taken as zero
  (no stochastic field; a thermal field of that size is far below the
  exchange and would make the trajectory non-deterministic).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from . import krylov, spin, topo


@dataclass
class MMFParams:
    k: int = 1
    solver: str = "lanczos"        # "lanczos" | "block_lanczos" | "lobpcg"
    krylov_steps: int = 60         # Lanczos steps (block steps for block Lanczos)
    tol: float = 1e-6              # LOBPCG residual tolerance, relative
    max_iter: int = 200            # LOBPCG iteration cap
    lbfgs_mem: int = 5
    theta_max: float = 0.2         # rad
    gamma0: float = 0.02           # rad^2 / meV
    tau_F: float = 1e-3            # meV / rad
    max_steps: int = 300
    eta_theta: float = 0.1         # rad
    descent_max_steps: int = 5000
    optimizer: str = "lbfgs"       # "lbfgs" | "cg" (R16)
    subspace: bool = False         # reflect all k modes (R15) instead of v1
    descent: str = "optimizer"     # "optimizer" | "llg" (R20)
    llg_alpha: float = 1.0         # Gilbert damping
    llg_dt: float = 0.01           # hbar/meV
    llg_time: float = 50.0 / 0.6582119569  # 50 ps in hbar/meV
    tau_lambda: float = 0.0        # curvature threshold of the saddle test (R22)


def _dot(a, b) -> float:
    return float(np.dot(a.ravel(), b.ravel()))


def max_torque(x: np.ndarray) -> float:
    """max_i |x_i| over sites."""
    return float(np.sqrt(np.max(np.sum(x * x, axis=0))))


class LBFGS:
    """Tangent-space L-BFGS direction with step cap (reading R6)."""

    def __init__(self, mem: int, gamma0: float, theta_max: float):
        self.mem = mem
        self.gamma0 = gamma0
        self.theta_max = theta_max
        self.S, self.Y = [], []
        self.d_prev = None
        self.G_prev = None

    def reset(self):
        self.S, self.Y = [], []

    def direction(self, m: np.ndarray, G: np.ndarray) -> np.ndarray:
        if self.d_prev is not None:
            s = spin.project(m, self.d_prev)
            y = G - spin.project(m, self.G_prev)
            sy = _dot(s, y)
            if sy > 1e-12 * math.sqrt(_dot(s, s) * _dot(y, y)):
                self.S.append(s)
                self.Y.append(y)
                if len(self.S) > self.mem:
                    self.S.pop(0)
                    self.Y.pop(0)
        # two-loop recursion
        q = G.copy()
        a = []
        for s, y in zip(reversed(self.S), reversed(self.Y)):
            rho = 1.0 / _dot(y, s)
            ai = rho * _dot(s, q)
            q = q - ai * y
            a.append(ai)
        if self.S:
            gamma = _dot(self.S[-1], self.Y[-1]) / _dot(self.Y[-1], self.Y[-1])
        else:
            gamma = self.gamma0
        r = gamma * q
        for (s, y), ai in zip(zip(self.S, self.Y), reversed(a)):
            rho = 1.0 / _dot(y, s)
            bi = rho * _dot(y, r)
            r = r + (ai - bi) * s
        d = -r
        if _dot(d, G) >= 0.0:
            self.reset()
            d = -self.gamma0 * G
        d = spin.project(m, d)
        tmax = max_torque(d)
        if tmax > self.theta_max:
            d = d * (self.theta_max / tmax)
        self.d_prev = d
        self.G_prev = G
        return d


class CG:
    """Tangent-space nonlinear CG, Polak-Ribiere+ with restarts and a spectral
    step length (reading R16)."""

    def __init__(self, gamma0: float, theta_max: float):
        self.gamma0 = gamma0
        self.theta_max = theta_max
        self.p_prev = None
        self.d_prev = None
        self.G_prev = None

    def reset(self):
        self.p_prev = None

    def direction(self, m: np.ndarray, G: np.ndarray) -> np.ndarray:
        alpha = self.gamma0
        if self.p_prev is None:
            p = -G
        else:
            y = G - spin.project(m, self.G_prev)
            s = spin.project(m, self.d_prev)
            beta = max(0.0, _dot(G, y) / _dot(self.G_prev, self.G_prev))
            p = -G + beta * spin.project(m, self.p_prev)
            if _dot(p, G) >= 0.0:
                p = -G
            sy = _dot(s, y)
            if sy > 1e-12 * math.sqrt(_dot(s, s) * _dot(y, y)):
                alpha = sy / _dot(y, y)
        d = alpha * p
        tmax = max_torque(d)
        if tmax > self.theta_max:
            d = d * (self.theta_max / tmax)
        self.p_prev = p
        self.d_prev = d
        self.G_prev = G
        return d


def make_optimizer(p: "MMFParams"):
    if p.optimizer == "lbfgs":
        return LBFGS(p.lbfgs_mem, p.gamma0, p.theta_max)
    if p.optimizer == "cg":
        return CG(p.gamma0, p.theta_max)
    raise ValueError(p.optimizer)


def min_mode(model, m, s, start, p: MMFParams):
    """Inner layer: (ritz values ascending, [v_1..v_k]) from warm start(s)."""
    if p.solver == "lanczos":
        lam, V = krylov.lanczos_modes(model, m, s, start[0], p.krylov_steps, p.k)
        return lam, V
    if p.solver == "block_lanczos":
        lam, V = krylov.block_lanczos_modes(model, m, s, start, p.krylov_steps, p.k)
        return lam, V
    if p.solver == "lobpcg":
        lam, V, _, _ = krylov.lobpcg_modes(model, m, s, start, p.k, p.tol, p.max_iter)
        return lam, V
    raise ValueError(p.solver)


@dataclass
class AscentResult:
    m: np.ndarray
    v1: np.ndarray
    lam: np.ndarray
    converged: bool
    steps: int
    trace: list = field(default_factory=list)


def reflected_force(F: np.ndarray, v1: np.ndarray) -> np.ndarray:
    """F_mmf = F - 2 (F . v1) v1 (Results, Bilayer MMF; Algorithm 1)."""
    return F - 2.0 * _dot(F, v1) * v1


def reflected_force_subspace(F: np.ndarray, V) -> np.ndarray:
    """F_mmf = F - 2 V (V^T F) for orthonormal V (Results, Bilayer MMF, the
    subspace variant with P_min = V V^T)."""
    out = F.copy()
    for v in V:
        out = out - 2.0 * _dot(F, v) * v
    return out


def saddle_test(fmax: float, lam, tau_F: float, tau_lambda: float = 0.0) -> bool:
    """|F_mmf| <= tau_F and lambda_1 < 0 < lambda_2 (Algorithm 1), read with
    the curvature threshold tau_lambda that Algorithm 1 takes as an input
    (R22): lambda_1 < -tau_lambda and lambda_2 > -tau_lambda; tau_lambda = 0
    is the printed test."""
    return fmax <= tau_F and lam[0] < -tau_lambda and lam[1] > -tau_lambda


def ascend(model, m0: np.ndarray, start: list, p: MMFParams) -> AscentResult:
    """Bilayer MMF from m0; ``start`` holds the k seeded start vectors of the
    first inner solve (later solves warm-start from the previous modes)."""
    m = m0.copy()
    opt = make_optimizer(p)
    V = [x.copy() for x in start]
    trace = []
    converged = False
    lam = None
    step = 0
    for step in range(p.max_steps + 1):
        g, s = spin.riemann_grad(model, m)
        lam, V = min_mode(model, m, s, V, p)
        v1 = V[0]
        F = -g
        Fm = reflected_force_subspace(F, V[:p.k]) if p.subspace else reflected_force(F, v1)
        fmax = max_torque(Fm)
        trace.append(dict(E=spin.energy(model, m), fmax=fmax, lam1=float(lam[0]), lam2=float(lam[1])))
        if saddle_test(fmax, lam, p.tau_F, p.tau_lambda):
            converged = True
            break
        if step == p.max_steps:
            break
        d = opt.direction(m, -Fm)
        m = spin.retract(m, d)
    return AscentResult(m=m, v1=V[0], lam=np.asarray(lam), converged=converged, steps=step, trace=trace)


@dataclass
class DescentResult:
    m: np.ndarray
    E: float
    Q: float
    Qint: int
    converged: bool
    steps: int


def relax(model, m0: np.ndarray, p: MMFParams):
    """RelaxDownhill: the optimiser on G = g until max_i |F_i| <= tau_F."""
    m = m0.copy()
    opt = make_optimizer(p)
    converged = False
    step = 0
    for step in range(p.descent_max_steps + 1):
        g, _ = spin.riemann_grad(model, m)
        if max_torque(g) <= p.tau_F:
            converged = True
            break
        if step == p.descent_max_steps:
            break
        d = opt.direction(m, g)
        m = spin.retract(m, d)
    return m, converged, step


def llg_rate(model, m: np.ndarray, alpha: float):
    """dm/dt of the damped LLG equation (R20) and the gradient it used."""
    g, _ = spin.riemann_grad(model, m)
    mxg = np.stack([m[1] * g[2] - m[2] * g[1], m[2] * g[0] - m[0] * g[2], m[0] * g[1] - m[1] * g[0]])
    return (mxg - alpha * g) / (1.0 + alpha * alpha), g


def _unit(m: np.ndarray) -> np.ndarray:
    return m / np.sqrt(np.sum(m * m, axis=0))[None]


def llg_step(model, m: np.ndarray, alpha: float, dt: float):
    """One Heun step with renormalisation (R20); returns (m_new, g at m)."""
    k1, g = llg_rate(model, m, alpha)
    mp = _unit(m + dt * k1)
    k2, _ = llg_rate(model, mp, alpha)
    return _unit(m + 0.5 * dt * (k1 + k2)), g


def llg_relax(model, m0: np.ndarray, p: MMFParams):
    """Damped spin dynamics until max_i |g_i| <= tau_F or llg_time (R20)."""
    m = m0.copy()
    nmax = int(math.ceil(p.llg_time / p.llg_dt - 1e-9))
    for step in range(nmax + 1):
        g, _ = spin.riemann_grad(model, m)
        if max_torque(g) <= p.tau_F:
            return m, True, step
        if step == nmax:
            break
        m, _ = llg_step(model, m, p.llg_alpha, p.llg_dt)
    return m, False, nmax


def descent_seeds(m_saddle: np.ndarray, v1: np.ndarray, p: MMFParams):
    """x_saddle +- eta v1, retracted (reading R9)."""
    eta = p.eta_theta / max_torque(v1)
    return spin.retract(m_saddle, eta * v1), spin.retract(m_saddle, -eta * v1)


def descend(model, m_saddle: np.ndarray, v1: np.ndarray, p: MMFParams):
    """Two-sided descent: returns (DescentResult for +, DescentResult for -)."""
    out = []
    for seed in descent_seeds(m_saddle, v1, p):
        if p.descent == "llg":
            m, conv, steps = llg_relax(model, seed, p)
        else:
            m, conv, steps = relax(model, seed, p)
        q = topo.topo_charge(m)
        out.append(DescentResult(m=m, E=spin.energy(model, m), Q=q, Qint=int(round(q)), converged=conv, steps=steps))
    return out[0], out[1]
