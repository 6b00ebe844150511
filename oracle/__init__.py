"""FP64 CPU oracle for the bilayer minimum-mode kernel (arXiv 2509.26269).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import anything from this package.  The
product path (``paper_2509_26269_gb300``) never imports it and has no CPU
fallback.

The oracle is a plain, slow, obviously-correct restatement of what the paper
computes, in float64 numpy, written from the paper's definitions:

* ``model``  -- lattice shells and model parameters (Methods, "Spin Hamiltonian
  and manifold gradient", Eq. param-hamiltonian).
* ``spin``   -- energy, Euclidean and Riemannian gradient, tangent HVP, explicit
  dense Hessian (Methods, "Gradient, HVP, and Hessian via the autograd engine";
  "Explicit Hessian for benchmarking").
* ``krylov`` -- Lanczos, block Lanczos and LOBPCG for the k smallest tangent
  eigenpairs (Results, "Bilayer MMF", inner layer; Supplementary Note 1).
* ``mmf``    -- reflected-force ascent with retraction, saddle test, two-sided
  descent (Results, "Bilayer MMF" and "Deterministic bidirectional saddle
  descent"; Algorithm 1).
* ``topo``   -- lattice topological charge Q (Results, Pd/Fe/Ir(111) networks:
  Q = +1 skyrmion, -1 antiskyrmion).
* ``pairs``  -- a general pair-list Hamiltonian (many shells, full DMI vectors)
  with its derivatives, of which the shell model is one instance.
* ``explorer`` -- masked perturbations x0 + P_Omega delta and the objectives
  of the initial-configuration explorer (Results, "Multi-objective
  initial-configuration explorer").

It shares no code with the CUDA path; both sides only share the seeded input
generators in ``inputs``.

Parity status: every function is pinned by a test against a closed form, an
invariant or a library routine (``tests/test_oracle_*.py``), except the
trajectory of the ascent itself, whose end point is pinned by the saddle
signature of the dense spectrum (see ``mmf``).
"""
from .model import Model, SHELLS, model_from_workload  # noqa: F401
from . import spin, krylov, mmf, topo, explorer, pairs  # noqa: F401
