"""FP64 CPU oracle for one explicit inertial-coupling (IC) time step.

TEST INFRASTRUCTURE ONLY.  This package is the slow, plain, obviously-correct
statement of what the GPU path computes, written from the paper (Balboa
Usabiaga & Delgado-Buscalioni, "A minimal model for acoustic forces on
Brownian particles", arXiv 1307.0702).  Only ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.
The product path (``paper_1307_0702_gb300``) never imports, calls or links it,
and it shares no code with the CUDA library: the only common module is the
seeded workload generator, which holds no arithmetic of the method.

Modules
-------
peskin  : 3-point Roma-Peskin function, staggered kernel weights, J and S
          (Sec. 2, Eqs. (Jdis), (Sdis), (k1), (k2), (kvol); App. A.1).
philox  : Philox4x32-10 counter-based generator and the Box-Muller normal
          transform used for the stochastic stress (App. A.2, Eqs. for W_1..W_3).
fluid   : conservative staggered flux divergence and the SSP-RK3 substep
          (Sec. 4.2 Eqs. (eq:consvDens), (eq:consvMom), (totp); App. A.2).
ic      : the full IC time step, substeps 1-7 of App. A.2, with the particle
          pressure of Eqs. (eq:pressure), (omega).
slabs   : the same step with the box split into z-slabs over ranks (halo
          exchange, owner-computed particle gathers, replicated spreads),
          pinned bit for bit to ``ic`` over gloo ranks.
adjoint : the reverse-mode derivative (transpose) of the deterministic step,
          for gradients of the time-averaged tether force (Sec. 6) with
          respect to m_e, kappa_p/kappa_f, the drive amplitude and the state;
          pinned by complex-step and central differences of the forward.
theory  : closed forms used as pins (Eqs. (eq:acousticForce2), (f1), (f2),
          (part_svel), (ke), (eq:densityVariance); discrete dispersion).

Parity status
-------------
Every function here is pinned by a ``-m "not gpu"`` test against something
other than itself (closed forms, invariants, published known answers, brute
force).  The nonlinear advection flux, whose discretisation the paper leaves
to a reference that is not available, is pinned to the paper's continuum
term -div(g v) (Eq. (eq:consvMom)): on a smooth flow its error falls at
second order in h, against exact spectral derivatives.  Which second-order
form (here products of two-point averages) is a reading; its rounding order
is checked against the GPU only by self-consistency.
"""
