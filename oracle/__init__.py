"""FP64 CPU oracle for the batched ECC-island LLG path -- test infrastructure.

Only the tests, the smoke check and the CPU-baseline leg of the benchmark may
import this package.  It shares no code with the CUDA library: it reads the
same seeded inputs (the synthetic mesh, jitter and head-map arrays) and
computes everything else itself in float64 with plain numpy, following the
textbook micromagnetics that the paper's solver rests on (Sec. II.A: a hybrid
FEM/BEM solver of the Landau-Lifshitz-Gilbert equation at 0 K) and the
readings that the paper leaves open (time integrator, discretisation, switch
criterion), each stated in the module that implements it.

Modules
  fem       P1 tetrahedral geometry, exchange stiffness, lumped volumes
  demag     Fredkin-Koehler FEM/BEM demagnetising operator (Lindholm weights)
  headfield trilinear lookup of the write-head field map
  llg       effective field, Heun integrator with renormalisation, switch detector
  mlp       surrogate MLP forward/backward, BCE loss, AdamW, screened error rates
  ber       bit-error-rate formulas of Sec. II.C (Eqs. 1-3)
  hcrit     critical-field search of Sec. II.C
  neb       nudged elastic band for the adjacent-track barrier (Sec. II.C, Eq. 3)
  ego       efficient global optimisation: maximin Latin hypercube, kriging, EI (Sec. II.A)

Parity status: every module is pinned (tests/test_oracle_*.py).  The
dynamics of a meshed island are pinned through closed-form special cases
(macrospin precession, damped reversal, the Stoner-Wohlfarth astroid), the
linear modes of a meshed two-layer island (an eigenproblem of its exchange and
anisotropy operators) and invariants (|m| = 1, energy decay under damping).
The large-angle switching of a meshed island has no closed form, and the paper
prints no trajectory: it rests on those pins.
"""
