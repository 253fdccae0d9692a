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

Parity status: the full switching dynamics of an island is pinned only
through its invariants and closed-form special cases (no trajectory is printed
in the paper) -- "parity unpinned" beyond those, see tests/test_oracle_*.py.
"""
