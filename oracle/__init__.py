"""Reference oracle: TEST INFRASTRUCTURE, not part of the product.

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import, call, link or execute anything in this package.  The CUDA
library never routes through it and shares no code with it (no kernels,
headers, helpers or tables); the two meet only in the seeded input generators
of the ``workloads`` package, which hold none of the method's arithmetic.

Tiers (each function cites the passage it follows):

* ``bruteforce`` -- O1: literal sums over histories (Eqs. 3-5) and over
  internal-wire assignments (Sec. II-A) for tiny circuits.
* ``dense`` -- O2: dense state-vector simulation (Eq. 1 applied to all
  outputs at once) for up to ~24 qubits.
* ``feynman`` -- O3: the reduced-history method restated plainly in C
  (analysis, Algorithm 1, Algorithm 2, Eq. (gateops), autotuning) with
  compensated summation.
* ``closed_forms`` -- O4: QFT closed form, coined-walk offset-space
  simulation, fidelity.

Every function here is pinned by ``tests/test_oracle_*.py`` against values the
paper prints, closed forms, invariants or brute force.
"""
