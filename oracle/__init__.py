"""Plain, slow FP64 CPU oracle for two-flavour Wilson-fermion HMC.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this
package: only the tests, the smoke check of ``__graft_entry__`` and the
CPU-baseline / reference legs of ``bench.py`` may use it.  It shares no
code with the CUDA library and does not import it.

Every function writes out the definition it follows, with no fusion,
blocking or reordering beyond what that definition states.  The paper
(Chakrabarty & Majumdar, "Hybrid Monte Carlo with Wilson Dirac operator on
the Fermi GPU") names the pieces but prints no formulas; the conventions
used here (listed in ``conventions``) are the readings this project takes,
each pinned by tests against mathematics that does not depend on them:
closed forms, adjointness, gauge covariance, brute-force dense algebra,
finite differences, reversibility and the epsilon^2 scaling of Delta H.

Modules
  conventions  gamma matrices, su(3) generators, lattice neighbours
  wilson       hopping term H, M = 1 - kappa H, M^dag, M^dag M   (Eq. 4)
  cg           conjugate gradient on M^dag M                     (Sec. 1, Sec. 3)
  gauge        plaquette, Wilson gauge action, gauge force       (Eq. 1, Sec. 3 kernel 2)
  fermion      pseudofermion action and fermion force            (Eq. 3-5, Sec. 3 kernel 3)
  su3          exp(i eps p), reunitarisation, link update        (Sec. 2, Sec. 3 kernel 4)
  hmc          Hamiltonian, leapfrog, Metropolis, trajectory     (Eq. 5, Sec. 2, Sec. 3)
"""
from . import conventions, wilson, cg, gauge, fermion, su3, hmc  # noqa: F401
