"""FP64 CPU oracle for the staggered RHMC hot path (Bonati, Cossu, D'Elia,
Di Giacomo, "Staggered fermions simulations on GPUs", Lattice 2010).

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, obviously correct
restatement of what the method computes, written from the paper and the works
it cites.  Only the tests, the smoke check and the CPU-baseline leg of the
benchmark may import it; the product path (the CUDA library and its Python
binding) never does, and the oracle imports nothing from the product.

Modules
  lattice     geometry, parity, staggered phases, boundary signs     (Sec. 2)
  su3         SU(3) algebra: generators, exp, projections, reunitarise (Sec. 4)
  dirac       unimproved staggered D, even/odd blocks, A = m^2 - D_eo D_oe (Sec. 2)
  asqtad      improved (asqtad) staggered D: fat and Naik links, its force (not in the paper)
  hisq        HISQ links (fat7, U(3) projection, fat7 + Lepage, Naik) and force (not in the paper)
  solvers     CG and multi-shift CG (Jegerlehner, hep-lat/9612014)     (Sec. 6)
  rational    Remez minimax rational approximation, partial fractions  (Sec. 2)
  actions     Wilson gauge action and force; fermion action and force (Sec. 2, 4)
  integrator  2nd-order minimum-norm multi-step MD and the RHMC trajectory (Sec. 2, 4)
  philox      counter-based Philox4x64-10 generator and Gaussian draws
  surrogate   loop features and the MLP force surrogate (forward + backward)

Every function works in float64 / complex128 on whole-lattice numpy arrays:
  gauge  U[mu, t, z, y, x, 3, 3]   (mu = 0..3 for x, y, z, t)
  field  psi[t, z, y, x, 3]
so that U.reshape(4, V, 3, 3) is the canonical lexicographic order
site = x + Lx*(y + Ly*(z + Lz*t)).

Parity status: every function listed above is pinned by tests that do not
use the oracle itself (closed forms, identities, dense linear algebra, finite
differences, library special cases).  The ensemble averages of a full RHMC
chain (plaquette at a given beta) have no printed value in the paper and are
parity unpinned.
"""
