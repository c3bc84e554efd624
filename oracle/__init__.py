"""FP64 CPU oracle for the fused lattice-Boltzmann + Tau-orthogonal LES step.

TEST INFRASTRUCTURE ONLY.  This package is the plain, slow, literal statement of
what the method computes, used to check the CUDA library.  Only the tests, the
package smoke check and the benchmark's CPU-baseline / reference legs may import
it.  It shares no code with the CUDA path: the only common inputs come from the
separate ``synthetic`` package of seeded generators.

Every function follows the paper's equations in the paper's order, in float64,
with numpy array operations standing in for loops over lattice nodes:

  lattice.py    D2Q9 / D3Q19 velocity sets (Sec. 2)
  lbm.py        equilibrium, moments, BGK relaxation, forcing, streaming (Sec. 2, Eqs. LES-1..3)
  substrate.py  Smagorinsky and WALE effective relaxation time (Sec. 5)
  filters.py    Gaussian, Laplacian and binomial convolution kernels (Eqs. gaussian, laplace)
  to.py         QoIs, sensitivities, Gram matrix, patterns, SGS increment (Sec. 4, App. A)
  lrs.py        linear regression with stochastic residuals (Eq. LRS)
  philox.py     Philox4x64-10 counter-based generator and Box-Muller normals
  ks.py         two-sample Kolmogorov-Smirnov distance (Eq. KS)
  sim.py        the full time step, composed from the above

Parity status: every function is pinned by a ``-m "not gpu"`` test against a
closed form, an invariant, a library routine or brute force (see tests/).
"""
