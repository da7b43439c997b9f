"""FP64 CPU oracle for the explicit MTP scheme with SAT time stepping (Maxwell).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.

It is a plain, slow, deliberately independent implementation of what the
paper defines (arXiv:1906.11029):

* ``simplex``  Bernstein basis on each element (not the GPU path's orthonormal
  basis), exact integration of barycentric monomials, Duffy / Gauss-Legendre
  quadrature for projecting non-polynomial data.
* ``mesh``     topology and affine geometry of a conforming simplicial mesh.
* ``maxwell``  the conservation-law pieces of Sec. 3: skew, g(u), f(u), the
  mapped mass operator u -> g(u) - f(u) grad(phi), its closed-form inverse
  (end of Sec. 4), and the upwind / PEC numerical fluxes.
* ``pitch``    tent pitching (Sec. 2) under the causality condition.
* ``mtp``      per-tent assembly of M(t), M', A on the vertex patch (Sec. 3)
  and the q-stage SAT recursion over m sub-intervals (Sec. 4), the layer-by-
  layer evolution, projection, lattice evaluation, L2 error and energy.
* ``brute``    brute-force cross-checks: a global (non-tent) upwind DG + classical
  RK4 solver built by quadrature, and the Y-substituted classical RK4 tent stepper
  that Sec. 3 and Sec. 5.1 contrast with SAT.
* ``adjoint``  the discrete adjoint of the tent evolution (dense transposes).

Every function cites the paper passage (section / equation) it follows.
Readings of the paper where it is silent or garbled are listed in the
module docstrings where they are used.
"""
