"""Reference oracle for the matrix-free Q_k hex operators (test infrastructure only).

This package is a plain, slow, fp64 CPU restatement of what the GPU path computes.
It is used only by ``tests/``, by ``__graft_entry__.smoke()`` and by the CPU-baseline
leg of ``bench.py``; the library itself never imports, links or calls it, and it
shares no code with the CUDA path (only the seeded generators in ``synthetic``).

The method (a matrix-free, sum-factorised operator evaluation) reproduces, up to
rounding order, the action of the globally assembled matrix built from the same
element integrals with the same Gauss rule.  So the oracle *is* that definition:

* ``basis``    Lagrange Q_k shape functions on equispaced nodes and the tensor
               Gauss rule with (k+1)^3 points (Appendix B: continuous Lagrange
               elements, Gaussian quadrature with (k_i+1)^dim points);
* ``coeffs``   coefficient laws of Section 2.3 (eqs. heaviside, muEff, rhoEff),
               the tanh-regularised Heaviside read from eq. initial_phi, k(T),
               and the Gaussian laser flux of eq. laser_gauss;
* ``mesh``     lattice numbering of uniform meshes and of 2:1 octree leaf lists,
               hanging-node constraints by interpolation from the coarse side;
* ``assemble`` element matrices by full quadrature (every basis function
               evaluated at every point, no sum factorisation), assembly into
               CSR, constraints as C^T A C, Dirichlet rows/columns as identity;
* ``krylov``   textbook CG, right-preconditioned restarted GMRES, Jacobi,
               Chebyshev and Lanczos (Appendix B: CG for symmetric and GMRES
               for nonsymmetric systems);
* ``heat``     one implicit heat step, the box objective and its adjoint
               gradients with respect to the laser parameters and k_q;
* ``interface`` the interface source terms of Section 2.4 (smoothed delta,
               mass flux, dilation, cooling, hybrid recoil) as load vectors;
* ``patch``    single rows of full-size operators from 2 x 2 x 2-cell patches
               (parity of the benchmark-size applies);
* ``step``     one step of Algorithm algo:meltpooldg (predictors, level-set
               advection and reinitialisation, heat, Navier-Stokes) by direct
               sparse solves, in stage functions.
"""
