"""Oracle: a plain, slow, single-threaded-by-construction FP64 CPU flux
reconstruction (FR) solver for the compressible Euler and Navier-Stokes
equations on mixed prism/tetrahedral meshes.

TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
benchmark's CPU-baseline leg may import anything from this package.  It
shares no code with the CUDA path and the CUDA path never calls it.

What it follows (the paper fixes the scheme's shape, not its details):
  * the FR method with the correction that recovers nodal DG (Sec. 3.4),
    written as constant operator matrices applied to row-major state
    matrices, C <- c1 A B + c2 C (Sec. 2.1, Eq. 1);
  * the volume-to-surface interpolation operator M0 whose sizes Table 2 lists;
  * point-wise flux, Rusanov interface and boundary work (Sec. 2.1, Sec. 3.4);
  * compressible Navier-Stokes with constant viscosity (Sec. 3.4), no-slip
    isothermal walls and Riemann-invariant far-field boundaries (Sec. 3.2);
  * classic RK4 time stepping (one of the steppers of Table 1).
Where the paper is silent (point sets, operator definitions, LDG viscous
interface treatment, boundary ghost states, wave-speed estimate) the oracle
takes the readings listed in each module's docstring.

Module map:
  basis.py    exact (rational / 60-digit decimal) points and operators
  geometry.py element maps, Jacobians, metric terms, normals
  mesh.py     face connectivity, periodic matching, flux-point pairing
  physics.py  fluxes, Rusanov, LDG, boundary states
  solver.py   RHS pipeline, RK4, reductions, time step
"""
