"""FP64 CPU oracle for the wall-bounded DISCOS particle-grid hot path.

This package is TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import it. The product path
(``paper_2204_14167_gb300``) never imports it, and nothing here imports the
product: the two share no code, headers, tables or constant generators.

Everything is written plainly in numpy/scipy, in float64, following the
method of Ladiges et al., "Modeling electrokinetic flows with the discrete ion
stochastic continuum overdamped solvent algorithm" (arXiv 2204.14167):

  kernels.py    IB kernels: 4-point Peskin (App. B, Eq. peskin1d), 6-point
                Peskin (cited in Sec. II.A; rebuilt from its moment
                conditions), ES kernel (App. B, Eq. eskernel)
  gridops.py    spreading / interpolation with wall images and ghost cells
                (Sec. II.A Eqs. kernel1-kernel2, Fig. folded; Sec. II.B.1),
                per column over a metal strip, and with a hydrodynamic
                kernel per species (App. B)
  poisson.py    7-point Poisson with Dirichlet / Neumann walls
                (Eqs. poisson, esbc1, esbc3), assembled and solved by CG;
                a metal strip in a dielectric wall (Sec. IV.B)
  greens.py     lattice Green's function of the 7-point Laplacian and the
                pre-tabulated grid pair force F^P (Sec. II.B.1, Eq. LC)
  particles.py  cell binning, P3M near-field correction with images
                (Eqs. coulomb, fullElectro, LC), LJ/WCA (Eqs. potential,
                closerange), wall repulsion (Sec. II.B.2)
  mobility.py   near-wall mobility fit (Eq. fitfunction), channel formula
                (Eqs. mob_analytic, singlewall), dry tensor (Eqs. diff1-diff2)
  stokes.py     staggered MAC Stokes with no-slip or slip walls (Eqs.
                disc_stokes, fluidbc), stochastic stress, RFD thermal forcing
                (Eq. thermforce), the assembled MAC residual
  philox.py     Philox4x32-10 counter-based generator + Box-Muller
  integrate.py  the four-stage time step (Sec. II.D): forces, dry
                Euler-Maruyama update (Eq. ions3) and the midpoint scheme
                (Eqs. step1-step2)

Functions whose result is not fixed by a pin (a closed form, an invariant, a
special case or brute force) say "parity unpinned" in their docstring.
"""
