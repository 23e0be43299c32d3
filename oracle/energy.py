"""Discrete electrostatic energy of the grid (particle-mesh) problem.

Test infrastructure only (see ``oracle/__init__``).

The paper defines no energy; reading: with rho = S^es q (images included) and
phi the solution of Eq. poisson with the wall conditions of Eqs. esbc1 /
esbc3,
    U = dV sum_j rho_j (phi^rho_j / 2 + phi^b_j),
where phi^rho solves the homogeneous-wall problem and phi^b is the discrete
lift of the wall data (the solution with rho = 0).  Since phi = phi^rho +
phi^b this is U = (1/2) sum_j rho_j (phi_j + phi^b_j).  The near-field
(P3M) pair energy is not included.  The oracle evaluates U plainly; its
gradients are checked by finite differences of this function.
"""
import numpy as np

from . import gridops, poisson


def lift(dims, bc, lB, phi_b, surf_charge):
    """phi^b: the grid solution with rho = 0 and the wall data."""
    Nx, Ny, Nz = dims
    return poisson.solve(np.zeros((Nz, Ny, Nx)), bc, lB, phi_b, surf_charge)


def energy(p, pos, q, phi_b=None):
    phi_b = p['phi_b'] if phi_b is None else phi_b
    rho = gridops.spread_charge(p['kernel_es'], pos, q, p['dims'], p['bc'])
    phi = poisson.solve(rho, p['bc'], p['lB'], phi_b, p['surf_charge'])
    phib = lift(p['dims'], p['bc'], p['lB'], phi_b, p['surf_charge'])
    return 0.5 * float(np.sum(rho * (phi + phib)))
