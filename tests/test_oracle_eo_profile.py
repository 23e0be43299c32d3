"""Electro-osmotic flow of the Debye-Hueckel theory (Sec. IV.A.1): with the
body force rho(y) E_x of the linearised Poisson-Boltzmann charge density
between two walls of equal surface charge (rho = -eps phi''), the no-slip
Stokes solution is the profile of Eq. fluidvel1.  The oracle's staggered
Stokes solve reproduces it at second order in the grid spacing.

Reading: Eq. PhiWalls as printed gives -eps dphi/dy = -varsigma at y = 0,
the opposite of the boundary condition stated with it (phi_zeta =
lambda varsigma / eps, Eq. potentials); the potential that meets the
stated condition is phi^0 - phi_zeta [1 - cosh((L - 2y) / 2 lambda)]
csch(L / 2 lambda), and Eq. fluidvel1, as printed, follows from it."""
import numpy as np

from oracle import stokes


def eo_force_and_profile(Ny, lam, eps, zeta, E, eta):
    """rho(y) E_x at the cell centres and Eq. fluidvel1 there."""
    L = float(Ny)
    y = np.arange(Ny) + 0.5
    csch = 1.0 / np.sinh(L / (2 * lam))
    coth = np.cosh(L / (2 * lam)) / np.sinh(L / (2 * lam))
    c = np.cosh((L - 2 * y) / (2 * lam))
    rho = -eps * zeta / lam ** 2 * c * csch         # -eps phi'' (reading above)
    v = -(eps * zeta * E / eta) * (coth - c * csch)  # Eq. fluidvel1
    return rho * E, v


def _solve(Ny, lam):
    Nx = Nz = 4
    eps, zeta, E, eta = 0.08, 0.3, 0.05, 1.0 / (6 * np.pi)
    fxy, v = eo_force_and_profile(Ny, lam, eps, zeta, E, eta)
    fx = np.broadcast_to(fxy[None, :, None], (Nz, Ny, Nx)).copy()
    fy = np.zeros((Nz, Ny + 1, Nx))
    fz = np.zeros((Nz, Ny, Nx))
    u, vv, w, p = stokes.solve(fx, fy, fz, eta)
    return u[0, :, 0], v, (vv, w)


def test_eo_profile_second_order():
    errs = []
    for Ny in (32, 64):
        lam = Ny / 8.0
        u, v, (vv, w) = _solve(Ny, lam)
        assert np.abs(vv).max() < 1e-12 and np.abs(w).max() < 1e-12
        errs.append(np.abs(u - v).max() / np.abs(v).max())
    assert errs[0] < 1e-2
    # halving the spacing (at fixed L / lambda) quarters the error
    assert 3.0 < errs[0] / errs[1] < 5.0
