"""Pins of the oracle's discrete electrostatic energy (oracle/energy.py)
against facts that do not come from the oracle itself: the closed-form lift
of the wall data, summation by parts, the kernel's moment conditions, and
the electrostatic force of Eq. efieldop."""
import numpy as np
import pytest

from oracle import energy as oe, gridops, poisson
from paper_2204_14167_gb300 import RunConfig
from helpers import oracle_params, rel_l2

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")


def _params(bc=(0, 0), phi_b=(0.5, -0.5), surf=(0.0, 0.0), n=(16, 16, 16), lB=7.0):
    cfg = RunConfig(Nx=n[0], Ny=n[1], Nz=n[2], bc=bc, phi_b=phi_b, surf_charge=surf, lB=lB, kernel_es=1)
    return oracle_params(cfg)


def _ions(rng, n, dims, margin):
    Nx, Ny, Nz = dims
    pos = np.stack([rng.uniform(0, Nx, n), rng.uniform(margin, Ny - margin, n), rng.uniform(0, Nz, n)])
    q = np.array([1.0, -1.0] * (n // 2))
    return pos, q


@pytest.mark.parametrize("bc,phi_b,surf", [((0, 0), (0.5, -0.5), (0, 0)),
                                           ((0, 1), (0.3, 0.0), (0.0, 0.02)),
                                           ((1, 0), (0.0, -0.2), (0.05, 0.0))])
def test_lift_is_the_linear_profile(bc, phi_b, surf):
    # A linear function of y is harmonic for the 7-point Laplacian and meets
    # the ghost-cell rules of Eqs. esbc1 / esbc3 exactly, so the discrete lift
    # must be the straight line fixed by the wall data.
    p = _params(bc, phi_b, surf, n=(8, 12, 8))
    Ny = 12
    lift = oe.lift(p['dims'], bc, p['lB'], phi_b, surf)
    y = np.arange(Ny) + 0.5
    g0, g1 = -4 * np.pi * p['lB'] * surf[0], 4 * np.pi * p['lB'] * surf[1]
    if bc == (0, 0):
        ref = phi_b[0] + (phi_b[1] - phi_b[0]) * y / Ny
    elif bc == (0, 1):
        ref = phi_b[0] + g1 * y
    else:
        ref = phi_b[1] + g0 * (y - Ny)
    np.testing.assert_allclose(lift, np.broadcast_to(ref[None, :, None], lift.shape), atol=1e-11)


def test_energy_is_the_field_energy():
    # Summation by parts with grounded walls: (1/2) rho.phi equals (eps/2)
    # times the sum of squared potential differences over the interior and
    # periodic faces, plus 2 phi^2 for each wall cell (its ghost-cell row,
    # phi_ghost = -phi).  A wrong factor or sign in U fails this.
    p = _params(phi_b=(0.0, 0.0))
    rng = np.random.default_rng(3)
    pos, q = _ions(rng, 24, p['dims'], 1.0)
    U = oe.energy(p, pos, q)
    rho = gridops.spread_charge(p['kernel_es'], pos, q, p['dims'], p['bc'])
    phi = poisson.solve(rho, p['bc'], p['lB'], (0.0, 0.0), (0.0, 0.0))
    eps = 1.0 / (4 * np.pi * p['lB'])
    s = np.sum((np.roll(phi, -1, 2) - phi) ** 2) + np.sum((np.roll(phi, -1, 0) - phi) ** 2)
    s += np.sum((phi[:, 1:, :] - phi[:, :-1, :]) ** 2)
    s += 2 * np.sum(phi[:, 0, :] ** 2) + 2 * np.sum(phi[:, -1, :] ** 2)
    assert U > 0
    assert abs(U - 0.5 * eps * s) <= 1e-9 * U


def test_energy_wall_term_from_kernel_moments():
    # U is quadratic in q, and U(phi_b) - U(0) = sum_j rho_j phi^b_j.  For ions
    # whose stencil stays clear of the walls the kernel reproduces linear
    # functions exactly (first moment condition, App. B), so the wall term is
    # sum_i q_i phi^b(y_i) with the linear lift.
    p = _params()
    rng = np.random.default_rng(4)
    pos, q = _ions(rng, 16, p['dims'], 3.01)
    U0 = oe.energy(p, pos, q, phi_b=(0.0, 0.0))
    U2 = oe.energy(p, pos, 2.0 * q, phi_b=(0.0, 0.0))
    assert abs(U2 - 4.0 * U0) <= 1e-10 * abs(U0)
    Ub = oe.energy(p, pos, q)
    y = pos[1]
    wall = np.sum(q * (0.5 + (-0.5 - 0.5) * y / 16.0))
    assert abs((Ub - U0) - wall) <= 1e-10 * max(abs(wall), 1.0)


def test_minus_grad_energy_is_the_field_force():
    # -dU/dx_i (central differences of U) against q_i E^P of Eq. efieldop.
    # The identity is exact only for the gradient-kernel force; the face-field
    # force of the paper differs by discretisation error (about 2% here), so
    # the gate is 5e-2.  A sign error or a missing factor 2 fails it.
    p = _params()
    rng = np.random.default_rng(1)
    pos, q = _ions(rng, 16, p['dims'], 3.5)
    rho = gridops.spread_charge(p['kernel_es'], pos, q, p['dims'], p['bc'])
    phi = poisson.solve(rho, p['bc'], p['lB'], p['phi_b'], p['surf_charge'])
    sl = poisson.wall_slopes(p['bc'], p['surf_charge'], p['lB'])
    F = q * gridops.efield_at_ions(p['kernel_es'], pos, phi, p['bc'], p['phi_b'], sl)
    h = 1e-4
    k = 6
    G = np.zeros((3, k))
    for i in range(k):
        for d in range(3):
            a = pos.copy(); a[d, i] += h
            b = pos.copy(); b[d, i] -= h
            G[d, i] = (oe.energy(p, a, q) - oe.energy(p, b, q)) / (2 * h)
    assert rel_l2(-G, F[:, :k]) < 5e-2
