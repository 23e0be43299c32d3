"""Pins of the oracle's metal strip (a Dirichlet patch inside a dielectric
wall, Sec. IV.B, Fig. EOgeometry; mixed conditions on one wall, Sec. II.B.1):

* no strip cells: the dielectric (Neumann) bottom wall of the plain solver;
* the strip covering the whole wall: the conducting (Dirichlet) wall;
* the mixed operator is symmetric (self-adjoint solve);
* discrete maximum principle: with no charge, the strip at potential 1 and a
  grounded top wall, 0 < phi < 1 inside (an M-matrix operator; a wrong sign
  in the strip's ghost rows breaks it);
* the strip potential of Sec. IV.B makes phi + phi_E constant on the strip.
"""
import numpy as np

from oracle import poisson

DIR, NEU = poisson.DIRICHLET, poisson.NEUMANN


def _rho(dims, seed=0):
    Nx, Ny, Nz = dims
    return np.random.default_rng(seed).normal(size=(Nz, Ny, Nx))


def test_no_strip_is_dielectric_wall():
    dims = (8, 6, 4)
    rho = _rho(dims)
    none = np.zeros((dims[2], dims[0]), dtype=bool)
    a = poisson.solve_strip(rho, 0.7, none, np.zeros_like(none, dtype=float), DIR, phi_b_top=0.3,
                            surf=(0.02, 0.0))
    b = poisson.solve(rho, (NEU, DIR), 0.7, (0.0, 0.3), (0.02, 0.0))
    assert np.allclose(a, b, rtol=0, atol=1e-10 * np.abs(b).max())


def test_full_strip_is_conducting_wall():
    dims = (8, 6, 4)
    rho = _rho(dims, 1)
    full = np.ones((dims[2], dims[0]), dtype=bool)
    a = poisson.solve_strip(rho, 0.7, full, np.full(full.shape, -0.4), NEU, surf=(0.0, 0.01))
    b = poisson.solve(rho, (DIR, NEU), 0.7, (-0.4, 0.0), (0.0, 0.01))
    assert np.allclose(a, b, rtol=0, atol=1e-10 * np.abs(b).max())


def test_strip_operator_symmetric():
    dims = (12, 6, 4)
    strip = poisson.strip_columns(dims, 3.0, 7.0)
    A = poisson.assemble_strip(dims, NEU, strip)
    assert abs(A - A.T).max() == 0.0
    # non-singular although both walls are dielectric apart from the strip
    x = np.random.default_rng(2).normal(size=A.shape[0])
    assert np.linalg.norm(A @ x) > 1e-3 * np.linalg.norm(x)


def test_strip_maximum_principle():
    dims = (16, 8, 4)
    strip = poisson.strip_columns(dims, 5.0, 11.0)
    phi = poisson.solve_strip(np.zeros((4, 8, 16)), 1.0, strip, np.ones((4, 16)), DIR, phi_b_top=0.0)
    assert phi.min() > 0.0 and phi.max() < 1.0
    # largest above the strip, next to the wall
    j = np.unravel_index(np.argmax(phi), phi.shape)
    assert j[1] == 0 and strip[j[0], j[2]]


def test_strip_potential_cancels_applied_field():
    dims = (16, 8, 4)
    x0, x1, E = 4.0, 12.0, 0.3
    pm = poisson.strip_potential(dims, x0, x1, 0.25, E)
    xc = np.arange(16) + 0.5
    phi_E = -E * (xc - 0.5 * (x0 + x1))
    on = (xc >= x0) & (xc < x1)
    assert np.allclose((pm[0] + phi_E)[on], 0.25)


def test_full_strip_images_and_ghosts_are_conducting_wall():
    """A strip over the whole bottom wall turns every strip rule into the
    conducting wall's: the charge images (spreading), the ghost cells of the
    field interpolation and the near-field image partners."""
    from oracle import gridops, particles, kernels, greens
    dims = (16, 8, 16)
    rng = np.random.default_rng(4)
    N = 40
    pos = np.stack([rng.uniform(0, 16, N), rng.uniform(0.05, 8, N), rng.uniform(0, 16, N)])
    q = rng.choice([-1.0, 1.0], N)
    k = kernels.Kernel(kernels.PESKIN4)
    full = (0.0, 16.0, 0.0)
    a = gridops.spread_charge(k, pos, q, dims, (NEU, NEU), full)
    b = gridops.spread_charge(k, pos, q, dims, (DIR, NEU))
    assert np.allclose(a, b, atol=1e-14)
    phi = rng.normal(size=(16, 8, 16))
    Ea = gridops.efield_at_ions(k, pos, phi, (NEU, NEU), (0.0, 0.0), (0.0, 0.0), full, 0.0)
    Eb = gridops.efield_at_ions(k, pos, phi, (DIR, NEU), (0.0, 0.0), (0.0, 0.0))
    assert np.allclose(Ea, Eb, atol=1e-13)
    p = dict(dims=dims, lB=1.0, psi=4.0, lj_sigma=[[1.0]], lj_xi=[[0.0]], lj_rc=[[0.5]], bc=(NEU, NEU),
             strip=full)
    tab = greens.fp_table(kernels.PESKIN4, 4.0, 16)
    Fa, ca = particles.near_field(pos, q, np.zeros(N, int), p, tab)
    p2 = dict(p, bc=(DIR, NEU), strip=None)
    Fb, cb = particles.near_field(pos, q, np.zeros(N, int), p2, tab)
    assert np.array_equal(ca, cb) and np.allclose(Fa, Fb, atol=1e-13)
