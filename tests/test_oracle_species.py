"""Pins of the oracle's per-species hydrodynamic kernels (App. B: on one
hydrodynamic grid the cations spread and interpolate with the ES kernel of
w = 7, beta = 7 and the anions with w = 4, beta = 8), each fixed by the
paper's definitions rather than by the oracle's own code:

* every ion's footprint on the grid is its own species' kernel width along
  each axis (Eq. eskernel: support |z| <= w/2, so w grid points);
* per-species spreading and interpolation stay adjoint (Eq. adjoint,
  <S F, v> = <F, J v>) for any mix of species and wall conditions;
* with one kernel for every species they reduce to the single-kernel
  operators, and the thermal forcing of a run whose ions all belong to one
  species is the single-kernel forcing with that species' kernel.
"""
import numpy as np
import pytest

from oracle import gridops, kernels, stokes

K77 = kernels.Kernel(kernels.ES, 7, 7.0)
K48 = kernels.Kernel(kernels.ES, 4, 8.0)
DIMS = (16, 16, 16)


def _random_state(N, seed, dims=DIMS):
    Nx, Ny, Nz = dims
    rng = np.random.default_rng(seed)
    pos = np.stack([rng.uniform(0, Nx, N), rng.uniform(0.2, Ny - 0.2, N), rng.uniform(0, Nz, N)])
    pos[1, :4] = rng.uniform(0.1, 1.5, 4)          # near the walls: images in play
    pos[1, 4:8] = Ny - rng.uniform(0.1, 1.5, 4)
    sp = rng.integers(0, 2, N).astype(np.int32)
    F = rng.normal(size=(3, N))
    return pos, sp, F, rng


@pytest.mark.parametrize("species", [0, 1])
def test_footprint_is_the_species_kernel_width(species):
    pos = np.array([[8.3], [8.1], [7.6]])
    ks = [K77, K48]
    f = gridops.spread_force_species(ks, np.array([species]), pos, np.ones((3, 1)), DIMS)
    w = ks[species].w
    assert w == (7, 4)[species]
    for g in f:
        nz = np.nonzero(g)
        for axis in range(3):
            assert len(np.unique(nz[axis])) == w


@pytest.mark.parametrize("slip", [(False, False), (True, False)])
def test_species_operators_adjoint(slip):
    Nx, Ny, Nz = DIMS
    pos, sp, F, rng = _random_state(40, 21)
    u, w = rng.normal(size=(Nz, Ny, Nx)), rng.normal(size=(Nz, Ny, Nx))
    v = rng.normal(size=(Nz, Ny + 1, Nx))
    v[:, 0] = v[:, Ny] = 0.0
    ks = [K77, K48]
    f = gridops.spread_force_species(ks, sp, pos, F, DIMS, slip)
    V = gridops.interp_velocity_species(ks, sp, pos, u, v, w, slip)
    lhs = sum(np.sum(a * b) for a, b in zip(f, (u, v, w)))
    assert abs(lhs - np.sum(F * V)) < 1e-12 * abs(lhs)


def test_one_kernel_for_all_species_reduces():
    Nx, Ny, Nz = DIMS
    pos, sp, F, rng = _random_state(30, 22)
    u, w = rng.normal(size=(Nz, Ny, Nx)), rng.normal(size=(Nz, Ny, Nx))
    v = rng.normal(size=(Nz, Ny + 1, Nx))
    v[:, 0] = v[:, Ny] = 0.0
    a = gridops.spread_force_species([K48, K48], sp, pos, F, DIMS)
    b = gridops.spread_force(K48, pos, F, DIMS)
    for x, y in zip(a, b):
        assert np.allclose(x, y, rtol=0, atol=1e-14)
    Va = gridops.interp_velocity_species([K48, K48], sp, pos, u, v, w)
    Vb = gridops.interp_velocity(K48, pos, u, v, w)
    assert np.allclose(Va, Vb, rtol=0, atol=1e-14)


@pytest.mark.parametrize("species", [0, 1])
def test_thermal_forcing_of_one_species(species):
    pos, _, _, _ = _random_state(12, 23)
    sp = np.full(12, species, dtype=np.int32)
    ks = [K77, K48]
    a = stokes.rfd_forcing(ks, pos, DIMS, 1.0, 5, 0, 99, species=sp)
    b = stokes.rfd_forcing(ks[species], pos, DIMS, 1.0, 5, 0, 99)
    other = stokes.rfd_forcing(ks[1 - species], pos, DIMS, 1.0, 5, 0, 99)
    for x, y, z in zip(a, b, other):
        assert np.allclose(x, y, rtol=0, atol=1e-12)
        assert not np.allclose(x, z, rtol=0, atol=1e-6)


def test_thermal_forcing_of_es_kernels_is_at_its_limit():
    """The RFD of ES kernels is taken at delta = 1e-7: a ten times larger
    delta gives the same forcing to O(delta^2) for these positions (no
    stencil point within delta |W| of a support edge), i.e. the default sits
    at the delta -> 0 limit that the reading asks for."""
    pos, sp, _, _ = _random_state(40, 24)
    ks = [K77, K48]
    a = stokes.rfd_forcing(ks, pos, DIMS, 1.0, 5, 0, 99, species=sp)
    b = stokes.rfd_forcing(ks, pos, DIMS, 1.0, 5, 0, 99, delta=1e-6, species=sp)
    for x, y in zip(a, b):
        assert np.linalg.norm(x - y) < 1e-6 * np.linalg.norm(y)
