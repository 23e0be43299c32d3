"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Nothing here compares the oracle with itself: each test checks a closed form,
an invariant, a special case that reduces to a textbook construction, a
published known-answer vector, or brute force by an unrelated algorithm.
"""
import os

import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import kernels, philox, gridops, poisson, greens, particles, mobility, stokes, integrate

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ------------------------------------------------------------------ kernels
def _moments(kern, r):
    """Sums over the grid of z^m phi(z) for particle offsets r (z = r - j)."""
    j = np.arange(-8, 9)
    z = r[:, None] - j[None, :]
    ph = kern(z)
    even = np.where(j % 2 == 0, ph, 0).sum(1)
    odd = np.where(j % 2 != 0, ph, 0).sum(1)
    return ph, z, even, odd


def test_peskin4_conditions():
    """App. B, Eq. peskin1d: the 4-point kernel's defining properties."""
    r = np.linspace(0, 1, 10001)
    ph, z, even, odd = _moments(kernels.peskin4, r)
    assert np.allclose(even, 0.5, atol=1e-14) and np.allclose(odd, 0.5, atol=1e-14)
    assert np.allclose((z * ph).sum(1), 0.0, atol=1e-14)
    assert np.allclose((ph ** 2).sum(1), 3.0 / 8.0, atol=1e-14)
    assert kernels.peskin4(np.array([0.0, 1.0, 2.0]))[0] == 0.5
    assert np.allclose(kernels.peskin4(np.array([1.0, 2.0, 2.5])), [0.25, 0.0, 0.0])


def test_peskin6_conditions():
    """6-point kernel (cited in Sec. II.A): moments 0..3 and sum of squares."""
    K = kernels.K6
    r = np.linspace(0, 1, 2001)
    ph, z, even, odd = _moments(kernels.peskin6, r)
    assert np.allclose(even, 0.5, atol=1e-13) and np.allclose(odd, 0.5, atol=1e-13)
    assert np.allclose((z * ph).sum(1), 0.0, atol=1e-13)
    assert np.allclose((z ** 2 * ph).sum(1), K, atol=1e-13)
    assert np.allclose((z ** 3 * ph).sum(1), 0.0, atol=1e-12)
    # closed form of the sum of squares, derived by hand from the conditions
    C = 3 * K ** 2 / 32 - 11 * K / 32 + 67 / 128
    assert np.allclose((ph ** 2).sum(1), C, atol=1e-13)
    assert np.allclose(kernels.peskin6(np.array([3.0, -3.0, 3.5])), 0.0, atol=1e-15)
    assert abs(kernels.peskin6(np.array([0.0]))[0] - (5 / 8 - K / 4)) < 1e-14


def test_peskin6_is_C3_and_not_C4():
    """K = 59/60 - sqrt(29)/20 is the value that makes the kernel C^3."""
    h = 1e-3
    for z0 in (1.0, 2.0, 3.0, 0.0):
        # one-sided polynomial extrapolation of derivatives from each side
        zl = z0 - h * np.arange(1, 7)
        zr = z0 + h * np.arange(1, 7)
        fl = kernels.peskin6(zl)
        fr = kernels.peskin6(zr)
        pl = np.polyfit(zl - z0, fl, 5)
        pr = np.polyfit(zr - z0, fr, 5)
        for order in range(4):
            dl = np.polyval(np.polyder(pl, order), 0.0)
            dr = np.polyval(np.polyder(pr, order), 0.0)
            assert abs(dl - dr) < 1e-5 * max(1, 10 ** order), (z0, order, dl, dr)
    # a different K breaks third-derivative continuity at the edge of support
    zr = 3.0 - 1e-3 * np.arange(1, 7)
    f = kernels.peskin6(zr, K=0.70)
    d3 = np.polyval(np.polyder(np.polyfit(zr - 3.0, f, 5), 3), 0.0)
    assert abs(d3) > 1e-3


def test_es_kernel_normalised():
    """App. B, Eq. eskernel: unit integral; grid sums approach 1."""
    k = kernels.ESKernel(6, 8.0)
    from scipy import integrate
    val, _ = integrate.quad(k, -3, 3, epsabs=1e-14, limit=200)
    assert abs(val - 1.0) < 1e-12
    r = np.linspace(0, 1, 101)
    s = k(r[:, None] - np.arange(-5, 6)[None, :]).sum(1)
    assert np.all(np.abs(s - 1.0) < 1e-3)


# ------------------------------------------------------------------ Philox
def test_philox_known_answers():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for row in rows:
        c = [int(x, 16) for x in row[:4]]
        k = [int(x, 16) for x in row[4:6]]
        expect = [int(x, 16) for x in row[6:10]]
        out = philox.philox4x32(np.array([c[0]]), c[1], c[2], c[3], k[0] | (k[1] << 32))
        assert [int(o[0]) for o in out] == expect


def test_box_muller_moments():
    g = philox.normals4(np.arange(200000), 7, 0, 1, 12345)
    x = np.concatenate(g)
    assert abs(x.mean()) < 5e-3 and abs(x.var() - 1.0) < 5e-3
    assert abs(np.mean(x ** 4) - 3.0) < 3e-2


# ------------------------------------------------------------------ spreading / interpolation
@pytest.mark.parametrize("kind", [kernels.PESKIN4, kernels.PESKIN6])
def test_adjoint_identity_with_walls(kind):
    """Eq. adjoint: (J v).F = dV (S F).v, including image folds and ghosts."""
    rng = np.random.default_rng(1)
    dims = (8, 10, 6)
    Nx, Ny, Nz = dims
    k = kernels.Kernel(kind)
    pos = np.stack([rng.uniform(0, Nx, 40), rng.uniform(0.05, Ny - 0.05, 40), rng.uniform(0, Nz, 40)])
    pos[1, :4] = [0.0, 0.3, Ny - 0.2, Ny]        # on and near the walls
    F = rng.normal(size=(3, 40))
    u = rng.normal(size=(Nz, Ny, Nx)); w = rng.normal(size=(Nz, Ny, Nx))
    v = rng.normal(size=(Nz, Ny + 1, Nx)); v[:, 0, :] = 0; v[:, Ny, :] = 0
    fx, fy, fz = gridops.spread_force(k, pos, F, dims)
    V = gridops.interp_velocity(k, pos, u, v, w)
    lhs = np.sum(V * F)
    rhs = np.sum(fx * u) + np.sum(fy * v) + np.sum(fz * w)
    assert abs(lhs - rhs) < 1e-12 * np.sum(np.abs(V * F))
    # zero normal mobility on the wall: an ion on the wall spreads no f_y
    one = np.zeros((3, 1)); one[1] = 1.0
    for y in (0.0, float(Ny)):
        _, fy1, _ = gridops.spread_force(k, np.array([[3.3], [y], [2.2]]), one, dims)
        assert np.abs(fy1).max() < 1e-15


@pytest.mark.parametrize("kind", [kernels.PESKIN4, kernels.PESKIN6])
def test_charge_images(kind):
    """Neumann (like-charge images): dV sum(rho) = sum(q) exactly; Dirichlet
    (opposite images): an ion on the wall leaves no net charge."""
    rng = np.random.default_rng(2)
    dims = (8, 12, 8)
    k = kernels.Kernel(kind)
    pos = np.stack([rng.uniform(0, 8, 30), rng.uniform(0, 12, 30), rng.uniform(0, 8, 30)])
    q = rng.choice([-1.0, 1.0], 30)
    rho = gridops.spread_charge(k, pos, q, dims, (1, 1))
    assert abs(rho.sum() - q.sum()) < 1e-13
    rho = gridops.spread_charge(k, np.array([[2.5], [0.0], [3.1]]), np.array([1.0]), dims, (0, 1))
    assert abs(rho.sum()) < 1e-14
    far = gridops.spread_charge(k, np.array([[2.5], [6.0], [3.1]]), np.array([1.0]), dims, (0, 0))
    assert abs(far.sum() - 1.0) < 1e-14


def test_linear_potential_field_everywhere():
    """A potential linear in y (the discrete harmonic lift between Dirichlet
    walls, and a uniform slope between Neumann walls) gives the exact uniform
    field at every ion, including ions whose stencil crosses a wall."""
    dims = (8, 16, 8)
    Nx, Ny, Nz = dims
    rng = np.random.default_rng(3)
    pos = np.stack([rng.uniform(0, Nx, 50), rng.uniform(0, Ny, 50), rng.uniform(0, Nz, 50)])
    for kind in (kernels.PESKIN4, kernels.PESKIN6):
        k = kernels.Kernel(kind)
        phi = poisson.solve(np.zeros((Nz, Ny, Nx)), (0, 0), 1.0, phi_b=(0.3, -0.5))
        yc = np.arange(Ny) + 0.5
        assert np.allclose(phi, (0.3 + (-0.8) * yc / Ny)[None, :, None], atol=1e-12)
        E = gridops.efield_at_ions(k, pos, phi, (0, 0), (0.3, -0.5), (0, 0))
        assert np.allclose(E[1], 0.8 / Ny, atol=1e-12) and np.allclose(E[[0, 2]], 0, atol=1e-12)
        g = 0.07
        phiN = g * yc[None, :, None] * np.ones((Nz, Ny, Nx))
        E = gridops.efield_at_ions(k, pos, phiN, (1, 1), (0, 0), (g, g))
        assert np.allclose(E[1], -g, atol=1e-12)


# ------------------------------------------------------------------ Poisson
def _basis_y(Ny, bc):
    """Eigenvectors of the wall-row second difference in y (columns) and
    eigenvalues: DST-II (D-D), DCT-II (N-N), quarter-wave (D-N, N-D)."""
    j = np.arange(Ny) + 0.5
    m = np.arange(Ny)
    if bc == (0, 0):
        th = np.pi * (m + 1) / Ny; B = np.sin(np.outer(j, th))
    elif bc == (1, 1):
        th = np.pi * m / Ny; B = np.cos(np.outer(j, th))
    elif bc == (0, 1):
        th = np.pi * (m + 0.5) / Ny; B = np.sin(np.outer(j, th))
    else:
        th = np.pi * (m + 0.5) / Ny; B = np.cos(np.outer(j, th))
    return B, 2 - 2 * np.cos(th)


@pytest.mark.parametrize("bc", [(0, 0), (1, 1), (0, 1), (1, 0)])
def test_poisson_against_explicit_eigenbasis(bc):
    """The CG solution equals the explicit spectral solution built from the
    textbook eigenbases (DFT in x, z; DST/DCT variants in y) by O(N^2) sums."""
    rng = np.random.default_rng(4)
    Nx, Ny, Nz = 6, 10, 4
    rho = rng.normal(size=(Nz, Ny, Nx))
    if bc == (1, 1):
        rho -= rho.mean()
    lB = 0.7
    phi = poisson.solve(rho, bc, lB)
    By, ly = _basis_y(Ny, bc)
    By = By / np.linalg.norm(By, axis=0)
    Fx = np.exp(-2j * np.pi * np.outer(np.arange(Nx), np.arange(Nx)) / Nx)
    Fz = np.exp(-2j * np.pi * np.outer(np.arange(Nz), np.arange(Nz)) / Nz)
    lx = 2 - 2 * np.cos(2 * np.pi * np.arange(Nx) / Nx)
    lz = 2 - 2 * np.cos(2 * np.pi * np.arange(Nz) / Nz)
    b = 4 * np.pi * lB * rho
    bh = np.einsum('ak,kji,ib->ajb', Fz, b, Fx)           # DFT in z and x
    bh = np.einsum('jm,ajb->amb', By, bh)                  # project onto y-basis
    lam = lz[:, None, None] + ly[None, :, None] + lx[None, None, :]
    with np.errstate(divide='ignore', invalid='ignore'):
        ph = np.where(lam > 1e-14, bh / lam, 0.0)
    ph = np.einsum('jm,amb->ajb', By, ph)
    ref = np.einsum('ka,ajb,bi->kji', Fz.conj(), ph, Fx.conj()).real / (Nx * Nz)
    if bc == (1, 1):
        ref -= ref.mean()
    assert np.abs(phi - ref).max() < 1e-11 * np.abs(ref).max()


def test_poisson_neumann_requires_neutrality():
    rho = np.zeros((4, 6, 4)); rho[1, 2, 3] = 1.0
    with pytest.raises(ValueError):
        poisson.solve(rho, (1, 1), 1.0)
    # neutral once the walls carry the opposite surface charge
    sc = -1.0 / (2 * 16)
    phi = poisson.solve(rho, (1, 1), 1.0, surf_charge=(sc, sc))
    r, b = poisson.residual(phi, rho, (1, 1), 1.0, surf_charge=(sc, sc))
    assert np.abs(r).max() < 1e-10 * np.abs(b).max()


# ------------------------------------------------------------------ Green's function and F^P
def test_lattice_green_watson():
    """G(0) = W/6 with Watson's integral W = pi^-3 int dk / (1 - sum cos k / 3)
    in its Gamma-function closed form;
    the lattice Laplacian of G is the unit impulse; far field 1/(4 pi r)."""
    from scipy.special import gamma
    W = np.sqrt(6) / (32 * np.pi ** 3) * gamma(1 / 24) * gamma(5 / 24) * gamma(7 / 24) * gamma(11 / 24)
    assert abs(greens.lattice_green(0, 0, 0) - W / 6) < 1e-13
    G = greens.green_box(4)
    R = 4
    lap = 6 * G[1:-1, 1:-1, 1:-1] - (G[2:, 1:-1, 1:-1] + G[:-2, 1:-1, 1:-1] + G[1:-1, 2:, 1:-1]
                                     + G[1:-1, :-2, 1:-1] + G[1:-1, 1:-1, 2:] + G[1:-1, 1:-1, :-2])
    delta = np.zeros_like(lap); delta[R - 1, R - 1, R - 1] = 1.0
    assert np.abs(lap - delta).max() < 1e-12
    r = np.sqrt(12 ** 2 + 5 ** 2)
    assert abs(greens.lattice_green(12, 5, 0) * 4 * np.pi * r - 1.0) < 2e-3


def test_grid_pair_force_far_field_is_coulomb():
    """Beyond the kernel the grid pair force approaches Coulomb 1/r^2 along
    +xhat_ij (like charges repel), the deviation shrinking with distance."""
    k = kernels.Kernel(kernels.PESKIN4)
    R = 26
    G = greens.green_box(R)
    xj = np.array([10.3, 10.6, 10.1])
    u = np.array([1.0, 2.0, 2.0]) / 3.0
    devs = []
    for r in (6.0, 12.0, 20.0):
        F = greens.pair_grid_force(k, xj + r * u, xj, G, R)
        devs.append(abs(F @ u * r * r - 1.0))
        assert np.linalg.norm(F - (F @ u) * u) * r * r < 0.5 * devs[-1] + 1e-6
    assert devs[0] < 0.015 and devs[1] < 0.005 and devs[2] < 0.002
    assert devs[0] > devs[1] > devs[2]


# ------------------------------------------------------------------ near field
def _base_params(dims, bc, kind=kernels.PESKIN4, psi=2.0, lB=1.0, n_tab=32):
    return dict(dims=dims, bc=bc, phi_b=(0.0, 0.0), surf_charge=(0.0, 0.0),
                kernel_es=kernels.Kernel(kind), kernel_hy=kernels.Kernel(kind),
                lB=lB, psi=psi, fp_table=greens.fp_table(kind, psi, n_tab),
                lj_sigma=[[1.0]], lj_xi=[[0.0]], lj_rc=[[0.0]],
                wall_sigma=[1.0], wall_xi=[0.0], wall_rc=[0.0], E_ext=(0, 0, 0))


def test_single_ion_image_force_matches_image_series():
    """Sec. III.B: the P3M force on one ion between grounded (Dirichlet) walls
    against the method of images (alternating image series).  As in the paper,
    forces are averaged over random (x, z) placements to remove the kernels'
    translational variance.  psi = 4 (the 4-point kernel's support width),
    where the grid pair force has reached Coulomb to 0.2%.  Gates: normal
    force within 3%, mean lateral force below 0.01 l_B q^2 (the translational
    variance floor of a single charge)."""
    dims = (64, 16, 64)
    p = _base_params(dims, (0, 0), psi=4.0, n_tab=64)
    L = dims[1]
    rng = np.random.default_rng(0)
    for y0 in (0.7, 1.5, 2.5, 4.0, 7.0):
        Fs = []
        for _ in range(6):
            pos = np.array([[rng.uniform(0, 64)], [y0], [rng.uniform(0, 64)]])
            F, counts, parts = integrate.forces(p, pos, np.array([1.0]), np.array([0]))
            Fs.append(F[:, 0])
        Fm = np.mean(Fs, axis=0)
        n = np.arange(-4000, 4001)
        d = 2.0 * (y0 - n * L)
        ref = -np.sum(np.sign(d) / d ** 2)
        assert abs(Fm[1] - ref) < 0.03 * abs(ref), (y0, Fm[1], ref)
        assert abs(Fm[0]) < 0.01 and abs(Fm[2]) < 0.01


def test_pair_table_matches_channel_grid_force():
    """The unbounded lattice-Green pair force equals the force the Poisson
    pipeline (spread, channel solve, face field, interpolation) gives for
    the same pair far from the walls of a wide Dirichlet channel."""
    k = kernels.Kernel(kernels.PESKIN4)
    R = 12
    G = greens.green_box(R)
    dims = (48, 48, 48)
    p = _base_params(dims, (0, 0), psi=4.0, n_tab=8)
    xj = np.array([24.3, 24.1, 23.8])
    for r, u in ((1.5, np.array([1.0, 0, 0])), (2.7, np.array([1.0, 1.0, 1.0]) / np.sqrt(3))):
        xi = xj + r * u
        pos = np.stack([xi, xj], axis=1)
        _, _, E = integrate.electrostatic_field(p, pos[:, 1:], np.array([1.0]))
        rho, phi, _ = integrate.electrostatic_field(p, pos[:, 1:], np.array([1.0]))
        Ei = gridops.efield_at_ions(k, pos[:, :1], phi, (0, 0), (0, 0), (0, 0))[:, 0]
        Fg = greens.pair_grid_force(k, xi, xj, G, R)
        assert np.linalg.norm(Ei - Fg) < 2e-3 * np.linalg.norm(Fg), (r, Ei, Fg)


def test_near_field_counts_against_kdtree():
    """Partner counts (real and image pairs within psi) by brute force equal
    those of an independent k-d tree search."""
    from scipy.spatial import cKDTree
    rng = np.random.default_rng(5)
    dims = (16, 12, 16)
    N = 300
    pos = np.stack([rng.uniform(0, 16, N), rng.uniform(0, 12, N), rng.uniform(0, 16, N)])
    p = _base_params(dims, (0, 1))
    _, counts = particles.near_field(pos, np.ones(N), np.zeros(N, int), p, p['fp_table'])
    psi = p['psi']
    # periodic in x, z via tiling; images as mirrored copies
    pts, ids = [], []
    for sx in (-16, 0, 16):
        for sz in (-16, 0, 16):
            for img in range(3):
                y = pos[1] if img == 0 else (-pos[1] if img == 1 else 24 - pos[1])
                pts.append(np.stack([pos[0] + sx, y, pos[2] + sz], 1)); ids.append(np.arange(N) + img * N)
    pts = np.concatenate(pts); ids = np.concatenate(ids)
    tree = cKDTree(pts)
    ref = np.zeros(N, int)
    for i in range(N):
        hits = tree.query_ball_point(pos[:, i], psi * (1 - 1e-12))
        ref[i] = sum(1 for h in hits if ids[h] != i)
    assert np.array_equal(counts, ref)


def test_lj_force_is_minus_gradient():
    """Eq. closerange: F^R = -xhat dU/dr for the truncated-shifted 12-6 LJ."""
    p = _base_params((16, 16, 16), (0, 0))
    p.update(lj_sigma=[[1.2]], lj_xi=[[0.8]], lj_rc=[[3.0]])
    p['fp_table'] = np.zeros_like(p['fp_table'])
    p['lB'] = 0.0
    U = lambda r: 4 * 0.8 * ((1.2 / r) ** 12 - (1.2 / r) ** 6) - 4 * 0.8 * ((1.2 / 3) ** 12 - (1.2 / 3) ** 6)
    for r in (1.1, 1.5, 2.5):
        pos = np.array([[5.0, 5.0 + r], [8.0, 8.0], [7.0, 7.0]])
        F, _ = particles.near_field(pos, np.zeros(2), np.zeros(2, int), p, p['fp_table'])
        h = 1e-6
        dU = (U(r + h) - U(r - h)) / (2 * h)
        assert abs(F[0, 1] - (-dU)) < 1e-6 * abs(dU) + 1e-9
        assert abs(F[0, 0] + F[0, 1]) < 1e-12


# ------------------------------------------------------------------ mobility
def test_channel_mobility_reduces_to_single_wall():
    """Eq. mob_analytic -> Eq. singlewall as L -> infinity; and a fit of
    Eq. fitfunction reproduces its own derivative."""
    y = np.linspace(0.8, 5, 20)
    for perp in (False, True):
        g = mobility.gamma_channel(y, 1e6, 1.0, perp)
        assert np.allclose(g, mobility.gamma_single(y, 1.0, perp), atol=1e-6)
    c = [1.0, -0.5, 0.6, 0.05, 0.3, -0.01, 0.9]
    g, dg = mobility.fit_gamma(y, c)
    h = 1e-6
    num = (mobility.fit_gamma(y + h, c)[0] - mobility.fit_gamma(y - h, c)[0]) / (2 * h)
    assert np.allclose(dg, num, atol=1e-8)


def test_dry_step_free_diffusion_special_case():
    """With Gamma = 1, no force and no walls in reach, Eq. ions3 reduces to
    x' = x + sqrt(2 D dt) W with W the Philox normals."""
    dims = (16, 32, 16)
    p = _base_params(dims, (0, 0))
    p['lB'] = 0.0
    p.update(gamma_coef=[[[[1, 0, 1, 0, 1, 0, 1]] * 2] * 2], D_tot=[0.7], D_wet=[0.0],
             dt=0.01, kT=1.0, seed=99, drift=True)
    pos = np.array([[3.0, 9.0], [12.0, 20.0], [5.0, 11.0]])
    inc = integrate.dry_increment(p, pos, [0, 0], np.zeros((3, 2)), step=5)
    W = philox.ion_normals(2, 5, 0, philox.TAG_DRY, 99)
    assert np.allclose(inc, np.sqrt(2 * 0.7 * 0.01) * W, atol=1e-15)


# ------------------------------------------------------------------ Stokes
def test_stokes_divergence_free_and_self_adjoint():
    rng = np.random.default_rng(6)
    Nx, Ny, Nz = 6, 8, 4
    f = [rng.normal(size=(Nz, Ny, Nx)), rng.normal(size=(Nz, Ny + 1, Nx)), rng.normal(size=(Nz, Ny, Nx))]
    g = [rng.normal(size=(Nz, Ny, Nx)), rng.normal(size=(Nz, Ny + 1, Nx)), rng.normal(size=(Nz, Ny, Nx))]
    for a in (f, g):
        a[1][:, 0, :] = 0; a[1][:, Ny, :] = 0
    u1 = stokes.solve(*f, eta=0.8)
    u2 = stokes.solve(*g, eta=0.8)
    assert np.abs(stokes.divergence(*u1[:3])).max() < 1e-12
    lhs = sum(np.sum(a * b) for a, b in zip(f, u2[:3]))
    rhs = sum(np.sum(a * b) for a, b in zip(u1[:3], g))
    assert abs(lhs - rhs) < 1e-11 * abs(lhs)


def test_stokes_poiseuille_second_order():
    """A uniform body force f_x gives plane Poiseuille flow f y (L - y) / (2 eta),
    reached at second order in the grid spacing."""
    errs = []
    for Ny in (8, 16):
        Nx = Nz = 4
        scale = 1.0 / Ny                    # refine the same channel
        fx = np.ones((Nz, Ny, Nx)) * scale ** 2
        u, v, w, pr = stokes.solve(fx, np.zeros((Nz, Ny + 1, Nx)), np.zeros((Nz, Ny, Nx)), 1.0)
        y = (np.arange(Ny) + 0.5) * scale
        exact = y * (1 - y) / 2.0
        errs.append(np.abs(u[0, :, 0] - exact).max())
        assert np.abs(v).max() < 1e-12 and np.abs(w).max() < 1e-12
    assert errs[0] < 1e-2 and 3.5 < errs[0] / errs[1] < 4.5


def test_stress_noise_fluctuation_dissipation():
    """Discrete FDT: the stochastic stress divergence D satisfies
    D D^T = L + Div^T Div exactly, L the no-slip viscous operator."""
    import scipy.sparse as sp
    Nx, Ny, Nz = 4, 4, 3
    shapes = [(Nz, Ny, Nx)] * 3 + [(Nz, Ny + 1, Nx), (Nz, Ny, Nx), (Nz, Ny + 1, Nx)]
    cols = []
    for c, shp in enumerate(shapes):
        for e in range(int(np.prod(shp))):
            Z = [np.zeros(s) for s in shapes]
            Z[c].flat[e] = 1.0
            if c < 3:
                Z[c] *= np.sqrt(2)
            if c in (3, 5):
                Z[c][:, 0, :] *= np.sqrt(2); Z[c][:, Ny, :] *= np.sqrt(2)
            dx, dy, dz = stokes.stress_divergence(*Z)
            cols.append(np.concatenate([dx.ravel(), dy[:, 1:Ny, :].ravel(), dz.ravel()]))
    D = np.array(cols).T
    Lu, Lv, Lw, Gx, Gy, Gz = stokes._ops((Nx, Ny, Nz))
    L = sp.block_diag([Lu, Lv, Lw]).toarray()
    G = sp.vstack([Gx, Gy, Gz]).toarray()
    assert np.abs(D @ D.T - (L + G @ G.T)).max() < 1e-13


def test_stress_noise_variances():
    """The Philox-drawn stress has variance 2 on the diagonal, 1 on interior
    edges and 2 on the wall edges of Zxy and Zyz (the sqrt 2 wall scaling)."""
    dims = (16, 6, 16)
    Z = stokes.stress_fields(dims, step=3, replica=0, seed=7)
    Zxx, Zyy, Zzz, Zxy, Zxz, Zyz = Z
    for a in (Zxx, Zyy, Zzz):
        assert abs(a.var() - 2.0) < 0.15
    for e in (Zxy, Zyz):
        assert abs(e[:, 1:-1, :].var() - 1.0) < 0.08
        assert abs(np.concatenate([e[:, 0, :], e[:, -1, :]]).var() - 2.0) < 0.3
    assert abs(Zxz.var() - 1.0) < 0.08
