"""Parity of the CUDA path (through the libdiscos C ABI) with the FP64 oracle.

Tolerances (relative L2 against the oracle):
  FP64 path:  grids and forces 1e-10 (transform + banded solve against CG
              rounding), integer outputs bit-exact;
  MIXED path: charge density 1e-6, potential 1e-5, forces, velocities and
              step displacements 1e-4 (the stated accuracy targets of the
              single-precision bulk with double wall-normal solves).
Sizes span several thread blocks and ragged tails: grids of 32 x 16 x 32 and
16 x 8 x 16 cells, ion counts that are not multiples of a warp.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from helpers import oracle_params, rel_l2, min_image_disp, mac_split, mac_join  # noqa: E402
import paper_2204_14167_gb300 as dg  # noqa: E402
from paper_2204_14167_gb300 import presets, synth  # noqa: E402
from oracle import gridops, poisson, particles, stokes, integrate  # noqa: E402

TOL = {dg.FP64: dict(grid=1e-10, phi=1e-10, force=1e-10, vel=1e-10, step=1e-9),
       dg.MIXED: dict(grid=1e-6, phi=1e-5, force=1e-4, vel=1e-4, step=1e-4)}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.init()


def _dtype(prec):
    return torch.float64 if prec == dg.FP64 else torch.float32


def _setup(cfg, rec, prec):
    cfg.precision = prec
    pos, q, sp = synth.ions(cfg.dims, rec["n_pos"], rec["n_neg"], rec["seed"], rec["ymargin"], rec["min_sep"])
    dt = _dtype(prec)
    xd = torch.tensor(pos, dtype=dt, device="cuda").contiguous()
    qd = torch.tensor(q, dtype=dt, device="cuda")
    # the oracle sees exactly the values the GPU holds
    pos_h = xd.double().cpu().numpy()
    q_h = qd.double().cpu().numpy()
    return xd, qd, pos_h, q_h, sp


def _small_dry(bc=(0, 0), kernel=dg.KERNEL_PESKIN6, n=301, Ny=16, phi_b=(0.0, 0.0), surf=(0.0, 0.0)):
    cfg, rec = presets.dry_channel_32()
    cfg.Nx, cfg.Ny, cfg.Nz = 32, Ny, 32
    cfg.bc = bc
    cfg.phi_b = phi_b
    cfg.surf_charge = surf
    cfg.kernel_es = kernel
    cfg.kernel_hy = kernel
    cfg.lB = 1.3
    cfg.lj_sigma, cfg.lj_rc = [[1.0]], [[2.0 ** (1 / 6)]]
    cfg.max_ions = n
    rec = dict(rec, n_pos=n // 2, n_neg=n - n // 2, min_sep=0.8, ymargin=0.05)
    return cfg, rec


PRECS = [dg.FP64, dg.MIXED]
# kernels: the 4- and 6-point widths run the unrolled kernels, the 5-point
# ES kernel the general-width ones
KERNELS = [(dg.KERNEL_PESKIN4, 4), (dg.KERNEL_PESKIN6, 6), (dg.KERNEL_ES, 5)]


def _with_kernel(cfg, kernel):
    kind, w = kernel
    cfg.kernel_es = cfg.kernel_hy = kind
    cfg.es_w = (w, w)
    return cfg
BCS = [(0, 0), (1, 1), (0, 1), (1, 0)]


# fx_pairs = 0: the bulk-staged persistent x transform
# fz_tile = 0: the TMA-tiled z transform (single precision only; the FP64 handle rejects it)
SHAPES = [(1, 32, 1), (4, 64, 4), (16, 256, 16), (32, 512, 2), (0, 32, 4), (0, 32, 16), (0, 32, 0), (4, 64, 0)]


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("shape", SHAPES)
def test_transform_shapes(prec, shape):
    """Every launch shape the transform autotuner may pick gives the same
    Poisson and Stokes solutions (32 x 16 x 32: 1..64 row pairs per x block
    or the staged x kernel, 1..16 columns per z block)."""
    rng = np.random.default_rng(13)
    cfg, rec = _small_dry((0, 1), phi_b=(0.3, -0.2), surf=(0.0, 0.01))
    cfg.precision = prec
    cfg.eta = 0.7
    cfg.wet = True
    h = dg.Discos(cfg)
    if shape[2] == 0 and prec == dg.FP64:
        with pytest.raises(dg.DiscosError):
            h.set_transform_shape(*shape)
        return
    h.set_transform_shape(*shape)
    Nx, Ny, Nz = cfg.dims
    rho = rng.normal(size=(Nz, Ny, Nx))
    rd = torch.tensor(rho, dtype=_dtype(prec), device="cuda")
    phi = h.solve_poisson(rd).double().cpu().numpy()
    ref = poisson.solve(rd.double().cpu().numpy(), cfg.bc, cfg.lB, cfg.phi_b, cfg.surf_charge)
    assert rel_l2(phi, ref) < TOL[prec]["phi"]
    f = torch.tensor(rng.normal(size=Nx * Nz * (3 * Ny + 1)), dtype=_dtype(prec), device="cuda")
    u, v, w = mac_split(f.cpu().numpy(), cfg.dims)
    v[:, 0, :] = 0.0
    v[:, -1, :] = 0.0
    f = torch.tensor(mac_join(u, v, w), dtype=_dtype(prec), device="cuda")
    vel = h.solve_stokes(f.clone()).double().cpu().numpy()
    fh = mac_split(f.double().cpu().numpy(), cfg.dims)
    ref = stokes.solve(fh[0], fh[1], fh[2], cfg.eta)[:3]
    assert rel_l2(vel, mac_join(*ref)) < TOL[prec]["vel"]


@pytest.mark.parametrize("prec", PRECS)
def test_unaligned_grids(prec):
    """Grids that start off a 16-byte boundary (a caller's offset view) take
    the per-row x transform and the lane-group spreading and interpolation
    kernels instead of the bulk-staged and vector-access ones, with the same
    results."""
    rng = np.random.default_rng(14)
    cfg, rec = _small_dry((0, 1), phi_b=(0.3, -0.2), surf=(0.0, 0.01))
    cfg.precision = prec
    h = dg.Discos(cfg)
    Nx, Ny, Nz = cfg.dims
    G = Nx * Ny * Nz
    rho = rng.normal(size=G)
    a = torch.tensor(rho, dtype=_dtype(prec), device="cuda")
    b = torch.zeros(G + 1, dtype=_dtype(prec), device="cuda")[1:]
    b.copy_(a)
    pa = h.solve_poisson(a).double().cpu().numpy().ravel()
    pb = h.solve_poisson(b, out=torch.zeros(G + 1, dtype=_dtype(prec), device="cuda")[1:]).double().cpu().numpy().ravel()
    ref = poisson.solve(rho.reshape(Nz, Ny, Nx), cfg.bc, cfg.lB, cfg.phi_b, cfg.surf_charge).ravel()
    assert rel_l2(pa, ref) < TOL[prec]["phi"]
    assert rel_l2(pb, ref) < TOL[prec]["phi"]
    xd, qd, pos, q, _ = _setup(cfg, rec, prec)
    ra = h.spread_charge(xd, qd).double().cpu().numpy().ravel()
    rb = h.spread_charge(xd, qd, out=torch.zeros(G + 1, dtype=_dtype(prec), device="cuda")[1:])
    assert rel_l2(rb.double().cpu().numpy().ravel(), ra) < TOL[prec]["grid"]
    ea = h.interpolate_efield(xd, torch.tensor(pa, dtype=_dtype(prec), device="cuda")).double().cpu().numpy()
    ub = torch.zeros(G + 1, dtype=_dtype(prec), device="cuda")[1:]
    ub.copy_(torch.tensor(pa, dtype=_dtype(prec), device="cuda"))
    eb = h.interpolate_efield(xd, ub).double().cpu().numpy()
    assert rel_l2(eb, ea) < TOL[prec]["force"]


@pytest.mark.parametrize("prec", PRECS)
def test_transform_tuner(prec):
    cfg, rec = _small_dry((0, 0))
    cfg.precision = prec
    h = dg.Discos(cfg)
    pp, th, tk, ms = h.tune_transforms()
    # 0: the bulk-staged x kernel / the TMA-tiled z kernel
    assert (pp == 0 or (1 <= pp and pp * cfg.Nx <= 2048)) and th % 32 == 0 and tk in (0, 1, 2, 4, 8, 16)
    assert min(ms) > 0
    xd, qd, pos, q, _ = _setup(cfg, rec, prec)
    rho = h.spread_charge(xd, qd)
    phi = h.solve_poisson(rho).double().cpu().numpy()
    ref = poisson.solve(rho.double().cpu().numpy(), cfg.bc, cfg.lB, cfg.phi_b, cfg.surf_charge)
    assert rel_l2(phi, ref) < TOL[prec]["phi"]
    with pytest.raises(dg.DiscosError):
        h.set_transform_shape(-1, 32, 1)
    with pytest.raises(dg.DiscosError):
        h.set_transform_shape(1, 33, 1)
    with pytest.raises(dg.DiscosError):
        h.set_transform_shape(1, 32, 3)


@pytest.mark.parametrize("bc", BCS)
def test_poisson_refinement(bc):
    """Mixed precision with double-precision residual refinement: the
    residual history falls, and the refined potential is closer to the
    oracle than the single-precision solve, to within the float rounding of
    phi itself."""
    rng = np.random.default_rng(12)
    cfg, rec = _small_dry(bc, phi_b=(0.3, -0.2), surf=(0.004, 0.002) if bc == (1, 1) else (0.01, -0.02))
    Nx, Ny, Nz = cfg.dims
    rho = rng.normal(size=(Nz, Ny, Nx))
    if bc == (1, 1):
        rho -= rho.mean() - (-(cfg.surf_charge[0] + cfg.surf_charge[1]) * Nx * Nz) / rho.size
    cfg.precision = dg.MIXED
    h0 = dg.Discos(cfg)
    cfg.max_refine = 2
    h2 = dg.Discos(cfg)
    rd = torch.tensor(rho, dtype=torch.float32, device="cuda")
    ref = poisson.solve(rd.double().cpu().numpy(), bc, cfg.lB, cfg.phi_b, cfg.surf_charge)
    e0 = rel_l2(h0.solve_poisson(rd).double().cpu().numpy(), ref)
    e2 = rel_l2(h2.solve_poisson(rd).double().cpu().numpy(), ref)
    hist = h2.refine_history()
    assert len(hist) == 3 and hist[1] < 0.5 * hist[0] and hist[2] <= hist[1] * 1.5
    assert e2 <= max(0.5 * e0, 3e-7)
    assert h0.refine_history() == []


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("bc", BCS)
@pytest.mark.parametrize("kernel", KERNELS)
def test_spread_charge(prec, bc, kernel):
    cfg, rec = _small_dry(bc)
    _with_kernel(cfg, kernel)
    xd, qd, pos, q, _ = _setup(cfg, rec, prec)
    h = dg.Discos(cfg)
    rho = h.spread_charge(xd, qd).double().cpu().numpy()
    ref = gridops.spread_charge(oracle_params(cfg)["kernel_es"], pos, q, cfg.dims, bc)
    assert rel_l2(rho, ref) < TOL[prec]["grid"]


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("bc", BCS)
def test_poisson(prec, bc):
    rng = np.random.default_rng(11)
    cfg, rec = _small_dry(bc, phi_b=(0.3, -0.2), surf=(0.004, 0.002) if bc == (1, 1) else (0.01, -0.02))
    Nx, Ny, Nz = cfg.dims
    rho = rng.normal(size=(Nz, Ny, Nx))
    if bc == (1, 1):
        rho -= rho.mean() - (-(cfg.surf_charge[0] + cfg.surf_charge[1]) * Nx * Nz) / rho.size
    cfg.precision = prec
    h = dg.Discos(cfg)
    rd = torch.tensor(rho, dtype=_dtype(prec), device="cuda")
    rho_h = rd.double().cpu().numpy()
    phi = h.solve_poisson(rd).double().cpu().numpy()
    ref = poisson.solve(rho_h, bc, cfg.lB, cfg.phi_b, cfg.surf_charge)
    assert rel_l2(phi, ref) < TOL[prec]["phi"]


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("bc", BCS)
@pytest.mark.parametrize("kernel", KERNELS)
def test_efield_interpolation(prec, bc, kernel):
    cfg, rec = _small_dry(bc, phi_b=(0.25, -0.5), surf=(0.01, -0.02))
    _with_kernel(cfg, kernel)
    xd, qd, pos, q, _ = _setup(cfg, rec, prec)
    rng = np.random.default_rng(12)
    Nx, Ny, Nz = cfg.dims
    phi = rng.normal(size=(Nz, Ny, Nx))
    h = dg.Discos(cfg)
    pd = torch.tensor(phi, dtype=_dtype(prec), device="cuda")
    E = h.interpolate_efield(xd, pd).double().cpu().numpy()
    p = oracle_params(cfg)
    slopes = poisson.wall_slopes(bc, cfg.surf_charge, cfg.lB)
    ref = gridops.efield_at_ions(p["kernel_es"], pos, pd.double().cpu().numpy(), bc, cfg.phi_b, slopes)
    assert rel_l2(E, ref) < TOL[prec]["force"]


@pytest.mark.parametrize("prec", PRECS)
def test_cell_list_bit_exact(prec):
    cfg, rec = _small_dry((0, 1), n=517)
    cfg.psi = 4.0
    xd, qd, pos, q, _ = _setup(cfg, rec, prec)
    h = dg.Discos(cfg)
    start, perm = h.cell_list(xd)
    k = int(np.ceil(max(cfg.psi, max(max(r) for r in cfg.lj_rc))))
    cid, ref_start, ref_perm = particles.cell_list(pos, cfg.dims, k)
    assert np.array_equal(start.cpu().numpy(), ref_start)
    assert np.array_equal(perm.cpu().numpy(), ref_perm)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("bc", BCS)
def test_near_field(prec, bc):
    cfg, rec = _small_dry(bc, n=419)
    xd, qd, pos, q, sp = _setup(cfg, rec, prec)
    h = dg.Discos(cfg)
    F, cnt = h.near_field(xd, qd)
    p = oracle_params(cfg)
    pair_dt = np.float64 if prec == dg.FP64 else np.float32
    ref, ref_cnt = particles.near_field(pos, q, sp, p, p["fp_table"], pair_dtype=pair_dt)
    ref[1] += particles.wall_force(pos, sp, p)
    assert np.array_equal(cnt.cpu().numpy(), ref_cnt)
    assert rel_l2(F.double().cpu().numpy(), ref) < TOL[prec]["force"]


@pytest.mark.parametrize("prec", PRECS)
def test_near_field_periodic_images_of_positions(prec):
    """x and z are periodic: positions handed in outside [0, L) (shifted by
    +-L) give the near field of their images inside the box.  Coordinates on
    a 1/1024 lattice make every shift exact in both precisions, so the
    partner counts stay bit-exact against the oracle on the wrapped
    positions."""
    cfg, rec = _small_dry((0, 1), n=419)
    xd, qd, pos, q, sp = _setup(cfg, rec, prec)
    pos = np.round(pos * 1024.0) / 1024.0
    pos[1] = np.clip(pos[1], 1.0 / 1024.0, cfg.Ny - 1.0 / 1024.0)
    rng = np.random.default_rng(3)
    shifted = pos.copy()
    for ax, L in ((0, cfg.Nx), (2, cfg.Nz)):
        shifted[ax] += L * rng.integers(-1, 2, size=pos.shape[1])
    h = dg.Discos(cfg)
    xs = torch.tensor(shifted, dtype=_dtype(prec), device="cuda").contiguous()
    F, cnt = h.near_field(xs, qd)
    p = oracle_params(cfg)
    pair_dt = np.float64 if prec == dg.FP64 else np.float32
    ref, ref_cnt = particles.near_field(pos, q, sp, p, p["fp_table"], pair_dtype=pair_dt)
    ref[1] += particles.wall_force(pos, sp, p)
    assert np.array_equal(cnt.cpu().numpy(), ref_cnt)
    assert rel_l2(F.double().cpu().numpy(), ref) < TOL[prec]["force"]
    start, perm = h.cell_list(xs)
    k = int(np.ceil(max(cfg.psi, max(max(r) for r in cfg.lj_rc))))
    _, ref_start, ref_perm = particles.cell_list(pos, cfg.dims, k)
    assert np.array_equal(start.cpu().numpy(), ref_start) and np.array_equal(perm.cpu().numpy(), ref_perm)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("bc", [(0, 0), (1, 1), (0, 1)])
def test_total_forces(prec, bc):
    cfg, rec = _small_dry(bc, n=300, phi_b=(0.2, -0.1))
    cfg.E_ext = (0.05, 0.0, -0.02)
    xd, qd, pos, q, sp = _setup(cfg, rec, prec)
    if bc == (1, 1):
        assert abs(q.sum()) < 1e-12
    h = dg.Discos(cfg)
    F, cnt = h.forces(xd, qd, counts=True)
    p = oracle_params(cfg)
    pair_dt = np.float64 if prec == dg.FP64 else np.float32
    ref, ref_cnt, _ = integrate.forces(p, pos, q, sp, pair_dtype=pair_dt)
    assert np.array_equal(cnt.cpu().numpy(), ref_cnt)
    assert rel_l2(F.double().cpu().numpy(), ref) < TOL[prec]["force"]


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("kernel", KERNELS)
def test_spread_force(prec, kernel):
    cfg, rec = _small_dry((0, 0), kernel=dg.KERNEL_PESKIN4, n=205)
    _with_kernel(cfg, kernel)
    xd, qd, pos, q, sp = _setup(cfg, rec, prec)
    rng = np.random.default_rng(13)
    Fh = rng.normal(size=(3, pos.shape[1]))
    Fd = torch.tensor(Fh, dtype=_dtype(prec), device="cuda")
    h = dg.Discos(cfg)
    f = h.spread_force(xd, Fd).double().cpu().numpy()
    p = oracle_params(cfg)
    ref = mac_join(*gridops.spread_force(p["kernel_hy"], pos, Fd.double().cpu().numpy(), cfg.dims))
    assert rel_l2(f, ref) < TOL[prec]["grid"]


# thin, tall boxes reach every rows-per-lane variant of the wall-normal
# solves (Ny <= 32, 64, 128, 256)
STOKES_DIMS = [(16, 8, 16), (32, 30, 16), (16, 64, 16), (16, 128, 16), (16, 160, 16)]


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("dims", STOKES_DIMS)
def test_stokes(prec, dims):
    cfg, rec = _small_dry((0, 0), kernel=dg.KERNEL_PESKIN4)
    cfg.Nx, cfg.Ny, cfg.Nz = dims
    cfg.eta = 0.7
    cfg.wet = True
    cfg.precision = prec
    rng = np.random.default_rng(14)
    Nx, Ny, Nz = cfg.dims
    fx = rng.normal(size=(Nz, Ny, Nx)); fz = rng.normal(size=(Nz, Ny, Nx))
    fy = rng.normal(size=(Nz, Ny + 1, Nx)); fy[:, 0] = 0; fy[:, Ny] = 0
    fd = torch.tensor(mac_join(fx, fy, fz), dtype=_dtype(prec), device="cuda")
    h = dg.Discos(cfg)
    v, pr = h.solve_stokes(fd, pressure=True)
    fh = mac_split(fd.double().cpu().numpy(), cfg.dims)
    u, vv, w, p = stokes.solve(fh[0], fh[1], fh[2], cfg.eta)
    assert rel_l2(v.double().cpu().numpy(), mac_join(u, vv, w)) < TOL[prec]["vel"]
    assert rel_l2(pr.double().cpu().numpy(), p) < TOL[prec]["vel"]


def test_stokes_refinement():
    """Mixed precision with double-precision residual refinement of the MAC
    system (Eq. disc_stokes): the residual, measured with the velocity and
    pressure carried in double, falls by orders of magnitude per sweep, below
    the rounding of a single-precision velocity; the rounded result is at
    least as close to the oracle as the plain single-precision solve, to
    within that rounding."""
    cfg, rec = _small_dry((0, 0), kernel=dg.KERNEL_PESKIN4)
    cfg.Nx, cfg.Ny, cfg.Nz = 32, 16, 32
    cfg.eta = 0.7
    cfg.wet = True
    cfg.precision = dg.MIXED
    rng = np.random.default_rng(24)
    Nx, Ny, Nz = cfg.dims
    fx = rng.normal(size=(Nz, Ny, Nx)); fz = rng.normal(size=(Nz, Ny, Nx))
    fy = rng.normal(size=(Nz, Ny + 1, Nx)); fy[:, 0] = 0; fy[:, Ny] = 0
    fd = torch.tensor(mac_join(fx, fy, fz), dtype=torch.float32, device="cuda")
    h0 = dg.Discos(cfg)
    cfg.max_refine = 2
    h2 = dg.Discos(cfg)
    v0, p0 = h0.solve_stokes(fd.clone(), pressure=True)
    v2, p2 = h2.solve_stokes(fd.clone(), pressure=True)
    hist = h2.refine_history_stokes()
    assert h0.refine_history_stokes() == []
    assert len(hist) == 3 and hist[1] < 1e-2 * hist[0] and hist[2] <= 1.5 * hist[1] and hist[2] < 1e-8, hist
    fh = mac_split(fd.double().cpu().numpy(), cfg.dims)
    u, vv, w, p = stokes.solve(fh[0], fh[1], fh[2], cfg.eta)
    ref = mac_join(u, vv, w)
    e0 = rel_l2(v0.double().cpu().numpy(), ref)
    e2 = rel_l2(v2.double().cpu().numpy(), ref)
    assert e2 <= max(e0, 1e-7), (e0, e2)
    assert rel_l2(p2.double().cpu().numpy(), p) <= max(rel_l2(p0.double().cpu().numpy(), p), 1e-7)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("kernel", KERNELS)
def test_velocity_interpolation(prec, kernel):
    cfg, rec = _small_dry((0, 0), kernel=dg.KERNEL_PESKIN4, n=203)
    _with_kernel(cfg, kernel)
    xd, qd, pos, q, sp = _setup(cfg, rec, prec)
    rng = np.random.default_rng(15)
    Nx, Ny, Nz = cfg.dims
    u = rng.normal(size=(Nz, Ny, Nx)); w = rng.normal(size=(Nz, Ny, Nx))
    v = rng.normal(size=(Nz, Ny + 1, Nx)); v[:, 0] = 0; v[:, Ny] = 0
    vd = torch.tensor(mac_join(u, v, w), dtype=_dtype(prec), device="cuda")
    h = dg.Discos(cfg)
    V = h.interpolate_velocity(xd, vd).double().cpu().numpy()
    p = oracle_params(cfg)
    uh = mac_split(vd.double().cpu().numpy(), cfg.dims)
    ref = gridops.interp_velocity(p["kernel_hy"], pos, *uh)
    assert rel_l2(V, ref) < TOL[prec]["vel"]


@pytest.mark.parametrize("prec", PRECS)
def test_dry_step_full_size(prec):
    """32^3 Dirichlet channel, 256 ions, l_B = 7, 6-point kernel: forces and one
    Euler-Maruyama step from the same state."""
    cfg, rec = presets.dry_channel_32(prec)
    xd, qd, pos, q, sp = _setup(cfg, rec, prec)
    h = dg.Discos(cfg)
    F_gpu = torch.empty_like(xd)
    x0 = xd.clone()
    h.step(xd, qd, step0=7, nsteps=1, F_out=F_gpu)
    torch.cuda.synchronize()
    p = oracle_params(cfg)
    pair_dt = np.float64 if prec == dg.FP64 else np.float32
    new, F, cnt = integrate.dry_step(p, pos, q, sp, 7, pair_dtype=pair_dt)
    assert rel_l2(F_gpu.double().cpu().numpy(), F) < TOL[prec]["force"]
    d_gpu = min_image_disp(xd.double().cpu().numpy(), x0.double().cpu().numpy(), cfg.dims)
    d_ref = min_image_disp(new, pos, cfg.dims)
    assert rel_l2(d_gpu, d_ref) < TOL[prec]["step"]


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("drift", [True, False])
def test_wet_step(prec, drift):
    """Neumann channel 32 x 16 x 32, 300 ions, fluctuating Stokes, midpoint:
    forces and displacements of one step from the same state."""
    cfg, rec = presets.wet_channel_small(prec)
    cfg.drift = drift
    xd, qd, pos, q, sp = _setup(cfg, rec, prec)
    h = dg.Discos(cfg)
    F_gpu = torch.empty_like(xd)
    x0 = xd.clone()
    h.step(xd, qd, step0=3, nsteps=1, F_out=F_gpu)
    torch.cuda.synchronize()
    p = oracle_params(cfg)
    pair_dt = np.float64 if prec == dg.FP64 else np.float32
    new, F, cnt, parts = integrate.wet_step(p, pos, q, sp, 3, pair_dtype=pair_dt)
    assert rel_l2(F_gpu.double().cpu().numpy(), F) < TOL[prec]["force"]
    d_gpu = min_image_disp(xd.double().cpu().numpy(), x0.double().cpu().numpy(), cfg.dims)
    d_ref = min_image_disp(new, pos, cfg.dims)
    assert rel_l2(d_gpu, d_ref) < TOL[prec]["step"]


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("Ny", [64, 128])
def test_wet_step_tall(prec, Ny):
    """The wet step on thin, tall channels (16 x Ny x 16, 200 ions): the
    wall-normal solves with 2 and 4 rows per lane, as on the 128 x 64 x 128
    and 256 x 128 x 256 channels, against the oracle's step."""
    cfg, rec = presets.wet_channel_small(prec, Nx=16, Ny=Ny, Nz=16, n=200)
    xd, qd, pos, q, sp = _setup(cfg, rec, prec)
    h = dg.Discos(cfg)
    F_gpu = torch.empty_like(xd)
    x0 = xd.clone()
    h.step(xd, qd, step0=5, nsteps=1, F_out=F_gpu)
    torch.cuda.synchronize()
    p = oracle_params(cfg)
    pair_dt = np.float64 if prec == dg.FP64 else np.float32
    new, F, cnt, parts = integrate.wet_step(p, pos, q, sp, 5, pair_dtype=pair_dt)
    assert rel_l2(F_gpu.double().cpu().numpy(), F) < TOL[prec]["force"]
    d_gpu = min_image_disp(xd.double().cpu().numpy(), x0.double().cpu().numpy(), cfg.dims)
    d_ref = min_image_disp(new, pos, cfg.dims)
    assert rel_l2(d_gpu, d_ref) < TOL[prec]["step"]


def test_invalid_arguments_rejected():
    cfg, rec = _small_dry()
    cfg.Nx = 48
    with pytest.raises(dg.DiscosError):
        dg.Discos(cfg)
    cfg, rec = _small_dry()
    h = dg.Discos(cfg)
    x = torch.zeros((3, cfg.max_ions + 1), dtype=torch.float64, device="cuda")
    with pytest.raises(dg.DiscosError):
        h.spread_charge(x, torch.zeros(cfg.max_ions + 1, dtype=torch.float64, device="cuda"))
