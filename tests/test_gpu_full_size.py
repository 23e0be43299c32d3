"""The 256 x 128 x 256 channel with 400,000 ions (conducting bottom wall,
dielectric top wall, full wet step): checks at full size that the oracle can
make one sample at a time, or that hold at any size.

- FP64 path: Poisson residual of the oracle's assembled operator <= 1e-10
  relative (the operator applied once, no solve); MIXED: <= 1e-5.
- Near field on 64 sampled ions against the oracle's all-pairs loop with
  images: partner counts bit-exact, forces 1e-10 (FP64) / 1e-4 (MIXED).
- MIXED forces against FP64 forces on all ions: relative L2 <= 1e-4 (the
  stated single-precision target), and one full wet step from the same state
  (same Philox noise): displacements within 1e-4 relative plus one float ulp
  of the coordinates (the MIXED path stores positions in float).
- Stokes on the 128 x 64 x 128 and 256 x 128 x 256 grids under white-noise
  forcing: the GPU velocity and pressure in the oracle's MAC operator
  (Eq. disc_stokes, applied by stencils): momentum residual and divergence
  <= 1e-10 relative (FP64) / 2e-5 (MIXED: float storage of v and p).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from helpers import oracle_params, rel_l2, min_image_disp  # noqa: E402
import paper_2204_14167_gb300 as dg  # noqa: E402
from paper_2204_14167_gb300 import presets, synth  # noqa: E402
from oracle import poisson, particles  # noqa: E402


@pytest.fixture(scope="module")
def state():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.init()
    cfg, rec = presets.iceo_channel_256x128x256(dg.FP64)
    pos, q, sp = synth.ions(cfg.dims, rec["n_pos"], rec["n_neg"], rec["seed"], rec["ymargin"], rec["min_sep"])
    return cfg, rec, pos, q, sp


def _handle(cfg, prec):
    c, _ = presets.iceo_channel_256x128x256(prec)
    return dg.Discos(c), c


@pytest.mark.parametrize("prec", [dg.FP64, dg.MIXED])
def test_full_size_poisson_residual(state, prec):
    cfg, rec, pos, q, sp = state
    h, c = _handle(cfg, prec)
    dt = torch.float64 if prec == dg.FP64 else torch.float32
    x = torch.tensor(pos, dtype=dt, device="cuda").contiguous()
    qd = torch.tensor(q, dtype=dt, device="cuda")
    rho = h.spread_charge(x, qd)
    phi = h.solve_poisson(rho)
    r, b = poisson.residual(phi.double().cpu().numpy(), rho.double().cpu().numpy(), c.bc, c.lB, c.phi_b,
                            c.surf_charge)
    rel = np.linalg.norm(r) / np.linalg.norm(b)
    assert rel <= (1e-10 if prec == dg.FP64 else 1e-5)


@pytest.mark.parametrize("prec", [dg.FP64, dg.MIXED])
def test_full_size_near_field_sampled(state, prec):
    cfg, rec, pos, q, sp = state
    h, c = _handle(cfg, prec)
    dt = torch.float64 if prec == dg.FP64 else torch.float32
    x = torch.tensor(pos, dtype=dt, device="cuda").contiguous()
    qd = torch.tensor(q, dtype=dt, device="cuda")
    F, cnt = h.near_field(x, qd)
    p = oracle_params(c)
    targets = np.random.default_rng(5).choice(pos.shape[1], 64, replace=False)
    # the near-wall ions are the ones with image partners
    targets[:8] = np.argsort(pos[1])[:8]
    targets[8:16] = np.argsort(-pos[1])[:8]
    pair_dt = np.float64 if prec == dg.FP64 else np.float32
    xh = x.double().cpu().numpy()
    ref, ref_cnt = particles.near_field(xh, qd.double().cpu().numpy(), sp, p, p["fp_table"], pair_dtype=pair_dt,
                                        targets=targets)
    ref[1] += particles.wall_force(xh[:, targets], sp[targets], p)
    assert np.array_equal(cnt.cpu().numpy()[targets], ref_cnt)
    assert rel_l2(F.double().cpu().numpy()[:, targets], ref) < (1e-10 if prec == dg.FP64 else 1e-4)


def test_full_size_mixed_against_fp64(state):
    cfg, rec, pos, q, sp = state
    h64, c64 = _handle(cfg, dg.FP64)
    hm, cm = _handle(cfg, dg.MIXED)
    x64 = torch.tensor(pos, dtype=torch.float64, device="cuda").contiguous()
    q64 = torch.tensor(q, dtype=torch.float64, device="cuda")
    xm = x64.float().contiguous()
    qm = q64.float()
    xm64 = xm.double()          # both paths start from the same (single-precision) positions
    x64.copy_(xm64)
    F64 = h64.forces(x64, q64)
    Fm = hm.forces(xm, qm)
    assert rel_l2(Fm.double().cpu().numpy(), F64.cpu().numpy()) <= 1e-4
    h64.step(x64, q64, step0=11, nsteps=1)
    hm.step(xm, qm, step0=11, nsteps=1)
    torch.cuda.synchronize()
    x0 = xm64.cpu().numpy()
    d64 = min_image_disp(x64.cpu().numpy(), x0, c64.dims)
    dm = min_image_disp(xm.double().cpu().numpy(), x0, c64.dims)
    # the single-precision path stores x + dx in float: one ulp of the largest
    # coordinate (3e-5 at 256) is a floor on top of the 1e-4 relative target
    rms = lambda a: float(np.sqrt(np.mean(np.square(a))))
    ulp = float(np.spacing(np.float32(max(c64.dims))))
    assert rms(dm - d64) <= 1e-4 * rms(d64) + ulp


# Stokes at the two single-channel sizes the bench runs: white-noise forcing
# (the hardest case: every mode excited), the GPU velocity and pressure put
# into the oracle's MAC operator (stencils, no solve).
STOKES_SIZES = {"128x64x128": ("wet_channel_128x64x128", 1e-10, 2e-5),
                "256x128x256": ("iceo_channel_256x128x256", 1e-10, 2e-5)}


@pytest.mark.parametrize("prec", [dg.FP64, dg.MIXED])
@pytest.mark.parametrize("size", sorted(STOKES_SIZES))
def test_full_size_stokes_residual(prec, size):
    from helpers import mac_split, mac_join
    from oracle import stokes
    preset, tol64, tol32 = STOKES_SIZES[size]
    c, _ = getattr(presets, preset)(prec)
    h = dg.Discos(c)
    Nx, Ny, Nz = c.dims
    rng = np.random.default_rng(21)
    fx = rng.normal(size=(Nz, Ny, Nx)); fz = rng.normal(size=(Nz, Ny, Nx))
    fy = rng.normal(size=(Nz, Ny + 1, Nx)); fy[:, 0] = 0.0; fy[:, Ny] = 0.0
    dt = torch.float64 if prec == dg.FP64 else torch.float32
    fd = torch.tensor(mac_join(fx, fy, fz), dtype=dt, device="cuda")
    v, p = h.solve_stokes(fd.clone(), pressure=True)
    fh = mac_split(fd.double().cpu().numpy(), c.dims)
    u_, v_, w_ = mac_split(v.double().cpu().numpy(), c.dims)
    (rx, ry, rz), div = stokes.residual(u_, v_, w_, p.double().cpu().numpy().reshape(Nz, Ny, Nx), *fh, c.eta)
    nf = np.sqrt(sum(np.sum(a ** 2) for a in fh))
    rel = np.sqrt(np.sum(rx ** 2) + np.sum(ry ** 2) + np.sum(rz ** 2)) / nf
    # divergence relative to the velocity's own differences
    vscale = np.sqrt(sum(np.sum(a ** 2) for a in (u_, v_, w_)) / (3 * Nx * Ny * Nz))
    drel = float(np.sqrt(np.mean(div ** 2)) / vscale)
    tol = tol64 if prec == dg.FP64 else tol32
    assert rel <= tol, (rel, drel)
    assert drel <= tol, (rel, drel)
