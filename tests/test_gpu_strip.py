"""The metal strip in a dielectric bottom wall (Sec. IV.B, Fig. EOgeometry;
mixed wall conditions, Sec. II.B.1) through the C ABI, against the oracle:
the Poisson solve (transform solver plus the capacitance correction on the
strip cells) against CG on the assembled mixed operator, with a dielectric
or a conducting top wall; the total forces (strip images in spreading,
ghost cells and near field) and one wet step.  Tolerances as in
test_gpu_parity.py."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from helpers import oracle_params, rel_l2, min_image_disp  # noqa: E402
import paper_2204_14167_gb300 as dg  # noqa: E402
from paper_2204_14167_gb300 import presets, synth  # noqa: E402
from oracle import poisson, integrate  # noqa: E402

TOL = {dg.FP64: dict(phi=1e-10, force=1e-10, step=1e-9), dg.MIXED: dict(phi=1e-5, force=1e-4, step=1e-4)}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.init()


def _cfg(prec, top=dg.BC_NEUMANN, dims=(32, 16, 32), n=300):
    cfg, rec = presets.wet_channel_small(prec, *dims, n=n)
    cfg.bc = (dg.BC_NEUMANN, top)
    cfg.phi_b = (0.0, -0.2)
    cfg.surf_charge = (0.0, 0.0)
    cfg.strip = True
    cfg.strip_x = (9.3, 21.0)
    cfg.strip_phi = 0.15
    cfg.E_ext = (0.05, 0.0, 0.0)
    return cfg, rec


@pytest.mark.parametrize("prec", [dg.FP64, dg.MIXED])
@pytest.mark.parametrize("top", [dg.BC_NEUMANN, dg.BC_DIRICHLET])
def test_strip_poisson(prec, top):
    cfg, _ = _cfg(prec, top)
    Nx, Ny, Nz = cfg.dims
    rho = np.random.default_rng(8).normal(size=(Nz, Ny, Nx))
    h = dg.Discos(cfg)
    dt = torch.float64 if prec == dg.FP64 else torch.float32
    rd = torch.tensor(rho, dtype=dt, device="cuda")
    phi = h.solve_poisson(rd).double().cpu().numpy()
    mask = poisson.strip_columns(cfg.dims, *cfg.strip_x)
    pm = poisson.strip_potential(cfg.dims, cfg.strip_x[0], cfg.strip_x[1], cfg.strip_phi, cfg.E_ext[0])
    ref = poisson.solve_strip(rd.double().cpu().numpy(), cfg.lB, mask, pm, top, cfg.phi_b[1], cfg.surf_charge)
    assert rel_l2(phi, ref) < TOL[prec]["phi"]


@pytest.mark.parametrize("prec", [dg.FP64, dg.MIXED])
def test_strip_forces_and_wet_step(prec):
    cfg, rec = _cfg(prec)
    pos, q, sp = synth.ions(cfg.dims, rec["n_pos"], rec["n_neg"], rec["seed"], rec["ymargin"], rec["min_sep"])
    dt = torch.float64 if prec == dg.FP64 else torch.float32
    xd = torch.tensor(pos, dtype=dt, device="cuda").contiguous()
    qd = torch.tensor(q, dtype=dt, device="cuda")
    pos_h, q_h = xd.double().cpu().numpy(), qd.double().cpu().numpy()
    h = dg.Discos(cfg)
    F, cnt = h.forces(xd, qd, counts=True)
    p = oracle_params(cfg)
    pair_dt = np.float64 if prec == dg.FP64 else np.float32
    ref, ref_cnt, _ = integrate.forces(p, pos_h, q_h, sp, pair_dtype=pair_dt)
    assert np.array_equal(cnt.cpu().numpy(), ref_cnt)
    assert rel_l2(F.double().cpu().numpy(), ref) < TOL[prec]["force"]
    x0 = xd.clone()
    Fs = torch.empty_like(xd)
    h.step(xd, qd, step0=2, nsteps=1, F_out=Fs)
    torch.cuda.synchronize()
    new, Fr, _, _ = integrate.wet_step(p, pos_h, q_h, sp, 2, pair_dtype=pair_dt)
    assert rel_l2(Fs.double().cpu().numpy(), Fr) < TOL[prec]["force"]
    d_gpu = min_image_disp(xd.double().cpu().numpy(), x0.double().cpu().numpy(), cfg.dims)
    assert rel_l2(d_gpu, min_image_disp(new, pos_h, cfg.dims)) < TOL[prec]["step"]


def test_strip_rejections():
    cfg, _ = _cfg(dg.FP64)
    cfg.bc = (dg.BC_DIRICHLET, dg.BC_NEUMANN)
    with pytest.raises(dg.DiscosError):
        dg.Discos(cfg)
    cfg, _ = _cfg(dg.FP64)
    cfg.strip_x = (5.2, 5.4)              # no cell centre inside
    with pytest.raises(dg.DiscosError):
        dg.Discos(cfg)
    cfg, _ = _cfg(dg.MIXED)
    cfg.max_refine = 1
    with pytest.raises(dg.DiscosError):
        dg.Discos(cfg)
