"""Slip walls (zero normal velocity and zero shear stress; like tangential
images) through the C ABI against the oracle: the Stokes solve (per-mode
factors with the slip rows), force spreading and velocity interpolation with
the slip images and ghosts, the stochastic stress without wall-edge shear,
and one wet step.  Tolerances as in test_gpu_parity.py."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from helpers import oracle_params, rel_l2, min_image_disp, mac_split, mac_join  # noqa: E402
import paper_2204_14167_gb300 as dg  # noqa: E402
from paper_2204_14167_gb300 import presets, synth  # noqa: E402
from oracle import gridops, stokes, integrate  # noqa: E402

TOL = {dg.FP64: dict(grid=1e-10, vel=1e-10, force=1e-10, step=1e-9),
       dg.MIXED: dict(grid=1e-6, vel=1e-4, force=1e-4, step=1e-4)}
SLIPS = [(1, 0), (0, 1)]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.init()


def _cfg(prec, slip, dims=(32, 16, 32), n=300):
    cfg, rec = presets.wet_channel_small(prec, *dims, n=n)
    cfg.bc_hy = slip
    return cfg, rec


@pytest.mark.parametrize("prec", [dg.FP64, dg.MIXED])
@pytest.mark.parametrize("slip", SLIPS)
@pytest.mark.parametrize("dims", [(32, 16, 32), (16, 64, 16)])
def test_slip_stokes(prec, slip, dims):
    cfg, _ = _cfg(prec, slip, dims)
    cfg.eta = 0.7
    Nx, Ny, Nz = dims
    rng = np.random.default_rng(31)
    fx = rng.normal(size=(Nz, Ny, Nx)); fz = rng.normal(size=(Nz, Ny, Nx))
    fy = rng.normal(size=(Nz, Ny + 1, Nx)); fy[:, 0] = 0; fy[:, Ny] = 0
    dt = torch.float64 if prec == dg.FP64 else torch.float32
    fd = torch.tensor(mac_join(fx, fy, fz), dtype=dt, device="cuda")
    h = dg.Discos(cfg)
    v, pr = h.solve_stokes(fd.clone(), pressure=True)
    fh = mac_split(fd.double().cpu().numpy(), cfg.dims)
    u, vv, w, p = stokes.solve(*fh, cfg.eta, slip=tuple(bool(s) for s in slip))
    assert rel_l2(v.double().cpu().numpy(), mac_join(u, vv, w)) < TOL[prec]["vel"]
    assert rel_l2(pr.double().cpu().numpy(), p) < TOL[prec]["vel"]


@pytest.mark.parametrize("prec", [dg.FP64, dg.MIXED])
@pytest.mark.parametrize("slip", SLIPS)
def test_slip_spread_and_interpolation(prec, slip):
    cfg, rec = _cfg(prec, slip, n=211)
    rec = dict(rec, ymargin=0.05)
    pos, q, sp = synth.ions(cfg.dims, rec["n_pos"], rec["n_neg"], rec["seed"], rec["ymargin"], rec["min_sep"])
    dt = torch.float64 if prec == dg.FP64 else torch.float32
    xd = torch.tensor(pos, dtype=dt, device="cuda").contiguous()
    pos_h = xd.double().cpu().numpy()
    rng = np.random.default_rng(32)
    Fd = torch.tensor(rng.normal(size=(3, pos.shape[1])), dtype=dt, device="cuda")
    h = dg.Discos(cfg)
    p = oracle_params(cfg)
    sl = tuple(bool(s) for s in slip)
    f = h.spread_force(xd, Fd).double().cpu().numpy()
    ref = mac_join(*gridops.spread_force(p["kernel_hy"], pos_h, Fd.double().cpu().numpy(), cfg.dims, sl))
    assert rel_l2(f, ref) < TOL[prec]["grid"]
    Nx, Ny, Nz = cfg.dims
    u = rng.normal(size=(Nz, Ny, Nx)); w = rng.normal(size=(Nz, Ny, Nx))
    v = rng.normal(size=(Nz, Ny + 1, Nx)); v[:, 0] = 0; v[:, Ny] = 0
    vd = torch.tensor(mac_join(u, v, w), dtype=dt, device="cuda")
    V = h.interpolate_velocity(xd, vd).double().cpu().numpy()
    refV = gridops.interp_velocity(p["kernel_hy"], pos_h, *mac_split(vd.double().cpu().numpy(), cfg.dims), sl)
    assert rel_l2(V, refV) < TOL[prec]["vel"]


@pytest.mark.parametrize("prec", [dg.FP64, dg.MIXED])
@pytest.mark.parametrize("slip", SLIPS)
def test_slip_wet_step(prec, slip):
    cfg, rec = _cfg(prec, slip)
    pos, q, sp = synth.ions(cfg.dims, rec["n_pos"], rec["n_neg"], rec["seed"], rec["ymargin"], rec["min_sep"])
    dt = torch.float64 if prec == dg.FP64 else torch.float32
    xd = torch.tensor(pos, dtype=dt, device="cuda").contiguous()
    qd = torch.tensor(q, dtype=dt, device="cuda")
    pos_h, q_h = xd.double().cpu().numpy(), qd.double().cpu().numpy()
    h = dg.Discos(cfg)
    x0 = xd.clone()
    Fs = torch.empty_like(xd)
    h.step(xd, qd, step0=4, nsteps=1, F_out=Fs)
    torch.cuda.synchronize()
    p = oracle_params(cfg)
    pair_dt = np.float64 if prec == dg.FP64 else np.float32
    new, Fr, _, _ = integrate.wet_step(p, pos_h, q_h, sp, 4, pair_dtype=pair_dt)
    assert rel_l2(Fs.double().cpu().numpy(), Fr) < TOL[prec]["force"]
    d_gpu = min_image_disp(xd.double().cpu().numpy(), x0.double().cpu().numpy(), cfg.dims)
    assert rel_l2(d_gpu, min_image_disp(new, pos_h, cfg.dims)) < TOL[prec]["step"]


def test_two_slip_walls_rejected():
    cfg, _ = _cfg(dg.FP64, (1, 1))
    with pytest.raises(dg.DiscosError):
        dg.Discos(cfg)
