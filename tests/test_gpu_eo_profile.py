"""The electro-osmotic profile of Eq. fluidvel1 (Sec. IV.A.1) through the C
ABI: the staggered Stokes solve of the Debye-Hueckel charge density's body
force (see test_oracle_eo_profile.py for the reading of Eq. PhiWalls)
against the closed form, at the discretisation error of the oracle's solve,
and against the oracle's solve itself."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from helpers import rel_l2, mac_join  # noqa: E402
import paper_2204_14167_gb300 as dg  # noqa: E402
from paper_2204_14167_gb300 import presets  # noqa: E402
from oracle import stokes  # noqa: E402
from test_oracle_eo_profile import eo_force_and_profile  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.init()


@pytest.mark.parametrize("prec", [dg.FP64, dg.MIXED])
def test_eo_profile(prec):
    Nx, Ny, Nz = 16, 64, 16
    cfg, _ = presets.wet_channel_small(prec, Nx, Ny, Nz, n=1)
    eta = cfg.eta
    fxy, v_theory = eo_force_and_profile(Ny, Ny / 8.0, 0.08, 0.3, 0.05, eta)
    fx = np.broadcast_to(fxy[None, :, None], (Nz, Ny, Nx)).copy()
    fy = np.zeros((Nz, Ny + 1, Nx))
    fz = np.zeros((Nz, Ny, Nx))
    dt = torch.float64 if prec == dg.FP64 else torch.float32
    h = dg.Discos(cfg)
    vel = h.solve_stokes(torch.tensor(mac_join(fx, fy, fz), dtype=dt, device="cuda")).double().cpu().numpy()
    G = Nx * Ny * Nz
    u = vel[:G].reshape(Nz, Ny, Nx)
    ref = stokes.solve(fx, fy, fz, eta)[0]
    assert rel_l2(u, ref) < (1e-10 if prec == dg.FP64 else 1e-4)
    prof = u.mean(axis=(0, 2))
    # the oracle's own discretisation error at this spacing is 2e-3 (max, relative)
    assert np.abs(prof - v_theory).max() / np.abs(v_theory).max() < 3e-3
    assert np.abs(vel[G:]).max() < 1e-6 * np.abs(prof).max()
