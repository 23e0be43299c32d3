"""Double-precision run diagnostics (discos_diagnostics) and the device fault
word (discos_fault, DISCOS_ERR_DEVICE_FAULT).

- sum q exact; dV sum rho equal to sum q for Neumann walls (like-signed images
  keep the kernel's partition of unity); sum F equal to the sum of the
  returned forces.
- A non-finite position sets bit 0 of the fault word during the step that
  moves it; the next discos_step refuses to run (status 5) until the word is
  cleared.  The kernels keep their indexing in bounds for such positions.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

import paper_2204_14167_gb300 as dg  # noqa: E402
from paper_2204_14167_gb300 import presets, synth  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.init()


def _setup(prec, bc=(1, 1), n=301):
    cfg, rec = presets.dry_channel_32(prec)
    cfg.Nx, cfg.Ny, cfg.Nz = 32, 16, 32
    cfg.bc = bc
    cfg.lB = 1.3
    cfg.lj_sigma, cfg.lj_rc = [[1.0]], [[2.0 ** (1 / 6)]]
    cfg.max_ions = n
    pos, q, _ = synth.ions(cfg.dims, n // 2, n - n // 2, 7, 1.0, 0.8)
    dt = torch.float64 if prec == dg.FP64 else torch.float32
    return cfg, torch.tensor(pos, dtype=dt, device="cuda").contiguous(), torch.tensor(q, dtype=dt, device="cuda")


@pytest.mark.parametrize("prec", [dg.FP64, dg.MIXED])
def test_diagnostics_sums(prec):
    cfg, x, q = _setup(prec)
    h = dg.Discos(cfg)
    F = h.forces(x, q)
    d = h.diagnostics(x, q, F)
    qs = float(q.double().sum())
    assert d["sum_q"] == qs
    tol = 1e-12 if prec == dg.FP64 else 1e-5
    assert abs(d["sum_rho"] - qs) <= tol * float(q.abs().sum())
    Fs = F.double().sum(dim=1).cpu().numpy()
    np.testing.assert_allclose(d["sum_F"], Fs, rtol=1e-9, atol=1e-9 * float(F.double().abs().sum()))
    assert d["nonfinite"] == 0 and d["escaped"] == 0


@pytest.mark.parametrize("prec", [dg.FP64, dg.MIXED])
def test_device_fault_word(prec):
    # the 32^3 Dirichlet channel with 256 ions at least 0.9 sigma apart, whose
    # steps keep every ion inside the channel
    cfg, rec = presets.dry_channel_32(prec)
    pos, qh, _ = synth.ions(cfg.dims, rec["n_pos"], rec["n_neg"], rec["seed"], rec["ymargin"], rec["min_sep"])
    dt = torch.float64 if prec == dg.FP64 else torch.float32
    x = torch.tensor(pos, dtype=dt, device="cuda").contiguous()
    q = torch.tensor(qh, dtype=dt, device="cuda")
    h = dg.Discos(cfg)
    h.step(x, q, step0=0, nsteps=1)
    assert h.fault(sync=True) == 0
    x0 = x.clone()
    x[:, 5] = float("nan")
    h.step(x, q, step0=1, nsteps=1)
    torch.cuda.synchronize()
    assert h.fault(sync=True) & 1
    assert h.diagnostics(x, q, with_rho=False)["nonfinite"] >= 1
    with pytest.raises(dg.DiscosError) as ei:
        h.step(x, q, step0=2, nsteps=1)
    assert ei.value.status == 5   # DISCOS_ERR_DEVICE_FAULT
    x.copy_(x0)       # the non-finite charge density has spread to every ion
    assert h.fault(sync=True, clear=True) & 1
    assert h.fault(sync=True) == 0
    h.step(x, q, step0=3, nsteps=1)
    torch.cuda.synchronize()
    assert h.fault(sync=True) == 0
