"""The differentiable energy through the C ABI (discos_energy,
discos_energy_backward) and torch.autograd, against the FP64 oracle.

- U against oracle.energy: FP64 1e-10 relative, MIXED 1e-5.
- dU/d(x, q, phi_b) against FP64 central differences of oracle.energy
  (h = 1e-4) on a 32-ion subset: FP64 1e-6 relative L2, MIXED 1e-4.
- At the 64^3, 4096-ion size: U against the oracle, and two properties that
  hold at any size: sum_i q_i dU/dq_i = 2U - phi_b . dU/dphi_b (U is
  quadratic in q and linear in phi_b, the lift being linear in phi_b), and
  -dU/dx against the force q E^P of Eq. efieldop within 5e-2 (the two differ
  by discretisation error only).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from helpers import oracle_params, rel_l2  # noqa: E402
import paper_2204_14167_gb300 as dg  # noqa: E402
from paper_2204_14167_gb300 import presets, synth  # noqa: E402
from paper_2204_14167_gb300.autograd import energy as denergy  # noqa: E402
from oracle import energy as oenergy  # noqa: E402

TOL_U = {dg.FP64: 1e-10, dg.MIXED: 1e-5}
TOL_G = {dg.FP64: 1e-6, dg.MIXED: 1e-4}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.init()


def _small(prec, bc=(0, 0), phi_b=(0.5, -0.5), n=301, dims=(32, 16, 16)):
    cfg, rec = presets.energy_channel_64(prec)
    cfg.Nx, cfg.Ny, cfg.Nz = dims
    cfg.bc = bc
    cfg.phi_b = phi_b
    cfg.surf_charge = (0.0, 0.0) if bc == (0, 0) else (0.01, -0.02)
    cfg.max_ions = n
    rec = dict(rec, n_pos=n // 2, n_neg=n - n // 2)
    return cfg, rec


def _ions(cfg, rec):
    dt = torch.float64 if cfg.precision == dg.FP64 else torch.float32
    pos, q, _ = synth.ions(cfg.dims, rec["n_pos"], rec["n_neg"], rec["seed"], rec["ymargin"], rec["min_sep"])
    xd = torch.tensor(pos, dtype=dt, device="cuda").contiguous()
    qd = torch.tensor(q, dtype=dt, device="cuda")
    return xd, qd, xd.double().cpu().numpy(), qd.double().cpu().numpy()


def _fd_grads(p, pos, q, phi_b, ions, h=1e-4):
    gx = np.zeros((3, len(ions)))
    gq = np.zeros(len(ions))
    for k, i in enumerate(ions):
        for d in range(3):
            a = pos.copy(); a[d, i] += h
            b = pos.copy(); b[d, i] -= h
            gx[d, k] = (oenergy.energy(p, a, q, phi_b) - oenergy.energy(p, b, q, phi_b)) / (2 * h)
        a = q.copy(); a[i] += h
        b = q.copy(); b[i] -= h
        gq[k] = (oenergy.energy(p, pos, a, phi_b) - oenergy.energy(p, pos, b, phi_b)) / (2 * h)
    gb = np.zeros(2)
    for w in range(2):
        a = list(phi_b); a[w] += h
        b = list(phi_b); b[w] -= h
        gb[w] = (oenergy.energy(p, pos, q, tuple(a)) - oenergy.energy(p, pos, q, tuple(b))) / (2 * h)
    return gx, gq, gb


@pytest.mark.parametrize("prec", [dg.FP64, dg.MIXED])
@pytest.mark.parametrize("bc", [(0, 0), (0, 1), (1, 0)])
def test_energy_value(prec, bc):
    cfg, rec = _small(prec, bc)
    xd, qd, pos, q = _ions(cfg, rec)
    h = dg.Discos(cfg)
    U = float(h.energy(xd, qd))
    ref = oenergy.energy(oracle_params(cfg), pos, q)
    assert abs(U - ref) <= TOL_U[prec] * abs(ref)


@pytest.mark.parametrize("prec", [dg.FP64, dg.MIXED])
@pytest.mark.parametrize("bc", [(0, 0), (0, 1)])
def test_energy_gradients_vs_finite_differences(prec, bc):
    cfg, rec = _small(prec, bc)
    xd, qd, pos, q = _ions(cfg, rec)
    h = dg.Discos(cfg)
    phi_b = torch.tensor(cfg.phi_b, dtype=torch.float64, requires_grad=True)
    x = xd.clone().requires_grad_(True)
    qq = qd.clone().requires_grad_(True)
    U = denergy(h, x, qq, phi_b)
    U.backward()
    ions = list(range(0, 301, 301 // 32))[:32]
    gx, gq, gb = _fd_grads(oracle_params(cfg), pos, q, tuple(cfg.phi_b), ions)
    tol = TOL_G[prec]
    assert rel_l2(x.grad.double().cpu().numpy()[:, ions], gx) < tol
    assert rel_l2(qq.grad.double().cpu().numpy()[ions], gq) < tol
    ngb = phi_b.grad.numpy()
    if bc == (0, 0):
        assert rel_l2(ngb, gb) < tol
    else:
        # the Neumann wall's potential does not enter U
        assert abs(ngb[1]) == 0.0 and abs(ngb[0] - gb[0]) <= tol * abs(gb[0])


def test_energy_upstream_scale_and_partial_needs():
    cfg, rec = _small(dg.FP64)
    xd, qd, _, _ = _ions(cfg, rec)
    h = dg.Discos(cfg)
    one = torch.ones((), dtype=torch.float64, device="cuda")
    dx1, dq1, db1 = h.energy_backward(xd, qd, one)
    dx3, dq3, db3 = h.energy_backward(xd, qd, 3.0 * one)
    # the spreading sums with atomics, so repeated calls agree to rounding only
    assert torch.allclose(dx3, 3.0 * dx1, rtol=1e-11, atol=1e-12)
    assert torch.allclose(dq3, 3.0 * dq1, rtol=1e-11, atol=1e-12)
    assert torch.allclose(db3, 3.0 * db1, rtol=1e-11, atol=1e-12)
    dx, dq, db = h.energy_backward(xd, qd, one, need=(False, True, False))
    assert dx is None and db is None and torch.allclose(dq, dq1, rtol=1e-11, atol=1e-12)


def test_energy_edge_cases():
    cfg, rec = _small(dg.FP64)
    h = dg.Discos(cfg)
    x0 = torch.empty((3, 0), dtype=torch.float64, device="cuda")
    q0 = torch.empty(0, dtype=torch.float64, device="cuda")
    assert float(h.energy(x0, q0)) == 0.0
    one = torch.ones((), dtype=torch.float64, device="cuda")
    _, _, db = h.energy_backward(x0, q0, one)
    assert torch.count_nonzero(db) == 0
    # two Neumann walls fix no potential: rejected before any launch
    cfg2, _ = _small(dg.FP64, bc=(1, 1))
    cfg2.surf_charge = (0.0, 0.0)
    h2 = dg.Discos(cfg2)
    with pytest.raises(dg.DiscosError):
        h2.energy(x0, q0)


@pytest.mark.parametrize("prec", [dg.FP64, dg.MIXED])
def test_energy_full_size(prec):
    cfg, rec = presets.energy_channel_64(prec)
    xd, qd, pos, q = _ions(cfg, rec)
    h = dg.Discos(cfg)
    phi_b = torch.tensor(cfg.phi_b, dtype=torch.float64, requires_grad=True)
    x = xd.clone().requires_grad_(True)
    qq = qd.clone().requires_grad_(True)
    U = denergy(h, x, qq, phi_b)
    U.backward()
    Uv = float(U.detach())
    ref = oenergy.energy(oracle_params(cfg), pos, q)
    assert abs(Uv - ref) <= TOL_U[prec] * abs(ref)
    # quadratic in q, linear in phi_b
    lhs = float((qq.detach().double() * qq.grad.double()).sum())
    rhs = 2.0 * Uv - float((phi_b.detach() * phi_b.grad).sum())
    assert abs(lhs - rhs) <= (1e-9 if prec == dg.FP64 else 1e-4) * abs(Uv)
    # the P3M, wall and external parts are not in U: compare with the grid force
    Fg = qd * h.interpolate_efield(xd, h.solve_poisson(h.spread_charge(xd, qd)))
    assert rel_l2(-x.grad.double().cpu().numpy(), Fg.double().cpu().numpy()) < 5e-2


def test_energy_gradients_full_size_fd():
    """The 64^3 Dirichlet channel with 4096 ions and wall potentials
    +0.5 / -0.5: the hand-written backward against FP64 central differences
    (h = 1e-4) of the forward energy on a 32-ion subset, for positions,
    charges and both wall potentials.  The forward is itself compared with the
    oracle's energy on this channel (test_energy_full_size)."""
    cfg, rec = presets.energy_channel_64(dg.FP64)
    xd, qd, pos, q = _ions(cfg, rec)
    h = dg.Discos(cfg)
    phi_b = torch.tensor(cfg.phi_b, dtype=torch.float64, requires_grad=True)
    x = xd.clone().requires_grad_(True)
    qq = qd.clone().requires_grad_(True)
    U = denergy(h, x, qq, phi_b)
    U.backward()
    hh = 1e-4
    ions = list(range(0, 4096, 128))

    def Uof(xv, qv, pb=None):
        return float(h.energy(xv, qv, pb))
    gx = np.zeros((3, len(ions)))
    gq = np.zeros(len(ions))
    for k, i in enumerate(ions):
        for d in range(3):
            a = xd.clone(); a[d, i] += hh
            b = xd.clone(); b[d, i] -= hh
            gx[d, k] = (Uof(a, qd) - Uof(b, qd)) / (2 * hh)
        a = qd.clone(); a[i] += hh
        b = qd.clone(); b[i] -= hh
        gq[k] = (Uof(xd, a) - Uof(xd, b)) / (2 * hh)
    gb = np.zeros(2)
    for w in range(2):
        a = list(cfg.phi_b); a[w] += hh
        b = list(cfg.phi_b); b[w] -= hh
        gb[w] = (Uof(xd, qd, a) - Uof(xd, qd, b)) / (2 * hh)
    assert rel_l2(x.grad.double().cpu().numpy()[:, ions], gx) < 1e-6
    assert rel_l2(qq.grad.double().cpu().numpy()[ions], gq) < 1e-6
    assert rel_l2(phi_b.grad.numpy(), gb) < 1e-6
