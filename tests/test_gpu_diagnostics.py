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


def _setup(prec, bc=(1, 1), n=300):
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


@pytest.mark.parametrize("prec", [dg.FP64, dg.MIXED])
def test_non_neutral_neumann_channel_rejected(prec):
    """Two Neumann walls fix the potential only up to a constant and need
    charge + surface charge = 0 (Sec. II.B.1).  discos_forces and
    discos_solve_poisson check it in double before any solve is launched
    (status 3); discos_step checks it on the device every step and refuses the
    next call.  A neutral channel with surface charge passes."""
    cfg, x, q = _setup(prec, bc=(1, 1))
    h = dg.Discos(cfg)
    h.forces(x, q)                                   # neutral: accepted
    q2 = q.clone()
    q2[0] += 1.0                                     # net charge +1 (or 0 -> 2, 1 -> 2)
    with pytest.raises(dg.DiscosError) as ei:
        h.forces(x, q2)
    assert ei.value.status == 3
    rho = h.spread_charge(x, q2)
    with pytest.raises(dg.DiscosError) as ei:
        h.solve_poisson(rho)
    assert ei.value.status == 3
    h.step(x.clone(), q2, step0=0, nsteps=1)         # enqueued; the device flags bit 2
    torch.cuda.synchronize()
    assert h.fault(sync=True) & 4
    with pytest.raises(dg.DiscosError) as ei:
        h.step(x.clone(), q2, step0=1, nsteps=1)
    assert ei.value.status == 3
    h.fault(sync=True, clear=True)
    # surface charge balancing the ions' net charge: neutral again
    Nx, Ny, Nz = cfg.dims
    net = float(q2.double().sum())
    cfg.surf_charge = (-0.5 * net / (Nx * Nz), -0.5 * net / (Nx * Nz))
    h2 = dg.Discos(cfg)
    h2.forces(x, q2)
    h2.solve_poisson(h2.spread_charge(x, q2))
    h2.step(x.clone(), q2, step0=0, nsteps=1)
    assert h2.fault(sync=True) == 0


def test_failing_allocator_gives_oom():
    """A discos_alloc_fn that returns NULL: discos_create frees what it got,
    returns DISCOS_ERR_OOM (2) and no handle; the free hook sees every
    pointer the alloc hook handed out."""
    import ctypes
    from paper_2204_14167_gb300 import _lib
    lib = _lib.load()
    cfg, _, _ = _setup(dg.FP64)
    c = cfg.to_c()
    ALLOC = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
    FREE = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)
    given, freed = [], []
    budget = [3]            # three allocations succeed, then the device is "full"

    def alloc(nbytes, ctx):
        if budget[0] <= 0:
            return None
        budget[0] -= 1
        t = torch.empty(int(nbytes), dtype=torch.uint8, device="cuda")
        given.append(t)
        return t.data_ptr()

    def free(ptr, ctx):
        freed.append(ptr)
    a, f = ALLOC(alloc), FREE(free)
    hnd = ctypes.c_void_p()
    st = lib.discos_create(ctypes.byref(c), a, f, None, ctypes.byref(hnd))
    assert st == _lib.ERR_OOM
    assert not hnd.value
    assert sorted(freed) == sorted(t.data_ptr() for t in given)
