"""Parity along trajectories: the 32^3 Dirichlet channel with 256 ions
(l_B = 7, 6-point kernel, FP64) run for 100 steps on the GPU, and 8
batched replicas run for 1000 steps.  At sampled states the next step is
taken from the same state by both the GPU and the FP64 oracle (with the
same Philox counters): forces and displacements within the FP64 tolerance
1e-9 (single channel) or the single-precision 1e-4 (replicas), neighbour
counts bit-exact, and the fault word clear (the trajectory stayed finite
and inside the channel)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from helpers import oracle_params, rel_l2, min_image_disp  # noqa: E402
import paper_2204_14167_gb300 as dg  # noqa: E402
from paper_2204_14167_gb300 import presets, synth  # noqa: E402
from oracle import integrate  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.init()


def test_dry_channel_100_steps_sampled():
    cfg, rec = presets.dry_channel_32(dg.FP64)
    pos, q, sp = synth.ions(cfg.dims, rec["n_pos"], rec["n_neg"], rec["seed"], rec["ymargin"], rec["min_sep"])
    h = dg.Discos(cfg)
    x = torch.tensor(pos, dtype=torch.float64, device="cuda").contiguous()
    qd = torch.tensor(q, dtype=torch.float64, device="cuda")
    states = {}
    for k in range(100):
        if k in (0, 33, 66, 99):
            states[k] = x.clone()
        h.step(x, qd, step0=k, nsteps=1)
    torch.cuda.synchronize()
    assert h.fault(sync=True) == 0
    p = oracle_params(cfg)
    for k, xs in states.items():
        x1 = xs.clone()
        F = torch.empty_like(x1)
        h.step(x1, qd, step0=k, nsteps=1, F_out=F)
        F_nb, cnt = h.forces(xs, qd, counts=True)
        torch.cuda.synchronize()
        ph = xs.cpu().numpy()
        new, Fo, co = integrate.dry_step(p, ph, q, sp, k)
        assert rel_l2(F.cpu().numpy(), Fo) < 1e-9, k
        assert np.array_equal(cnt.cpu().numpy(), co), k
        d = min_image_disp(x1.cpu().numpy(), ph, cfg.dims)
        assert rel_l2(d, min_image_disp(new, ph, cfg.dims)) < 1e-9, k


def test_batched_1000_steps_sampled():
    counts = [64, 200, 350, 512, 96, 128, 300, 450]
    cfg, rec = presets.batched_channels_32(R=len(counts), seed=17)
    rec = dict(rec, counts=counts)
    pos, q, sp, off = presets.batched_ions(cfg, rec)
    h = dg.Discos(cfg)
    x = torch.tensor(pos, dtype=torch.float32, device="cuda").contiguous()
    qd = torch.tensor(q, dtype=torch.float32, device="cuda")
    s = torch.tensor(sp, dtype=torch.int32, device="cuda")
    b = h.make_batch(x, qd, off, species=s)
    h.step_batched(b, step0=0, nsteps=1000)
    torch.cuda.synchronize()
    assert h.fault(sync=True) == 0
    F = torch.zeros_like(x)
    nbr = torch.zeros(off[-1], dtype=torch.int32, device="cuda")
    b2 = h.make_batch(x, qd, off, species=s, F_out=F, nbr=nbr)
    x0 = x.double().cpu().numpy()
    h.step_batched(b2, step0=1000, nsteps=1)
    torch.cuda.synchronize()
    p = oracle_params(cfg)
    qh = qd.double().cpu().numpy()
    for r in (0, 3, 6):
        a, e = off[r], off[r + 1]
        new, Fo, co = integrate.dry_step(p, x0[:, a:e], qh[a:e], sp[a:e], 1000, pair_dtype=np.float32, replica=r)
        assert rel_l2(F.double().cpu().numpy()[:, a:e], Fo) < 1e-4, r
        assert np.array_equal(nbr.cpu().numpy()[a:e], co), r
        d = min_image_disp(x.double().cpu().numpy()[:, a:e], x0[:, a:e], cfg.dims)
        assert rel_l2(d, min_image_disp(new, x0[:, a:e], cfg.dims)) < 1e-4, r
