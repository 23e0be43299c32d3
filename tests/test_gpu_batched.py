"""Batched replicas (discos_step_batched) against the FP64 oracle, replica by
replica, and the invariants of the batched machinery.

- One step of ragged replicas (0, 64, 97, 130, 257 and 512 ions, each with its
  own wall potentials): forces and displacements against oracle dry_step
  with the replica's Philox stream, relative L2 1e-4 (single-precision bulk);
  near-field partner counts bit-exact against the oracle's single-precision
  pair decisions; the FP64 sums against the charges and the returned forces.
- Step counting through graph replays and multi-step launches: 40 steps in
  one call (graph of 32 launches + 8 direct, and 4 steps per launch) against
  40 calls of one step, 1e-4 (only the order of float atomics differs; a
  wrong step index would change the noise by O(1)).
- Histogram: every step adds each ion once (exact totals), and one step's
  histogram is exactly the binning of the returned positions.
- The batched and the plain single-channel path agree on replica 0.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from helpers import oracle_params, rel_l2, min_image_disp  # noqa: E402
import paper_2204_14167_gb300 as dg  # noqa: E402
from paper_2204_14167_gb300 import presets  # noqa: E402
from oracle import integrate  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.init()


def _batch(counts, seed=11):
    cfg, rec = presets.batched_channels_32(R=len(counts), seed=seed)
    rec = dict(rec, counts=list(counts))
    pos, q, sp, off = presets.batched_ions(cfg, rec)
    return cfg, pos, q, sp, off


def _dev(pos, q, sp):
    x = torch.tensor(pos, dtype=torch.float32, device="cuda").contiguous()
    qd = torch.tensor(q, dtype=torch.float32, device="cuda")
    s = torch.tensor(sp, dtype=torch.int32, device="cuda")
    return x, qd, s


def test_batched_one_step_vs_oracle():
    counts = [64, 97, 0, 130, 257, 512]
    cfg, pos, q, sp, off = _batch(counts)
    R = len(counts)
    h = dg.Discos(cfg)
    x, qd, s = _dev(pos, q, sp)
    pos = x.double().cpu().numpy()
    q = qd.double().cpu().numpy()
    phib = np.array([[0.1 * r, -0.05 * r] for r in range(R)])
    phib_d = torch.tensor(phib, dtype=torch.float64, device="cuda")
    F = torch.zeros_like(x)
    nbr = torch.full((off[-1],), -1, dtype=torch.int32, device="cuda")
    sums = torch.zeros((R, 4), dtype=torch.float64, device="cuda")
    hist = torch.zeros((R, 1, cfg.Ny), dtype=torch.int32, device="cuda")
    b = h.make_batch(x, qd, off, species=s, phi_b=phib_d, hist=hist, sums=sums, F_out=F, nbr=nbr)
    x0 = x.clone()
    h.step_batched(b, step0=5, nsteps=1)
    torch.cuda.synchronize()
    Fg, xn, cnt = F.double().cpu().numpy(), x.double().cpu().numpy(), nbr.cpu().numpy()
    p = oracle_params(cfg)
    for r in range(R):
        a, e = off[r], off[r + 1]
        if e == a:
            continue
        pr = dict(p, phi_b=tuple(phib[r]))
        new, Fr, cr = integrate.dry_step(pr, pos[:, a:e], q[a:e], sp[a:e], 5, pair_dtype=np.float32, replica=r)
        assert rel_l2(Fg[:, a:e], Fr) < 1e-4, r
        d_gpu = min_image_disp(xn[:, a:e], x0.double().cpu().numpy()[:, a:e], cfg.dims)
        assert rel_l2(d_gpu, min_image_disp(new, pos[:, a:e], cfg.dims)) < 1e-4, r
        assert np.array_equal(cnt[a:e], cr), r
    S = sums.cpu().numpy()
    for r in range(R):
        a, e = off[r], off[r + 1]
        assert S[r, 0] == q[a:e].sum()
        np.testing.assert_allclose(S[r, 1:], Fg[:, a:e].sum(axis=1), rtol=1e-12, atol=1e-9)
    assert int(hist.sum()) == off[-1]


@pytest.mark.parametrize("spl", [1, 4])
def test_batched_step_counting(spl):
    counts = [128, 64, 300]
    cfg, pos, q, sp, off = _batch(counts, seed=3)
    h = dg.Discos(cfg)
    h.set_batched_shape(spl)
    x1, qd, s = _dev(pos, q, sp)
    x2 = x1.clone()
    b1 = h.make_batch(x1, qd, off, species=s)
    h.step_batched(b1, step0=100, nsteps=40)
    b2 = h.make_batch(x2, qd, off, species=s)
    for k in range(40):
        h.step_batched(b2, step0=100 + k, nsteps=1)
    torch.cuda.synchronize()
    d1 = min_image_disp(x1.double().cpu().numpy(), pos, cfg.dims)
    d2 = min_image_disp(x2.double().cpu().numpy(), pos, cfg.dims)
    assert rel_l2(d1, d2) < 1e-4


def test_batched_histogram():
    counts = [64, 200, 512]
    cfg, pos, q, sp, off = _batch(counts, seed=5)
    h = dg.Discos(cfg)
    x, qd, s = _dev(pos, q, sp)
    hist = torch.zeros((3, 1, cfg.Ny), dtype=torch.int32, device="cuda")
    b = h.make_batch(x, qd, off, species=s, hist=hist)
    h.step_batched(b, step0=0, nsteps=7)
    torch.cuda.synchronize()
    H = hist.cpu().numpy()
    for r, n in enumerate(counts):
        assert H[r].sum() == 7 * n
    hist.zero_()
    h.step_batched(b, step0=7, nsteps=1)
    torch.cuda.synchronize()
    y = x[1].cpu().numpy()
    for r in range(3):
        bins = np.clip(np.floor(y[off[r]:off[r + 1]]).astype(int), 0, cfg.Ny - 1)
        assert np.array_equal(hist[r, 0].cpu().numpy(), np.bincount(bins, minlength=cfg.Ny))


def test_batched_matches_plain_path():
    counts = [256, 100]
    cfg, pos, q, sp, off = _batch(counts, seed=9)
    h = dg.Discos(cfg)
    x, qd, s = _dev(pos, q, sp)
    F = torch.zeros_like(x)
    b = h.make_batch(x, qd, off, species=s, F_out=F)
    x0 = x.clone()
    h.step_batched(b, step0=3, nsteps=1)
    xp = x0[:, :256].contiguous()
    Fp = torch.empty_like(xp)
    h.step(xp, qd[:256].contiguous(), species=s[:256].contiguous(), step0=3, nsteps=1, F_out=Fp)
    torch.cuda.synchronize()
    assert rel_l2(F[:, :256].double().cpu().numpy(), Fp.double().cpu().numpy()) < 1e-4
    d_b = min_image_disp(x[:, :256].double().cpu().numpy(), x0[:, :256].double().cpu().numpy(), cfg.dims)
    d_p = min_image_disp(xp.double().cpu().numpy(), x0[:, :256].double().cpu().numpy(), cfg.dims)
    assert rel_l2(d_b, d_p) < 1e-4


def test_batched_tune_leaves_state():
    counts = [64, 128, 96, 320]
    cfg, pos, q, sp, off = _batch(counts, seed=13)
    h = dg.Discos(cfg)
    x, qd, s = _dev(pos, q, sp)
    x0 = x.clone()
    b = h.make_batch(x, qd, off, species=s)
    spl, ms = h.tune_batched(b, trial_steps=16)
    torch.cuda.synchronize()
    assert spl in (1, 2, 4, 8, 16) and ms > 0
    assert torch.equal(x, x0)


def test_batched_rejects():
    cfg, pos, q, sp, off = _batch([64, 64])
    x, qd, s = _dev(pos, q, sp)
    h = dg.Discos(cfg)
    with pytest.raises(dg.DiscosError):
        h.step_batched(h.make_batch(x, qd, [0, 64, 64 + 64, 0]), nsteps=1)   # decreasing offsets
    big_cfg, _ = presets.dry_channel_32(dg.MIXED)
    big_cfg.max_ions = 1024
    hb = dg.Discos(big_cfg)
    xb = torch.zeros((3, 600), dtype=torch.float32, device="cuda") + 5.0
    qb = torch.zeros(600, dtype=torch.float32, device="cuda")
    with pytest.raises(dg.DiscosError):
        hb.step_batched(hb.make_batch(xb, qb, [0, 600]), nsteps=1)          # > 512 ions
    cfg64, _ = presets.dry_channel_32(dg.FP64)
    h64 = dg.Discos(cfg64)
    with pytest.raises(dg.DiscosError):
        h64.step_batched(h64.make_batch(x.double(), qd.double(), off), nsteps=1)
