"""The synthetic input recipes (paper_2204_14167_gb300.synth / presets):
charge neutrality, ion counts, placement bounds and minimum separations,
reproducibility from the seed, and the batched replica counts."""
import numpy as np
import pytest
from scipy.spatial import cKDTree

from paper_2204_14167_gb300 import presets, synth


def _min_pair_distance(pos, dims):
    Nx, Ny, Nz = dims
    box = np.array([Nx, 4.0 * Ny + 16.0, Nz])
    tree = cKDTree(np.mod(pos.T, box), boxsize=box)
    d, _ = tree.query(np.mod(pos.T, box), k=2)
    return float(d[:, 1].min())


@pytest.mark.parametrize("name", ["dry_channel_32", "wet_channel_128x64x128", "energy_channel_64"])
def test_preset_ions(name):
    cfg, rec = presets.PRESETS[name]()
    pos, q, sp = synth.ions(cfg.dims, rec["n_pos"], rec["n_neg"], rec["seed"], rec["ymargin"], rec["min_sep"])
    Nx, Ny, Nz = cfg.dims
    assert pos.shape == (3, rec["n_pos"] + rec["n_neg"]) and pos.shape[1] <= cfg.max_ions
    assert q.sum() == rec["n_pos"] - rec["n_neg"] == 0
    assert np.all((pos[0] >= 0) & (pos[0] < Nx) & (pos[2] >= 0) & (pos[2] < Nz))
    assert np.all((pos[1] >= rec["ymargin"]) & (pos[1] <= Ny - rec["ymargin"]))
    if rec["min_sep"] > 0:
        assert _min_pair_distance(pos, cfg.dims) >= rec["min_sep"]
    pos2, q2, _ = synth.ions(cfg.dims, rec["n_pos"], rec["n_neg"], rec["seed"], rec["ymargin"], rec["min_sep"])
    assert np.array_equal(pos, pos2) and np.array_equal(q, q2)


def test_batched_replicas():
    cfg, rec = presets.batched_channels_32(R=24, seed=5)
    pos, q, sp, off = presets.batched_ions(cfg, rec)
    counts = np.diff(off)
    assert len(counts) == 24 and np.all(counts % 2 == 0)
    assert counts.min() >= 64 and counts.max() <= 512
    for r in range(24):
        a, e = off[r], off[r + 1]
        assert q[a:e].sum() == 0
        assert _min_pair_distance(pos[:, a:e], cfg.dims) >= rec["min_sep"]
    cfg512, rec512 = presets.batched_channels_32()
    assert len(rec512["counts"]) == 512 and min(rec512["counts"]) >= 64 and max(rec512["counts"]) <= 512


def test_stable_time_steps():
    # explicit Euler-Maruyama at WCA contact needs dt D U''(0.9 sigma) < 1
    for name in ["dry_channel_32", "iceo_channel_256x128x256"]:
        cfg, rec = presets.PRESETS[name]()
        sig = cfg.lj_sigma[0][0]
        r = 0.9 * sig
        u2 = 24.0 / r ** 2 * (26.0 * (sig / r) ** 12 - 7.0 * (sig / r) ** 6)
        D = cfg.D_tot[0]
        assert cfg.dt * D * u2 < 1.0, name
