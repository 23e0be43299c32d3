"""Equilibrium density of non-interacting ions between walls under the dry
update (Eqs. diff1-diff2, ions3): with the Ito drift term the uniform
density is stationary despite the near-wall mobility; without it ions pile
up at the walls, where the mobility is small (the biased profile the paper
reports for its run without the drift).  Pins the sign and size of the
oracle's drift and mobility terms independently of the GPU path."""
import numpy as np

from paper_2204_14167_gb300 import presets, mobility
from helpers import oracle_params
from oracle import integrate


def _profile(drift, steps=200, N=40000, Ny=8):
    cfg, _ = presets.dry_channel_32()
    cfg.Nx, cfg.Ny, cfg.Nz = 8, Ny, 8
    cfg.gamma_coef = [mobility.gamma_table(1.0, 1.0, float(Ny))]
    cfg.dt = 0.01
    cfg.drift = drift
    p = oracle_params(cfg)
    rng = np.random.default_rng(1)
    pos = np.stack([rng.uniform(0, 8, N), rng.uniform(0, Ny, N), rng.uniform(0, 8, N)])
    sp = np.zeros(N, dtype=np.int64)
    F = np.zeros((3, N))
    for k in range(steps):
        pos = integrate.wrap_reflect(pos + integrate.dry_increment(p, pos, sp, F, k), cfg.dims)
    h, _ = np.histogram(pos[1], bins=Ny, range=(0, Ny))
    return h / (N / Ny)


def test_drift_keeps_uniform_density():
    rel = _profile(True)
    # 5000 ions per bin: 1.4 % standard error; 6 % is over 4 sigma
    assert np.max(np.abs(rel - 1.0)) < 0.06


def test_no_drift_biases_toward_walls():
    rel = _profile(False)
    assert rel[0] > 1.3 and rel[-1] > 1.3
    assert np.all(rel[1:-1] < 0.95)
