"""The wet-mobility calibration of Sec. III.A (paper_2204_14167_gb300.calibrate).

CPU (no GPU): the host fit of Eq. fitfunction through measured points plus
(0, 0) reproduces the channel formula it is fed, and the radius solve inverts
the mid-channel mobility of Eq. mob_analytic.
GPU: the measured mobility V/F of one particle (spread, Stokes solve,
interpolation through libdiscos) equals the oracle's J L^-1 S at the same
positions (FP64 1e-10); and on a channel 32 cells high, four times wider,
the measured near-wall reductions follow Eq. mob_analytic within 5 % for
wall distances >= 0.7 a (the paper reports good agreement there, with no
number).  The formula superposes single-wall corrections, which is an
approximation of order a / L: on a channel 16 cells high the parallel
mobility at mid-channel already sits 6 % below it.
"""
import math

import numpy as np
import pytest

from paper_2204_14167_gb300 import calibrate, mobility


def test_fit_through_points_reproduces_profile():
    L, a = 16.0, 1.0
    y = np.linspace(0.7 * a, 0.5 * L, 60)
    for perp in (False, True):
        g = mobility.channel(y, L, a, perp)
        c = calibrate.fit_to_points(y, g, a)
        assert np.max(np.abs(mobility.fit_function(y, c) - g)) < 0.02
        assert abs(mobility.fit_function(np.array([0.0]), c)[0]) < 0.05


def test_radius_inverts_mid_channel_mobility():
    L, eta = 24.0, 1.0 / (6.0 * math.pi)
    for a in (0.6, 0.91, 1.4):
        mu = mobility.channel(np.array([0.5 * L]), L, a, True)[0] / (6.0 * math.pi * eta * a)
        assert abs(calibrate.hydrodynamic_radius(mu, L, eta) - a) < 1e-8


def _handle(dims, prec):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2204_14167_gb300 as dg
    from paper_2204_14167_gb300 import presets
    cfg, _ = presets.wet_channel_small(prec, *dims, n=2)
    cfg.kT = 0.0
    return dg.Discos(cfg), cfg


@pytest.mark.gpu
def test_measured_mobility_matches_oracle():
    import paper_2204_14167_gb300 as dg
    from helpers import oracle_params
    from oracle import gridops, stokes
    h, cfg = _handle((16, 12, 16), dg.FP64)
    ys = np.array([0.4, 1.3, 3.7, 6.0])
    mu = calibrate.measure_mobility(h, ys, n_offsets=1, seed=3)
    ox, oz = np.random.default_rng(3).uniform(0.0, 1.0, size=(1, 2))[0]
    p = oracle_params(cfg)
    ref = np.zeros_like(mu)
    for k, y in enumerate(ys):
        pos = np.array([[0.5 * cfg.Nx + ox], [y], [0.5 * cfg.Nz + oz]])
        for i, d in enumerate((0, 1)):
            F = np.zeros((3, 1))
            F[d, 0] = 1.0
            u, v, w, _ = stokes.solve(*gridops.spread_force(p["kernel_hy"], pos, F, cfg.dims), cfg.eta)
            ref[i, k] = gridops.interp_velocity(p["kernel_hy"], pos, u, v, w)[d, 0]
    assert np.max(np.abs(mu - ref)) <= 1e-10 * np.max(np.abs(ref))


@pytest.mark.gpu
def test_calibrated_gamma_follows_channel_formula():
    import paper_2204_14167_gb300 as dg
    h, cfg = _handle((128, 32, 128), dg.MIXED)
    res = calibrate.calibrate_gamma_wet(h, n_points=16, n_offsets=4)
    a = res["a_w"]
    assert 0.5 < a < 2.0
    ys, gam = res["ys"], res["gamma"]
    sel = ys >= 0.7 * a
    for i, perp in ((0, False), (1, True)):
        ref = mobility.channel(ys[sel], float(cfg.Ny), a, perp)
        assert np.max(np.abs(gam[i, sel] - ref) / ref) < 0.05, (gam[i, sel], ref)
        fit = mobility.fit_function(ys, res["coef"][i])
        assert np.max(np.abs(fit - gam[i])) < 0.03
