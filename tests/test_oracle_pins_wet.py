"""Pins of the oracle's wet-path and wall functions against what the paper and
the mathematics fix (no GPU):

* the RFD thermal forcing (Eq. thermforce, read as random finite
  differences): its mean over the random direction W is kT times the
  position derivative of the spreading operator, (div_x S) along each MAC
  component, which central differences of the spreading give independently;
* the dry tensor of Eq. diff2 with a wet part: the total near-wall diffusion
  D^dry Gamma + D^wet gamma^wet equals gamma^tot D^tot (the sum rule of
  Eq. diffSum with the confined diffusion of Sec. II.C); its Ito drift is
  the y derivative of D^dry Gamma_perp, checked by central differences;
* the wall force (Sec. II.B.2, Eq. LJ93 and the truncated-shifted 12-6
  form of Eq. potential): F_y = -dU/dy of the potential written out here,
  for both walls and both forms;
* the wet update (Eqs. step1-step2 with the midpoint scheme): for
  non-interacting ions the uniform density between no-slip walls stays
  stationary with the RFD term and the midpoint stage, and is biased toward
  the walls without them (the wet version of the Sec. III.D experiment).
"""
import numpy as np
import pytest

from paper_2204_14167_gb300 import presets
from helpers import oracle_params
from oracle import gridops, integrate, kernels, mobility, particles, stokes


# ------------------------------------------------------------------ RFD
@pytest.mark.parametrize("kind,pos0", [(kernels.PESKIN4, (3.3, 1.7, 4.1)), (kernels.PESKIN6, (2.6, 6.2, 5.45)),
                                      ((kernels.ES, 7, 7.0), (3.3, 1.7, 4.1))])
def test_rfd_mean_is_kT_div_S(kind, pos0):
    """E_W[f_th] = kT sum_c d/dx_c (S e_c)(x): the mean of Eq. thermforce's
    random finite difference over many directions W (one per ion copy, from
    Philox tag 2) against central differences of the spreading of a unit
    force along each axis.  Near a wall, so the image terms take part."""
    dims = (8, 8, 8)
    kT = 1.7
    kern = kernels.Kernel(*kind) if isinstance(kind, tuple) else kernels.Kernel(kind)
    M = 120000
    pos = np.tile(np.asarray(pos0, dtype=np.float64)[:, None], (1, M))
    fth = stokes.rfd_forcing(kern, pos, dims, kT, 3, 0, 20220428)
    mean = [f / M for f in fth]
    h = 1e-5
    ref = []
    one = np.asarray(pos0, dtype=np.float64)[:, None]
    for c in range(3):
        e = np.zeros((3, 1))
        e[c] = 1.0
        plus = gridops.spread_force(kern, one + h * e, e, dims)[c]
        minus = gridops.spread_force(kern, one - h * e, e, dims)[c]
        ref.append(kT * (plus - minus) / (2 * h))
    num = np.sqrt(sum(np.sum((a - b) ** 2) for a, b in zip(mean, ref)))
    den = np.sqrt(sum(np.sum(b ** 2) for b in ref))
    # standard error of the mean ~ 1/sqrt(M) of an O(1) per-draw spread:
    # about 1 % here; a factor 2 or a sign error is 50 % or 200 %
    assert num / den < 0.05, num / den


# ------------------------------------------------------------------ Eq. diff2
def _coef():
    # two different fitted profiles for the total and wet radii (a_t = 0.6, a_w = 1.2)
    from paper_2204_14167_gb300 import mobility as host_mobility
    return host_mobility.gamma_table(0.6, 1.2, 12.0)


@pytest.mark.parametrize("D_tot,D_wet", [(2.0, 1.0), (1.5, 0.3), (3.0, 2.7)])
def test_dry_tensor_sum_rule(D_tot, D_wet):
    """D^dry Gamma + D^wet gamma^wet = D^tot gamma^tot per direction
    (Eq. diff2 with Eq. diffSum: the total confined diffusion gamma^tot D^tot
    is the sum of its wet and dry parts), at wall distances on both halves of
    the channel; and dGamma_perp/dy against central differences of
    Gamma_perp, including the sign change past mid-channel."""
    Ny = 12
    coef = _coef()
    p = dict(gamma_coef=[coef], D_tot=[D_tot], D_wet=[D_wet])
    y = np.array([0.3, 0.9, 2.5, 5.1, 6.8, 9.4, 11.2, 11.8])
    sp = np.zeros(len(y), dtype=np.int64)
    G, dGp = mobility.dry_tensor(y, Ny, sp, p)
    yt = np.minimum(y, Ny - y)
    D_dry = D_tot - D_wet
    for direction, rows in ((0, (0, 2)), (1, (1,))):
        g_tot = mobility.fit_gamma(yt, coef[direction][0])[0]
        g_wet = mobility.fit_gamma(yt, coef[direction][1])[0]
        for r in rows:
            assert np.allclose(D_dry * G[r] + D_wet * g_wet, D_tot * g_tot, rtol=1e-13, atol=1e-13)
    h = 1e-6
    Gp = mobility.dry_tensor(y + h, Ny, sp, p)[0][1]
    Gm = mobility.dry_tensor(y - h, Ny, sp, p)[0][1]
    assert np.allclose(dGp, (Gp - Gm) / (2 * h), rtol=1e-6, atol=1e-8)


def test_dry_tensor_fully_wet_profiles_equal():
    """gamma^wet = gamma^tot (a 100 % wet measurement used for both, as in
    Fig. mobfit3's comparison) gives Gamma = gamma^tot for any split of D."""
    coef = _coef()
    same = [[coef[0][0], coef[0][0]], [coef[1][0], coef[1][0]]]
    y = np.linspace(0.1, 11.9, 23)
    for D_wet in (0.2, 0.9):
        p = dict(gamma_coef=[same], D_tot=[1.0], D_wet=[D_wet])
        G, _ = mobility.dry_tensor(y, 12, np.zeros(len(y), dtype=np.int64), p)
        yt = np.minimum(y, 12 - y)
        assert np.allclose(G[1], mobility.fit_gamma(yt, same[1][0])[0], rtol=1e-13)
        assert np.allclose(G[0], mobility.fit_gamma(yt, same[0][0])[0], rtol=1e-13)


# ------------------------------------------------------------------ wall force
def _u_126(d, sig, xi, rc):
    u = lambda r: 4.0 * xi * ((sig / r) ** 12 - (sig / r) ** 6)
    return np.where(d < rc, u(d) - u(rc), 0.0)


def _u_93(d, sig, xi, rc):
    u = lambda r: 1.5 * np.sqrt(3.0) * xi * ((sig / r) ** 9 - (sig / r) ** 3)
    return np.where(d < rc, u(d) - u(rc), 0.0)


@pytest.mark.parametrize("wall_type", [particles.WALL_WCA, particles.WALL_LJ93])
def test_wall_force_is_minus_gradient(wall_type):
    """F^W_y = -d/dy [U(y) + U(Ny - y)] with U the truncated, shifted wall
    potential (12-6 of Eq. potential in the wall distance, or Eq. LJ93), at
    points within the cutoff of either wall; zero beyond both cutoffs."""
    Ny = 10
    sig, xi = 0.8, 1.3
    rc = 2.0 ** (1.0 / 6.0) * sig if wall_type == particles.WALL_WCA else 3.5 * sig * 0.5
    U = _u_126 if wall_type == particles.WALL_WCA else _u_93
    p = dict(dims=(8, Ny, 8), wall_sigma=[sig], wall_xi=[xi], wall_rc=[rc], wall_type=wall_type)
    y = np.array([0.55, 0.7, 0.85, rc * 0.97, Ny - 0.6, Ny - 0.75, Ny - rc * 0.98, 3.0, 5.0])
    pos = np.stack([np.full(len(y), 1.0), y, np.full(len(y), 2.0)])
    F = particles.wall_force(pos, np.zeros(len(y), dtype=np.int64), p)
    h = 1e-7
    tot = lambda yy: U(yy, sig, xi, rc) + U(Ny - yy, sig, xi, rc)
    ref = -(tot(y + h) - tot(y - h)) / (2 * h)
    assert np.allclose(F, ref, rtol=1e-6, atol=1e-7)
    assert F[0] > 0 and F[4] < 0          # repulsive: away from each wall
    assert F[7] == 0.0 and F[8] == 0.0


# ------------------------------------------------------------------ wet update
def _wet_profile(drift, N=2000, steps=300, Ny=8, seed=1):
    cfg, _ = presets.wet_channel_small(Nx=8, Ny=Ny, Nz=8, n=2)
    cfg.dt = 0.01
    cfg.drift = drift
    p = oracle_params(cfg)
    rng = np.random.default_rng(seed)
    pos = np.stack([rng.uniform(0, 8, N), rng.uniform(0, Ny, N), rng.uniform(0, 8, N)])
    sp = np.zeros(N, dtype=np.int64)
    F = np.zeros((3, N))
    acc = np.zeros(Ny)
    for k in range(steps):
        inc, _ = integrate.wet_increment(p, pos, sp, F, k)
        pos = integrate.wrap_reflect(pos + inc, cfg.dims)
        if k >= steps // 3:
            acc += np.histogram(pos[1], bins=Ny, range=(0, Ny))[0]
    return acc / acc.sum() * Ny


def test_wet_update_keeps_uniform_density():
    """Non-interacting ions between no-slip walls, 50 % wet, kT = 1: with the
    RFD thermal forcing and the midpoint stage (Eqs. step1-step2) the uniform
    density is stationary (each bin within 10 %; 2000 ions averaged over 160
    steps, which sit about 3 % from uniform when nothing is missing)."""
    rel = _wet_profile(True, steps=240)
    assert np.max(np.abs(rel - 1.0)) < 0.10, rel


def test_wet_update_without_drift_is_biased():
    """The same ions with the RFD term removed and a single stage (V = J(x) v,
    the scheme without the stochastic drift) pile up at the walls, where the
    wet mobility vanishes: the wall bins double."""
    rel = _wet_profile(False, steps=240)
    assert rel[0] > 1.5 and rel[-1] > 1.5, rel
    assert np.all(rel[1:-1] < 0.9), rel


# ------------------------------------------------------------------ Stokes residual
def test_stokes_stencil_residual_matches_assembled_operator():
    """The stencil form of the MAC operator (used for residual checks at
    full size) equals the assembled saddle system of the solver on random
    fields, and vanishes on the solver's own solution."""
    dims = (8, 6, 10)
    Nx, Ny, Nz = dims
    rng = np.random.default_rng(3)
    eta = 0.7
    u, w, p = (rng.normal(size=(Nz, Ny, Nx)) for _ in range(3))
    v = rng.normal(size=(Nz, Ny + 1, Nx))
    v[:, 0] = v[:, -1] = 0.0
    fx, fz = rng.normal(size=(Nz, Ny, Nx)), rng.normal(size=(Nz, Ny, Nx))
    fy = rng.normal(size=(Nz, Ny + 1, Nx))
    fy[:, 0] = fy[:, -1] = 0.0
    (rx, ry, rz), div = stokes.residual(u, v, w, p, fx, fy, fz, eta)
    Lu, Lv, Lw, Gx, Gy, Gz = stokes._ops(dims)
    pr = p.ravel()
    assert np.allclose(rx.ravel(), fx.ravel() - (eta * (Lu @ u.ravel()) + Gx @ pr), atol=1e-12)
    assert np.allclose(rz.ravel(), fz.ravel() - (eta * (Lw @ w.ravel()) + Gz @ pr), atol=1e-12)
    assert np.allclose(ry[:, 1:Ny].ravel(), fy[:, 1:Ny].ravel() - (eta * (Lv @ v[:, 1:Ny].ravel()) + Gy @ pr),
                       atol=1e-12)
    # the divergence is minus the adjoint of the gradient
    assert np.allclose(div.ravel(), -(Gx.T @ u.ravel() + Gy.T @ v[:, 1:Ny].ravel() + Gz.T @ w.ravel()), atol=1e-12)
    us, vs, ws, ps = stokes.solve(fx, fy, fz, eta)
    (rx, ry, rz), div = stokes.residual(us, vs, ws, ps, fx, fy, fz, eta)
    nf = np.sqrt(np.sum(fx ** 2) + np.sum(fy ** 2) + np.sum(fz ** 2))
    assert np.sqrt(np.sum(rx ** 2) + np.sum(ry ** 2) + np.sum(rz ** 2)) < 1e-10 * nf
    assert np.max(np.abs(div)) < 1e-10
