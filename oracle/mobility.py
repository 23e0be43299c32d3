"""Near-wall mobility: analytic channel formula, fit function, dry tensor.

Test infrastructure only (see ``oracle/__init__``).

* Single-wall corrections, Eq. singlewall.  The printed powers are garbled;
  reading: gamma*_par = 1 - 9/16 (a/y) + 1/8 (a/y)^3 - 1/16 (a/y)^5 and
  gamma*_perp = 1 - 9/8 (a/y) + 1/2 (a/y)^3 - 1/8 (a/y)^5.
* Channel of height L, Eq. mob_analytic (reading: the outer braces are
  inverted, y measured from the lower wall):
      gamma = {1 + sum_n (-1)^n [1/gamma*(nL + y) - 1]
                 + sum_n (-1)^n [1/gamma*((n+1)L - y) - 1]}^-1.
  As L -> infinity this reduces to gamma*(y).
* Fit function, Eq. fitfunction:
      gamma_hat(yt) = c1 + c2/(c3+yt) + c4/(c5+yt)^3 + c6/(c7+yt)^5,
  yt = distance to the nearest wall.
* Dry tensor, Eqs. diff1-diff2: D^dry Gamma with
      Gamma = (gamma^tot D^tot - gamma^wet D^wet) / D^dry
  per direction (x, z parallel; y perpendicular), and the Ito drift
  div D^dry = D^dry dGamma_perp/dy along y (Eq. ions3).
"""
import numpy as np


def gamma_single(yt, a, perp):
    s = a / np.asarray(yt, dtype=np.float64)
    if perp:
        return 1.0 - 9.0 / 8.0 * s + 0.5 * s ** 3 - 0.125 * s ** 5
    return 1.0 - 9.0 / 16.0 * s + 0.125 * s ** 3 - 1.0 / 16.0 * s ** 5


def gamma_channel(y, L, a, perp, tol=1e-12, nmax=100000):
    """Eq. mob_analytic (reading above); y from the lower wall."""
    y = np.asarray(y, dtype=np.float64)
    acc = np.ones_like(y)
    for n in range(nmax):
        t = (-1.0) ** n * ((1.0 / gamma_single(n * L + y, a, perp) - 1.0)
                           + (1.0 / gamma_single((n + 1) * L - y, a, perp) - 1.0))
        acc = acc + t
        if np.max(np.abs(t)) < tol:
            break
    return 1.0 / acc


def fit_gamma(yt, c):
    """Eq. fitfunction and its derivative in yt."""
    yt = np.asarray(yt, dtype=np.float64)
    c1, c2, c3, c4, c5, c6, c7 = c
    g = c1 + c2 / (c3 + yt) + c4 / (c5 + yt) ** 3 + c6 / (c7 + yt) ** 5
    dg = -c2 / (c3 + yt) ** 2 - 3.0 * c4 / (c5 + yt) ** 4 - 5.0 * c6 / (c7 + yt) ** 6
    return g, dg


def dry_tensor(y, Ny, species, p):
    """Gamma (3, N) and dGamma_perp/dy (N,) at wall-normal positions y.

    p: dict with gamma_coef [ns][2 dir (par, perp)][2 (tot, wet)][7],
    D_tot [ns], D_wet [ns].  Gamma = (g_tot D_tot - g_wet D_wet) / D_dry.
    """
    y = np.asarray(y, dtype=np.float64)
    sp_ = np.asarray(species)
    yt = np.minimum(y, Ny - y)
    side = np.where(y <= Ny - y, 1.0, -1.0)      # d yt / d y
    coef = np.asarray(p['gamma_coef'], dtype=np.float64)
    Dt = np.asarray(p['D_tot'], dtype=np.float64)[sp_]
    Dw = np.asarray(p['D_wet'], dtype=np.float64)[sp_]
    Dd = Dt - Dw
    G = np.zeros((3, len(y)))
    dGp = np.zeros(len(y))
    for direction in (0, 1):
        gt, dgt = fit_gamma(yt, coef[sp_, direction, 0, :].T)
        gw, dgw = fit_gamma(yt, coef[sp_, direction, 1, :].T)
        Gam = (gt * Dt - gw * Dw) / Dd
        dGam = (dgt * Dt - dgw * Dw) / Dd * side
        if direction == 0:
            G[0] = Gam
            G[2] = Gam
        else:
            G[1] = Gam
            dGp = dGam
    return G, dGp
