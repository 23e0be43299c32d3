"""Near-wall wet mobility measured with this library's own Stokes solver, and
the coefficients of Eq. fitfunction fitted to it (Sec. III.A).

The paper measures the mobility reduction gamma(y) by placing a particle at a
given wall distance, setting kT = 0, applying a force and noting the
particle's velocity (Sec. III.A, Fig. mobfit1), then fits Eq. fitfunction to
the measured points together with the point (0, 0).  Here each measurement
is one spread (S^hy), one Stokes solve and one interpolation (J^hy) through
libdiscos, so the measured mobility is exactly the discrete J L^-1 S that the
wet step applies, for any kernel, grid and wet fraction.  Only the ratio V/F,
the averages over sub-cell offsets and the seven-parameter least-squares fit
run on the host (a few dozen numbers: parameter set-up, not the hot path).

Normalisation: gamma = mu / mu_0 with mu_0 = 1 / (6 pi eta a_w) the free-space
mobility of a particle of the kernel's hydrodynamic radius a_w.  The radius is
itself measured: it is the a_w for which the channel formula of Eq.
mob_analytic, gamma(L/2; a_w) / (6 pi eta a_w), equals the mobility measured
at mid-channel (solved by bisection); away from the walls the formula is
accurate (Sec. III.A), so the measurement fixes both the radius and the
near-wall profile.
"""
import math

import numpy as np

from . import mobility


def measure_mobility(handle, ys, n_offsets=4, seed=0, directions=(0, 1), stream=None):
    """Mobility V_d / F_d (d = 0: parallel to the walls, x; d = 1:
    perpendicular, y) of a single particle at each wall distance y in `ys`,
    averaged over `n_offsets` random sub-cell (x, z) positions (the kernels
    are not exactly translation invariant).  `handle` is a Discos created
    with wet = True; kT and the handle's ions are not used.
    Returns an array (len(directions), len(ys))."""
    import torch
    cfg = handle.cfg
    rng = np.random.default_rng(seed)
    dt = handle.dtype
    out = np.zeros((len(directions), len(ys)))
    offs = rng.uniform(0.0, 1.0, size=(n_offsets, 2))
    x0, z0 = 0.5 * cfg.Nx, 0.5 * cfg.Nz
    for k, y in enumerate(ys):
        for ox, oz in offs:
            x = torch.tensor([[x0 + ox], [float(y)], [z0 + oz]], dtype=dt, device=handle.device)
            for i, d in enumerate(directions):
                F = torch.zeros((3, 1), dtype=dt, device=handle.device)
                F[d, 0] = 1.0
                f = handle.spread_force(x, F, stream=stream)
                v = handle.solve_stokes(f, stream=stream)
                V = handle.interpolate_velocity(x, v, stream=stream)
                out[i, k] += float(V[d, 0]) / n_offsets
    return out


def hydrodynamic_radius(mu_mid, L, eta, lo=0.05, hi=None, tol=1e-10):
    """The radius a with gamma_perp(L/2; a) / (6 pi eta a) = mu_mid for the
    perpendicular mobility at mid-channel (Eq. mob_analytic, reading of
    Eq. singlewall as powers of a / y).  The left side falls monotonically
    with a; it is evaluated on a grid of radii at once (the channel series is
    vectorised over a), the bracketing interval is refined, and so on until
    the bracket is narrower than tol."""
    hi = 0.45 * L if hi is None else hi
    for _ in range(12):
        a = np.linspace(lo, hi, 65)
        f = mobility.channel(np.full_like(a, 0.5 * L), L, a, True) / (6.0 * math.pi * eta * a) - mu_mid
        if f[0] * f[-1] > 0:
            raise ValueError("mid-channel mobility outside the range of the channel formula")
        k = int(np.argmax(np.sign(f) != np.sign(f[0])))
        lo, hi = a[k - 1], a[k]
        if hi - lo < tol:
            break
    return 0.5 * (lo + hi)


def fit_to_points(yt, g, scale=1.0):
    """Least-squares coefficients c1..c7 of Eq. fitfunction through the
    measured points (yt, g) plus the point (0, 0) (Fig. mobfit1)."""
    from scipy.optimize import least_squares
    yt = np.concatenate([[0.0], np.asarray(yt, dtype=np.float64)])
    g = np.concatenate([[0.0], np.asarray(g, dtype=np.float64)])
    a = scale
    x0 = np.array([1.0, -1.0 * a, 0.5 * a, 0.1 * a ** 3, 0.5 * a, -0.01 * a ** 5, 0.5 * a])

    def res(c):
        return mobility.fit_function(yt, c) - g
    lo = np.array([-np.inf, -np.inf, 1e-3, -np.inf, 1e-3, -np.inf, 1e-3])
    sol = least_squares(res, x0, bounds=(lo, np.full(7, np.inf)), xtol=1e-14, ftol=1e-14, max_nfev=20000)
    return [float(v) for v in sol.x]


def calibrate_gamma_wet(handle, n_points=None, n_offsets=4, seed=0):
    """Measure gamma_parallel(y) and gamma_perpendicular(y) over the lower half
    of the handle's channel and fit Eq. fitfunction to each.
    Returns dict(a_w, ys, gamma (2, n), coef [[par c1..c7], [perp c1..c7]])."""
    cfg = handle.cfg
    L = float(cfg.Ny)
    n = n_points or max(8, cfg.Ny)
    ys = np.linspace(0.05 * L / n, 0.5 * L, n)
    mu = measure_mobility(handle, ys, n_offsets=n_offsets, seed=seed)
    a_w = hydrodynamic_radius(mu[1, -1], L, cfg.eta)
    mu0 = 1.0 / (6.0 * math.pi * cfg.eta * a_w)
    gam = mu / mu0
    coef = [fit_to_points(ys, gam[0], a_w), fit_to_points(ys, gam[1], a_w)]
    return dict(a_w=a_w, ys=ys, gamma=gam, coef=coef)
