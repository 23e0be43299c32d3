"""Near-wall mobility coefficients for the dry diffusion tensor (host set-up).

The method needs, per species and direction, the coefficients c1..c7 of the
fit function of Eq. fitfunction, gamma_hat(y) = c1 + c2/(c3+y) + c4/(c5+y)^3
+ c6/(c7+y)^5 in the distance y to the nearest wall.  The paper measures the
mobility with its own solver and fits it; the coefficients are not printed.
Here they are fitted by least squares to the channel formula Eq. mob_analytic
(single-wall corrections of Eq. singlewall read as powers of a/y, alternating
image sums), sampled on [0.7 a, L/2], plus the point (0, 0), as in Sec. III.A.  Below
0.7 a, where the channel formula is not valid and the paper fits measured
points, the target is the straight line from (0, 0) to the formula's value at
0.7 a, which keeps the fitted mobility non-negative and increasing there.
"""
import numpy as np


def single_wall(y, a, perp):
    s = a / np.asarray(y, dtype=np.float64)
    if perp:
        return 1.0 - 1.125 * s + 0.5 * s ** 3 - 0.125 * s ** 5
    return 1.0 - 0.5625 * s + 0.125 * s ** 3 - 0.0625 * s ** 5


def channel(y, L, a, perp, nmax=20000, tol=1e-13):
    y = np.asarray(y, dtype=np.float64)
    inv = np.ones_like(y)
    for n in range(nmax):
        sgn = 1.0 if n % 2 == 0 else -1.0
        t = sgn * ((1.0 / single_wall(n * L + y, a, perp) - 1.0)
                   + (1.0 / single_wall((n + 1) * L - y, a, perp) - 1.0))
        inv += t
        if np.max(np.abs(t)) < tol:
            break
    return 1.0 / inv


def fit_function(y, c):
    c1, c2, c3, c4, c5, c6, c7 = c
    return c1 + c2 / (c3 + y) + c4 / (c5 + y) ** 3 + c6 / (c7 + y) ** 5


def fit_coefficients(a, L, perp):
    """Seven coefficients of Eq. fitfunction for radius a in a channel of height L."""
    from scipy.optimize import least_squares
    y_lo = np.linspace(0.0, 0.7 * a, 15, endpoint=False)
    y_hi = np.linspace(0.7 * a, 0.5 * L, 200)
    g_hi = channel(y_hi, L, a, perp)
    y = np.concatenate([y_lo, y_hi])
    g = np.concatenate([g_hi[0] * y_lo / (0.7 * a), g_hi])
    x0 = np.array([1.0, -1.0 * a, 0.5 * a, 0.1 * a ** 3, 0.5 * a, -0.01 * a ** 5, 0.5 * a])

    def res(c):
        return fit_function(y, c) - g

    lo = np.array([-np.inf, -np.inf, 1e-3, -np.inf, 1e-3, -np.inf, 1e-3])
    sol = least_squares(res, x0, bounds=(lo, np.full(7, np.inf)), xtol=1e-14, ftol=1e-14, max_nfev=20000)
    return [float(v) for v in sol.x]


def gamma_table(a_tot, a_wet, L):
    """[direction][tot, wet][7] for one species (parallel, perpendicular)."""
    out = []
    for perp in (False, True):
        out.append([fit_coefficients(a_tot, L, perp), fit_coefficients(a_wet, L, perp)])
    return out
