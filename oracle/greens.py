"""Lattice Green's function and the pre-tabulated grid pair force F^P.

Test infrastructure only (see ``oracle/__init__``).

Sec. II.B.1 (Eq. LC) subtracts, for every pair closer than psi, the force the
grid computes between the two charges "in an unbounded domain", pre-tabulated
against separation (the construction is only cited, to the authors' earlier
periodic-domain paper).  Reading used here:

  * The unbounded grid solve is the lattice Green's function of the 7-point
    Laplacian, -lap_h G = delta_{n,0} on Z^3, written as
        G(n) = int_0^inf prod_d exp(-2t) I_{n_d}(2t) dt
    (the Laplace-transform form of its Fourier integral).  Here it is
    integrated by adaptive quadrature on [0, T] plus the tail in u = t^-1/2.
  * The grid force on unit charge i at x_i due to unit charge j at x_j, with
    l_B = 1: spread j (kernel), phi = 4 pi G * rho_j, E = -grad_h phi on the
    faces, interpolate each component at x_i (the Eq. efieldop pipeline).
  * f^P(r) is the component of that force along (x_i - x_j)/r, averaged over
    a fixed sample set: 8 sub-cell offsets of x_j, ((a + 1/2)/2 per axis,
    a in {0,1}), times 13 directions (the cube's axes, face diagonals and body
    diagonals, one of each +/- pair).  f^P(0) = 0.  The table holds f^P at
    r_k = k psi / n_tab, k = 0..n_tab, and is read by linear interpolation.
"""
import functools
import numpy as np
from scipy import integrate, special

from .kernels import Kernel


@functools.lru_cache(maxsize=None)
def lattice_green(n1, n2, n3, T=40.0):
    """G(n) of -lap_h on Z^3 (G(0) = 0.25273..., a sixth of Watson's integral)."""
    n = (abs(int(n1)), abs(int(n2)), abs(int(n3)))
    f = lambda t: special.ive(n[0], 2 * t) * special.ive(n[1], 2 * t) * special.ive(n[2], 2 * t)
    head, _ = integrate.quad(f, 0.0, T, epsabs=1e-15, epsrel=1e-13, limit=500)

    def g(u):
        t = 1.0 / (u * u)
        return f(t) * 2.0 / (u ** 3)
    tail, _ = integrate.quad(g, 0.0, 1.0 / np.sqrt(T), epsabs=1e-15, epsrel=1e-13, limit=500)
    return head + tail


def green_box(R):
    """G(n) for |n_d| <= R as an array indexed [n3+R, n2+R, n1+R]."""
    out = np.zeros((2 * R + 1,) * 3)
    for a in range(-R, R + 1):
        for b in range(-R, R + 1):
            for c in range(-R, R + 1):
                key = tuple(sorted((abs(a), abs(b), abs(c))))
                out[c + R, b + R, a + R] = lattice_green(*key)
    return out


SAMPLE_DIRS = np.array([
    [1, 0, 0], [0, 1, 0], [0, 0, 1],
    [1, 1, 0], [1, -1, 0], [1, 0, 1], [1, 0, -1], [0, 1, 1], [0, 1, -1],
    [1, 1, 1], [1, 1, -1], [1, -1, 1], [-1, 1, 1]], dtype=np.float64)
SAMPLE_DIRS /= np.linalg.norm(SAMPLE_DIRS, axis=1)[:, None]
SAMPLE_OFFS = np.array([[(ax + 0.5) / 2, (ay + 0.5) / 2, (az + 0.5) / 2]
                        for az in (0, 1) for ay in (0, 1) for ax in (0, 1)])


def pair_grid_force(kernel, xi, xj, G, R):
    """Force on unit charge at xi from unit charge at xj, unbounded grid, l_B = 1."""
    w = kernel.w
    # source weights on cells p (centres p + 1/2)
    src = []
    for d in range(3):
        idx, wt = kernel.stencil(np.array([xj[d] - 0.5]))
        src.append((idx[0], wt[0]))
    # target box of cells covering centre and face stencils of xi
    lo = [int(np.floor(xi[d] - w / 2.0)) - 1 for d in range(3)]
    hi = [int(np.floor(xi[d] + w / 2.0)) + 1 for d in range(3)]
    cx = np.arange(lo[0], hi[0] + 1)
    cy = np.arange(lo[1], hi[1] + 1)
    cz = np.arange(lo[2], hi[2] + 1)
    # phi(c) = 4 pi sum_p G(c - p) w(p)
    dx = cx[:, None] - src[0][0][None, :]
    dy = cy[:, None] - src[1][0][None, :]
    dz = cz[:, None] - src[2][0][None, :]
    if max(np.abs(dx).max(), np.abs(dy).max(), np.abs(dz).max()) > R:
        raise ValueError("Green's box too small")
    Gsub = G[(dz + R)[:, None, None, :, None, None],
             (dy + R)[None, :, None, None, :, None],
             (dx + R)[None, None, :, None, None, :]]        # (cz, cy, cx, pz, py, px)
    wsrc = src[2][1][:, None, None] * src[1][1][None, :, None] * src[0][1][None, None, :]
    phi = 4.0 * np.pi * np.einsum('abcdef,def->abc', Gsub, wsrc)   # (cz, cy, cx)
    # faces inside the box: x-face at x = cx[m] between cells cx[m-1] and cx[m]
    Ex = -(phi[:, :, 1:] - phi[:, :, :-1]); fxs = cx[1:]
    Ey = -(phi[:, 1:, :] - phi[:, :-1, :]); fys = cy[1:]
    Ez = -(phi[1:, :, :] - phi[:-1, :, :]); fzs = cz[1:]
    k = kernel
    F = np.zeros(3)
    # x component: faces at x = fxs, centres in y, z
    F[0] = np.einsum('k,j,i,kji->', k(xi[2] - (cz + 0.5)), k(xi[1] - (cy + 0.5)), k(xi[0] - fxs), Ex)
    F[1] = np.einsum('k,j,i,kji->', k(xi[2] - (cz + 0.5)), k(xi[1] - fys), k(xi[0] - (cx + 0.5)), Ey)
    F[2] = np.einsum('k,j,i,kji->', k(xi[2] - fzs), k(xi[1] - (cy + 0.5)), k(xi[0] - (cx + 0.5)), Ez)
    return F


@functools.lru_cache(maxsize=None)
def fp_table(kernel_kind, psi, n_tab, es_w=6, es_beta=8.0):
    """f^P(r_k), r_k = k psi / n_tab, k = 0..n_tab (l_B = 1, unit charges)."""
    kernel = Kernel(kernel_kind, es_w, es_beta)
    w = kernel.w
    R = w + 3 + int(np.ceil(psi))
    G = green_box(R)
    base = np.array([20.0, 20.0, 20.0])
    tab = np.zeros(n_tab + 1)
    for kk in range(1, n_tab + 1):
        r = kk * psi / n_tab
        acc = 0.0
        for off in SAMPLE_OFFS:
            xj = base + off
            for u in SAMPLE_DIRS:
                xi = xj + r * u
                F = pair_grid_force(kernel, xi, xj, G, R)
                acc += F @ u
        tab[kk] = acc / (len(SAMPLE_OFFS) * len(SAMPLE_DIRS))
    return tab


def fp_lookup(tab, psi, r):
    """Linear interpolation of the table at separations r < psi."""
    n_tab = len(tab) - 1
    t = np.asarray(r, dtype=np.float64) * (n_tab / psi)
    k = np.minimum(np.floor(t).astype(np.int64), n_tab - 1)
    fr = t - k
    return tab[k] + fr * (tab[k + 1] - tab[k])
