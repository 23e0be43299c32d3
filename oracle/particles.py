"""Particle forces: P3M near-field correction with images, LJ/WCA, wall.

Test infrastructure only (see ``oracle/__init__``).

* Coulomb pair force, Eq. coulomb: F^C_ij = l_B q_i q_j xhat_ij / r^2
  (eps = 1/(4 pi l_B)).
* Local correction, Eqs. fullElectro and LC: for every partner within psi,
  F^LC_ij = F^C_ij - F^P_ij with F^P_ij = l_B q_i q_j f^P(r) xhat_ij from the
  pre-tabulated grid pair force (greens.fp_table).
* Images (Sec. II.B.1): partners include the mirror image of every ion
  (itself included) across each wall, carrying charge -q (Dirichlet) or +q
  (Neumann), whenever that image lies within psi.
* Ion-ion short range, Eqs. potential and closerange: truncated and shifted
  12-6 LJ, F^R = xhat (24 xi / r) (2 (sigma/r)^12 - (sigma/r)^6), r < r_c.
* Wall short range (Sec. II.B.2): a repulsive 12-6 potential in the distance
  to each wall, cut at r_c; or the 9-3 form of Eq. LJ93.

Every pair is visited by brute force (all i, all j, all images); no cell list.
Whether a pair is within a cutoff is an integer decision, so it is taken in
the precision of the positions the caller supplies (`pair_dtype`), with the
operation order  dx = x_i - x_j, minimum image by +-L, r2 = (dx^2 + dy^2) + dz^2,
and image coordinates -y_j or (2 Ny) - y_j, each operation rounded once.
The force values themselves are accumulated in float64.
"""
import numpy as np

from .greens import fp_lookup

DIRICHLET, NEUMANN = 0, 1
WALL_WCA, WALL_LJ93 = 0, 1


def cell_index(pos, dims, k):
    """List-cell coordinates by the integer rule floor(x) div k, clamped so the
    last cell along each axis absorbs the remainder."""
    Nx, Ny, Nz = dims
    nc = (Nx // k, Ny // k, Nz // k)
    c = [np.minimum(np.floor(pos[d]).astype(np.int64) // k, nc[d] - 1) for d in range(3)]
    return c, nc


def cell_list(pos, dims, k):
    """(cell id per ion, cellStart of length n_cells+1, perm) with ions stable
    by id inside each cell; cell id = (cz * ncy + cy) * ncx + cx."""
    (cx, cy, cz), nc = cell_index(pos, dims, k)
    cid = (cz * nc[1] + cy) * nc[0] + cx
    ncell = nc[0] * nc[1] * nc[2]
    counts = np.bincount(cid, minlength=ncell)
    start = np.zeros(ncell + 1, dtype=np.int64)
    start[1:] = np.cumsum(counts)
    perm = np.lexsort((np.arange(len(cid)), cid))
    return cid, start, perm


def _min_image(d, L, dt):
    half = dt(0.5) * dt(L)
    d = np.where(d > half, d - dt(L), d)
    d = np.where(d < -half, d + dt(L), d)
    return d


def near_field(pos, q, species, p, table, pair_dtype=np.float64, targets=None):
    """Near-field force on `targets` (default all ions).

    p: dict with dims, bc, lB, psi, lj_sigma/lj_xi/lj_rc [ns][ns].
    Returns (F (3, n_t) float64, counts (n_t,) int64) where counts = number of
    partners (real or image) within psi, the ion itself excluded and its own
    images included.
    """
    dt = pair_dtype
    Nx, Ny, Nz = p['dims']
    lB, psi = p['lB'], p['psi']
    X = np.asarray(pos).astype(dt)
    q = np.asarray(q, dtype=np.float64)
    species = np.asarray(species, dtype=np.int64)
    N = X.shape[1]
    if targets is None:
        targets = np.arange(N)
    targets = np.asarray(targets)
    F = np.zeros((3, len(targets)))
    counts = np.zeros(len(targets), dtype=np.int64)
    psi2 = dt(psi) * dt(psi)
    wall_sign = [(-1.0 if b == DIRICHLET else 1.0) for b in p['bc']]
    sig = np.asarray(p['lj_sigma'], dtype=np.float64)
    xi_ = np.asarray(p['lj_xi'], dtype=np.float64)
    rc = np.asarray(p['lj_rc'], dtype=np.float64)
    rc2_dt = (rc.astype(dt) * rc.astype(dt))
    for t0 in range(0, len(targets), 256):
        ti = targets[t0:t0 + 256]
        xi, yi, zi = X[0, ti][:, None], X[1, ti][:, None], X[2, ti][:, None]
        qi = q[ti][:, None]
        si = species[ti][:, None]
        dx = _min_image(xi - X[0][None, :], Nx, dt)
        dz = _min_image(zi - X[2][None, :], Nz, dt)
        dy = yi - X[1][None, :]
        r2 = (dx * dx + dy * dy) + dz * dz
        notself = ti[:, None] != np.arange(N)[None, :]
        r = np.sqrt(r2.astype(np.float64))
        rs = np.where(notself & (r2 > 0), r, 1.0)
        # P3M correction with real partners
        m = notself & (r2 < psi2)
        coef = np.where(m, lB * qi * q[None, :] * (1.0 / rs ** 2 - fp_lookup(table, psi, np.minimum(rs, psi * (1 - 1e-15)))), 0.0)
        # LJ with real partners
        sij = sig[si, species[None, :]]
        xij = xi_[si, species[None, :]]
        mlj = notself & (r2 < rc2_dt[si, species[None, :]])
        sr6 = (sij / rs) ** 6
        coef += np.where(mlj, 24.0 * xij / rs * (2.0 * sr6 * sr6 - sr6), 0.0)
        F[0, t0:t0 + 256] += np.sum(coef * dx.astype(np.float64) / rs, axis=1)
        F[1, t0:t0 + 256] += np.sum(coef * dy.astype(np.float64) / rs, axis=1)
        F[2, t0:t0 + 256] += np.sum(coef * dz.astype(np.float64) / rs, axis=1)
        counts[t0:t0 + 256] += np.sum(m, axis=1)
        # images across each wall (the ion's own image included); with a
        # metal strip in the bottom wall, a partner's bottom image takes the
        # sign of the wall under it (-1 over the strip's columns)
        strip = p.get('strip')
        for w in range(2):
            yimg = -X[1] if w == 0 else dt(2 * Ny) - X[1]
            wsign = wall_sign[w]
            if w == 0 and strip is not None:
                col = np.floor(np.asarray(pos, dtype=np.float64)[0]) + 0.5
                wsign = np.where((col >= strip[0]) & (col < strip[1]), -1.0, 1.0)[None, :]
            dyi = yi - yimg[None, :]
            # the own image has dx = dz = 0 exactly
            dxo, dzo = dx, dz
            r2i = (dxo * dxo + dyi * dyi) + dzo * dzo
            mi = r2i < psi2
            ri = np.sqrt(np.where(mi, r2i, 1).astype(np.float64))
            ci = np.where(mi, lB * qi * (wsign * q[None, :]) *
                          (1.0 / ri ** 2 - fp_lookup(table, psi, np.minimum(ri, psi * (1 - 1e-15)))), 0.0)
            F[0, t0:t0 + 256] += np.sum(ci * dxo.astype(np.float64) / ri, axis=1)
            F[1, t0:t0 + 256] += np.sum(ci * dyi.astype(np.float64) / ri, axis=1)
            F[2, t0:t0 + 256] += np.sum(ci * dzo.astype(np.float64) / ri, axis=1)
            counts[t0:t0 + 256] += np.sum(mi, axis=1)
    return F, counts


def wall_force(pos, species, p):
    """Short-range wall force F^W (Sec. II.B.2), y component only.

    WCA-type wall: 12-6 form in the wall distance, cut at rc (truncated and
    shifted as Eq. potential); LJ93 wall: Eq. LJ93, cut at rc.
    """
    Ny = p['dims'][1]
    y = np.asarray(pos[1], dtype=np.float64)
    sp_ = np.asarray(species)
    sig = np.asarray(p['wall_sigma'], dtype=np.float64)[sp_]
    xi_ = np.asarray(p['wall_xi'], dtype=np.float64)[sp_]
    rc = np.asarray(p['wall_rc'], dtype=np.float64)[sp_]
    Fy = np.zeros_like(y)
    for dist, sgn in ((y, 1.0), (Ny - y, -1.0)):
        m = dist < rc
        d = np.where(m, dist, 1.0)
        if p.get('wall_type', WALL_WCA) == WALL_WCA:
            sr6 = (sig / d) ** 6
            f = 24.0 * xi_ / d * (2.0 * sr6 * sr6 - sr6)
        else:
            c = 1.5 * np.sqrt(3.0) * xi_
            f = c * (9.0 * sig ** 9 / d ** 10 - 3.0 * sig ** 3 / d ** 4)
        Fy += np.where(m, sgn * f, 0.0)
    return Fy
