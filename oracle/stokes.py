"""Staggered (MAC) steady Stokes solve with no-slip walls, stochastic stress
and RFD thermal forcing.

Test infrastructure only (see ``oracle/__init__``).

Eq. disc_stokes / stokes_temporal:  grad_h p - eta lap_h v = f,  div_h v = 0,
on the MAC grid (normal velocities on faces, p at centres), periodic in x and
z, no-slip walls at y = 0 and y = Ny (Eq. fluidbc): v_y = 0 on the wall faces,
tangential ghosts u(-1) = -u(0) so the velocity vanishes on the wall.  The
saddle-point system is solved in its Uzawa (Schur complement) form with
exact inner solves; the pressure gauge is sum(p) = 0.

Stochastic forcing sqrt(2 kT eta / (dV dt)) div_h Z (Eq. stokes_temporal),
reading of the cited staggered construction: Z symmetric, diagonal entries
sqrt(2) N(0,1) at cell centres, off-diagonal entries N(0,1) on edges (xy:
(x=i, y=j), j = 0..Ny; xz: (x=i, z=k); yz: (y=j, z=k), j = 0..Ny), with the
off-diagonal entries on the wall edges (y = 0, Ny) scaled by sqrt(2) so that
the noise covariance D D^T equals -L + Div^T Div with L the no-slip viscous
operator (fluctuation-dissipation balance; checked in the tests).  Normals
come from Philox counters (cell index in an Nx * (Ny+1) * Nz lattice, step,
replica, tag): tag 3 gives (Zxx, Zyy, Zzz, Zxy), tag 4 gives (Zxz, Zyz, -, -).

Thermal forcing, Eq. thermforce, by random finite differences (only cited;
reading): f_th = (kT/delta) [S(x + delta W/2) W - S(x - delta W/2) W] with W
from Philox tag 2 per ion and delta = 1e-4 (1e-7 for the ES kernel: see
rfd_forcing).
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import gridops, kernels, philox


def _ops(dims, slip=(False, False)):
    """Sparse blocks: (Lu, Lv, Lw) = -lap_h with the wall rules, gradients and
    divergences.  Unknown layout: u (Nz,Ny,Nx), v interior (Nz,Ny-1,Nx) for
    faces j = 1..Ny-1, w (Nz,Ny,Nx), p (Nz,Ny,Nx).  Tangential ghost below a
    no-slip wall u(-1) = -u(0) (diagonal 6 + 1), below a slip wall
    u(-1) = +u(0) (zero shear, diagonal 6 - 1), Eq. fluidbc."""
    Nx, Ny, Nz = dims
    nc = Nx * Ny * Nz
    nv = Nx * (Ny - 1) * Nz
    ic = np.arange(nc).reshape(Nz, Ny, Nx)
    iv = np.arange(nv).reshape(Nz, Ny - 1, Nx)

    def lap_cell():
        r, c, v = [], [], []
        for ax in (0, 2):
            for sh in (1, -1):
                r.append(ic.ravel()); c.append(np.roll(ic, sh, axis=ax).ravel()); v.append(-np.ones(nc))
        r.append(ic[:, 1:, :].ravel()); c.append(ic[:, :-1, :].ravel()); v.append(-np.ones(ic[:, 1:, :].size))
        r.append(ic[:, :-1, :].ravel()); c.append(ic[:, 1:, :].ravel()); v.append(-np.ones(ic[:, 1:, :].size))
        d = np.full((Nz, Ny, Nx), 6.0)
        d[:, 0, :] += -1.0 if slip[0] else 1.0      # ghost u(-1) = +-u(0)
        d[:, -1, :] += -1.0 if slip[1] else 1.0
        r.append(ic.ravel()); c.append(ic.ravel()); v.append(d.ravel())
        return sp.csr_matrix((np.concatenate(v), (np.concatenate(r), np.concatenate(c))), shape=(nc, nc))

    def lap_face():
        r, c, v = [], [], []
        for ax in (0, 2):
            for sh in (1, -1):
                r.append(iv.ravel()); c.append(np.roll(iv, sh, axis=ax).ravel()); v.append(-np.ones(nv))
        r.append(iv[:, 1:, :].ravel()); c.append(iv[:, :-1, :].ravel()); v.append(-np.ones(iv[:, 1:, :].size))
        r.append(iv[:, :-1, :].ravel()); c.append(iv[:, 1:, :].ravel()); v.append(-np.ones(iv[:, 1:, :].size))
        r.append(iv.ravel()); c.append(iv.ravel()); v.append(np.full(nv, 6.0))   # wall faces v = 0
        return sp.csr_matrix((np.concatenate(v), (np.concatenate(r), np.concatenate(c))), shape=(nv, nv))

    # gradients (cell -> face)
    Gx = sp.csr_matrix((np.concatenate([np.ones(nc), -np.ones(nc)]),
                        (np.concatenate([ic.ravel(), ic.ravel()]),
                         np.concatenate([ic.ravel(), np.roll(ic, 1, axis=2).ravel()]))), shape=(nc, nc))
    Gz = sp.csr_matrix((np.concatenate([np.ones(nc), -np.ones(nc)]),
                        (np.concatenate([ic.ravel(), ic.ravel()]),
                         np.concatenate([ic.ravel(), np.roll(ic, 1, axis=0).ravel()]))), shape=(nc, nc))
    # y-face j (1..Ny-1) = iv[:, j-1]: p(j) - p(j-1)
    Gy = sp.csr_matrix((np.concatenate([np.ones(nv), -np.ones(nv)]),
                        (np.concatenate([iv.ravel(), iv.ravel()]),
                         np.concatenate([ic[:, 1:, :].ravel(), ic[:, :-1, :].ravel()]))), shape=(nv, nc))
    Lc = lap_cell()
    return Lc, lap_face(), Lc, Gx, Gy, Gz


def solve(fx, fy, fz, eta, tol=1e-13, slip=(False, False)):
    """Velocity (u on x-faces, v on y-faces incl. zero wall faces, w) and p.

    fy has shape (Nz, Ny+1, Nx); its wall rows are ignored.  Uzawa form of
    the saddle-point system  eta L vel + G p = f,  G^T vel = 0:  the pressure
    solves the Schur complement system  G^T L^-1 G p = G^T L^-1 f  by
    conjugate gradients on mean-zero pressures (the constant is the null
    space), with every L^-1 applied by a sparse LU factorisation of the
    viscous operator; then vel = L^-1 (f - G p) / eta.  slip = (bottom, top)
    slip walls (at most one: with two, the tangential operator has the
    uniform flow as its null space).
    """
    Nz, Ny, Nx = fx.shape
    dims = (Nx, Ny, Nz)
    if slip[0] and slip[1]:
        raise ValueError("at most one slip wall")
    Lu, Lv, Lw, Gx, Gy, Gz = _ops(dims, slip)
    lu_c = spla.splu(Lu.tocsc())
    lu_f = spla.splu(Lv.tocsc())

    def Linv(bx, by, bz):
        return lu_c.solve(bx), lu_f.solve(by), lu_c.solve(bz)

    def G(p):
        return Gx @ p, Gy @ p, Gz @ p

    def GT(a, b, c):
        return Gx.T @ a + Gy.T @ b + Gz.T @ c

    f = (fx.ravel(), fy[:, 1:Ny, :].ravel(), fz.ravel())
    rhs = GT(*Linv(*f))
    rhs -= rhs.mean()
    n = rhs.size
    S = spla.LinearOperator((n, n), matvec=lambda p: (lambda r: r - r.mean())(GT(*Linv(*G(p - p.mean())))),
                            dtype=np.float64)
    p, info = spla.cg(S, rhs, rtol=tol, atol=0.0, maxiter=5000)
    if info != 0:
        raise RuntimeError(f"Schur CG did not converge (info={info})")
    p = p - p.mean()
    gp = G(p)
    ux, uy, uz = Linv(*(a - b for a, b in zip(f, gp)))
    u = ux.reshape(Nz, Ny, Nx) / eta
    v = np.zeros((Nz, Ny + 1, Nx))
    v[:, 1:Ny, :] = uy.reshape(Nz, Ny - 1, Nx) / eta
    w = uz.reshape(Nz, Ny, Nx) / eta
    return u, v, w, p.reshape(Nz, Ny, Nx)


def residual(u, v, w, p, fx, fy, fz, eta, slip=(False, False)):
    """Momentum residuals f - (eta L vel + G p) on the faces (interior y-faces
    for v; its wall rows are returned as zero) and the divergence div_h vel,
    for given velocity and pressure fields, with the operators of Eq.
    disc_stokes applied by their stencils (no assembly, so it runs at any
    grid size): -lap_h with the no-slip rules of Eq. fluidbc (tangential
    ghost = -interior, v = 0 on the wall faces) and p_i - p_{i-1} gradients."""
    def lap_cell(a):
        out = 6.0 * a - np.roll(a, 1, 2) - np.roll(a, -1, 2) - np.roll(a, 1, 0) - np.roll(a, -1, 0)
        out[:, 1:, :] -= a[:, :-1, :]
        out[:, :-1, :] -= a[:, 1:, :]
        out[:, 0, :] += -a[:, 0, :] if slip[0] else a[:, 0, :]     # ghost u(-1) = +-u(0)
        out[:, -1, :] += -a[:, -1, :] if slip[1] else a[:, -1, :]
        return out

    u = np.asarray(u, dtype=np.float64)
    v = np.asarray(v, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    p = np.asarray(p, dtype=np.float64)
    rx = fx - (eta * lap_cell(u) + (p - np.roll(p, 1, 2)))
    rz = fz - (eta * lap_cell(w) + (p - np.roll(p, 1, 0)))
    vi = v[:, 1:-1, :]
    lv = 6.0 * vi - np.roll(vi, 1, 2) - np.roll(vi, -1, 2) - np.roll(vi, 1, 0) - np.roll(vi, -1, 0) \
        - v[:, :-2, :] - v[:, 2:, :]
    ry = np.zeros_like(v)
    ry[:, 1:-1, :] = fy[:, 1:-1, :] - (eta * lv + (p[:, 1:, :] - p[:, :-1, :]))
    return (rx, ry, rz), divergence(u, v, w)


def divergence(u, v, w):
    """div_h v at cell centres."""
    return (np.roll(u, -1, axis=2) - u) + (v[:, 1:, :] - v[:, :-1, :]) + (np.roll(w, -1, axis=0) - w)


def stress_fields(dims, step, replica, seed, slip=(False, False)):
    """Z components from Philox: centres (Zxx, Zyy, Zzz), edges (Zxy, Zxz, Zyz)
    on an (Nz, Ny+1, Nx) lattice, wall edges of Zxy and Zyz scaled by sqrt 2
    at a no-slip wall and by 0 at a slip wall (no shear stress there; with
    these scalings D D^T = L + Div^T Div holds for either wall, checked in the
    tests)."""
    Nx, Ny, Nz = dims
    cell = np.arange(Nx * (Ny + 1) * Nz, dtype=np.uint64)
    a = philox.normals4(cell, step, replica, philox.TAG_STRESS_A, seed)
    b = philox.normals4(cell, step, replica, philox.TAG_STRESS_B, seed)
    sh = (Nz, Ny + 1, Nx)
    Zxx = np.sqrt(2.0) * a[0].reshape(sh)[:, :Ny, :]
    Zyy = np.sqrt(2.0) * a[1].reshape(sh)[:, :Ny, :]
    Zzz = np.sqrt(2.0) * a[2].reshape(sh)[:, :Ny, :]
    Zxy = a[3].reshape(sh).copy()
    Zxz = b[0].reshape(sh)[:, :Ny, :]
    Zyz = b[1].reshape(sh).copy()
    for Zw in (Zxy, Zyz):
        Zw[:, 0, :] *= 0.0 if slip[0] else np.sqrt(2.0)
        Zw[:, Ny, :] *= 0.0 if slip[1] else np.sqrt(2.0)
    return Zxx, Zyy, Zzz, Zxy, Zxz, Zyz


def stress_divergence(Zxx, Zyy, Zzz, Zxy, Zxz, Zyz):
    """div_h Z on the faces.  Edge placement: Zxy[k, j, i] at (x=i, y=j),
    Zxz[k, j, i] at (x=i, z=k), Zyz[k, j, i] at (y=j, z=k)."""
    Nz, Ny, Nx = Zxx.shape
    dx = (Zxx - np.roll(Zxx, 1, axis=2)) + (Zxy[:, 1:, :] - Zxy[:, :-1, :]) \
        + (np.roll(Zxz, -1, axis=0) - Zxz)
    dy = np.zeros((Nz, Ny + 1, Nx))
    dy[:, 1:Ny, :] = (np.roll(Zxy, -1, axis=2)[:, 1:Ny, :] - Zxy[:, 1:Ny, :]) \
        + (Zyy[:, 1:, :] - Zyy[:, :-1, :]) \
        + (np.roll(Zyz, -1, axis=0)[:, 1:Ny, :] - Zyz[:, 1:Ny, :])
    dz = (np.roll(Zxz, -1, axis=2) - Zxz) + (Zyz[:, 1:, :] - Zyz[:, :-1, :]) \
        + (Zzz - np.roll(Zzz, 1, axis=0))
    return dx, dy, dz


def noise_forcing(dims, eta, kT, dt, step, replica, seed, slip=(False, False)):
    amp = np.sqrt(2.0 * kT * eta / dt)
    Z = stress_fields(dims, step, replica, seed, slip)
    dx, dy, dz = stress_divergence(*Z)
    return amp * dx, amp * dy, amp * dz


def rfd_forcing(kernel, pos, dims, kT, step, replica, seed, delta=None, first_index=0, slip=(False, False),
                species=None):
    """Thermal forcing f_th by random finite differences (reading above).
    With species given, `kernel` is a list of per-species kernels and every
    ion spreads with its own (App. B); the draws W stay keyed by ion index.

    The RFD is read as its delta -> 0 limit.  delta = 1e-4 reaches it to
    O(delta^2) for the Peskin kernels, whose first derivative is continuous.
    The ES kernel (Eq. eskernel) drops from exp(-beta) to 0 at the edge of
    its support, and a finite difference that straddles the edge picks up
    that jump divided by delta; near the edge its third derivative is also
    unbounded, so the O(delta^2) error of the difference grows there.  For ES
    kernels delta = 1e-7 (in double), where truncation and rounding are both
    near 1e-9 relative and the stencil points of a few hundred ions stay
    clear of the edge."""
    ks = kernel if isinstance(kernel, (list, tuple)) else [kernel]
    if delta is None:
        delta = 1e-7 if any(k.kind == kernels.ES for k in ks) else 1e-4
    N = pos.shape[1]
    W = philox.ion_normals(N, step, replica, philox.TAG_RFD, seed, first_index)
    if species is None:
        def spread(x):
            return gridops.spread_force(kernel, x, W, dims, slip)
    else:
        def spread(x):
            return gridops.spread_force_species(kernel, species, x, W, dims, slip)
    plus = spread(pos + 0.5 * delta * W)
    minus = spread(pos - 0.5 * delta * W)
    return tuple((kT / delta) * (a - b) for a, b in zip(plus, minus))
