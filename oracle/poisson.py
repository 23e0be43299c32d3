"""Poisson solve -eps lap_h phi = rho with wall boundary conditions.

Test infrastructure only (see ``oracle/__init__``).

Eq. poisson with eps = 1/(4 pi l_B) (reduced units, Delta r = 1), i.e.
    -lap_h phi = 4 pi l_B rho
on cell centres with the 7-point Laplacian, periodic in x and z.  The wall
conditions enter through ghost cells:
  Dirichlet, Eq. esbc1:  phi(-1) = 2 phi_b - phi(0)         (phi = phi_b on the wall face)
  Neumann,   Eq. esbc3:  phi(-1) = phi(0) - g_bottom,  phi(Ny) = phi(Ny-1) + g_top
with g = dphi/dy on the wall.  Reading of Eq. esbc3: with n the inward
normal, -eps grad(phi).n = varsigma, so g_bottom = -4 pi l_B varsigma_0 and
g_top = +4 pi l_B varsigma_1.  This sign makes "ion charge + surface charge =
0" the solvability condition of an all-Neumann channel, which is what Sec.
II.B.1 states.  For an all-Neumann channel the potential is fixed by the gauge
mean(phi) = 0.

The operator is assembled as a sparse matrix and solved by conjugate
gradients to a relative residual of 1e-13 (plain definition, no transforms).
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

DIRICHLET, NEUMANN = 0, 1


def wall_slopes(bc, surf_charge, lB):
    """g = dphi/dy at (bottom, top) for Neumann walls (reading of Eq. esbc3)."""
    return (-4.0 * np.pi * lB * surf_charge[0], 4.0 * np.pi * lB * surf_charge[1])


def assemble(dims, bc):
    """Sparse 7-point operator A = -lap_h with the ghost-cell wall rows."""
    Nx, Ny, Nz = dims
    n = Nx * Ny * Nz
    idx = np.arange(n).reshape(Nz, Ny, Nx)
    rows, cols, vals = [], [], []

    def add(r, c, v):
        rows.append(r.ravel()); cols.append(c.ravel()); vals.append(np.full(r.size, v))

    # x and z neighbours (periodic)
    for ax in (0, 2):
        for sh in (1, -1):
            add(idx, np.roll(idx, sh, axis=ax), -1.0)
    diag = np.full((Nz, Ny, Nx), 6.0)
    # y neighbours
    add(idx[:, 1:, :], idx[:, :-1, :], -1.0)
    add(idx[:, :-1, :], idx[:, 1:, :], -1.0)
    # wall rows: the missing neighbour is the ghost cell
    for w, j in ((0, 0), (1, Ny - 1)):
        if bc[w] == DIRICHLET:
            diag[:, j, :] += 1.0       # -phi_ghost = +phi_j - 2 phi_b
        else:
            diag[:, j, :] -= 1.0       # -phi_ghost = -phi_j -/+ g
    rows.append(idx.ravel()); cols.append(idx.ravel()); vals.append(diag.ravel())
    A = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n))
    return A


def rhs(rho, bc, phi_b, slopes, lB):
    """4 pi l_B rho plus the ghost-cell terms of the wall rows."""
    b = 4.0 * np.pi * lB * np.asarray(rho, dtype=np.float64).copy()
    if bc[0] == DIRICHLET:
        b[:, 0, :] += 2.0 * phi_b[0]
    else:
        b[:, 0, :] -= slopes[0]
    if bc[1] == DIRICHLET:
        b[:, -1, :] += 2.0 * phi_b[1]
    else:
        b[:, -1, :] += slopes[1]
    return b


def solve(rho, bc, lB, phi_b=(0.0, 0.0), surf_charge=(0.0, 0.0), tol=1e-13, x0=None):
    """phi on cell centres, shape (Nz, Ny, Nx)."""
    Nz, Ny, Nx = rho.shape
    dims = (Nx, Ny, Nz)
    A = assemble(dims, bc)
    slopes = wall_slopes(bc, surf_charge, lB)
    b = rhs(rho, bc, phi_b, slopes, lB).ravel()
    singular = bc[0] == NEUMANN and bc[1] == NEUMANN
    if singular:
        resid = b.sum()
        if abs(resid) > 1e-9 * max(np.abs(b).sum(), 1.0):
            raise ValueError("all-Neumann channel is not electroneutral")
        b = b - b.mean()
    phi, info = spla.cg(A, b, rtol=tol, atol=0.0, maxiter=20000,
                        x0=None if x0 is None else np.asarray(x0).ravel())
    if info != 0:
        raise RuntimeError(f"CG did not converge (info={info})")
    if singular:
        phi = phi - phi.mean()
    return phi.reshape(Nz, Ny, Nx)


def residual(phi, rho, bc, lB, phi_b=(0.0, 0.0), surf_charge=(0.0, 0.0)):
    """b - A phi for a given potential (for checks at any grid size)."""
    Nz, Ny, Nx = rho.shape
    A = assemble((Nx, Ny, Nz), bc)
    b = rhs(rho, bc, phi_b, wall_slopes(bc, surf_charge, lB), lB).ravel()
    return (b - A @ np.asarray(phi, dtype=np.float64).ravel()).reshape(Nz, Ny, Nx), b.reshape(Nz, Ny, Nx)


def strip_columns(dims, x0, x1):
    """Bottom-wall cells (Nz, Nx) whose centre x + 1/2 lies on the metal strip
    [x0, x1) (the strip spans the channel in z, Fig. EOgeometry)."""
    Nx, Ny, Nz = dims
    xc = np.arange(Nx) + 0.5
    on = (xc >= x0) & (xc < x1)
    return np.broadcast_to(on[None, :], (Nz, Nx)).copy()


def strip_potential(dims, x0, x1, phi_total, E_x):
    """phi_m on the strip's cells (Nz, Nx): the fixed potential of the solve
    that makes the total potential phi + phi_E constant (= phi_total) on the
    metal, with phi_E = -E_x (x - x_c) the applied field's potential and x_c
    the strip's centre (Sec. IV.B; reading of where phi_E is zero)."""
    Nx, Ny, Nz = dims
    xc = np.arange(Nx) + 0.5
    pm = phi_total + E_x * (xc - 0.5 * (x0 + x1))
    return np.broadcast_to(pm[None, :], (Nz, Nx)).copy()


def assemble_strip(dims, bc_top, strip):
    """The 7-point operator with a mixed bottom wall: Dirichlet ghost rows
    (phi(-1) = 2 phi_m - phi(0)) on the strip cells, Neumann ghost rows
    (phi(-1) = phi(0) - g) elsewhere; the top wall of type bc_top."""
    Nx, Ny, Nz = dims
    A = assemble(dims, (NEUMANN, bc_top)).tolil()
    idx = np.arange(Nx * Ny * Nz).reshape(Nz, Ny, Nx)
    for k, i in zip(*np.nonzero(strip)):
        r = idx[k, 0, i]
        A[r, r] += 2.0          # Neumann -1 becomes Dirichlet +1
    return A.tocsr()


def solve_strip(rho, lB, strip, phi_m, bc_top, phi_b_top=0.0, surf=(0.0, 0.0), tol=1e-13):
    """Eq. poisson with a metal strip (Dirichlet patch, potential phi_m on
    its cells) inside a dielectric bottom wall (Neumann, surface charge
    surf[0]) and a top wall of type bc_top (Eqs. esbc1 / esbc3), by CG on the
    assembled operator.  The strip fixes the potential's constant, so no
    neutrality condition applies."""
    Nz, Ny, Nx = rho.shape
    dims = (Nx, Ny, Nz)
    A = assemble_strip(dims, bc_top, strip)
    slopes = wall_slopes((NEUMANN, bc_top), surf, lB)
    b = 4.0 * np.pi * lB * np.asarray(rho, dtype=np.float64).copy()
    b[:, 0, :] += np.where(strip, 2.0 * phi_m, -slopes[0])
    b[:, -1, :] += 2.0 * phi_b_top if bc_top == DIRICHLET else slopes[1]
    phi, info = spla.cg(A, b.ravel(), rtol=tol, atol=0.0, maxiter=20000)
    if info != 0:
        raise RuntimeError(f"CG did not converge (info={info})")
    return phi.reshape(Nz, Ny, Nx)
