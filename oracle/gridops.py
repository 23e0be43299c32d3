"""Spreading and interpolation between ions and the staggered grid.

Test infrastructure only (see ``oracle/__init__``).

Geometry (grid spacing 1, cell volume 1): x in [0, Nx) and z in [0, Nz)
periodic, walls at y = 0 and y = Ny.  Arrays are indexed [k][j][i] (z, y, x).

  cell centres   (i+1/2, j+1/2, k+1/2)   shape (Nz, Ny,   Nx)
  x-faces        (i,     j+1/2, k+1/2)   shape (Nz, Ny,   Nx)
  y-faces        (i+1/2, j,     k+1/2)   shape (Nz, Ny+1, Nx)   j = 0..Ny
  z-faces        (i+1/2, j+1/2, k    )   shape (Nz, Ny,   Nx)

Spreading (Eq. kernel2) near a wall follows the image construction of Sec.
II.A (Fig. folded) and Sec. II.B.1: the ion spreads its value, and its mirror
image across each wall (y -> -y, y -> 2 Ny - y) spreads sign * value, each
restricted to the grid points inside the domain.  The sign is -1 for the
normal hydrodynamic component and for no-slip tangential components, +1 for
slip tangential components; for charge it is -1 at a Dirichlet (fixed
potential) wall and +1 at a Neumann (dielectric) wall.

Interpolation (Eq. kernel1) fills ghost layers outside the domain so that the
boundary condition holds, then interpolates exactly as in the interior.
"""
import numpy as np

CELL, FACE = 0, 1     # y-placement of the grid points: centres or faces


def _axis_points(kernel, s):
    idx, wts = kernel.stencil(s)
    return idx, wts


def spread(kernel, pos, vals, shape, offs, ytype, signs, bottom_cols=None):
    """Spread vals[n] at positions pos[:, n] onto a grid of shape (Nz, Ny', Nx).

    offs = (ox, oy, oz): coordinate of grid point 0 along each axis (1/2 for
    cell-centred axes, 0 for face axes).  ytype: CELL (Ny points) or FACE
    (Ny+1 points).  signs = (s_bottom, s_top) for the two wall images;
    bottom_cols (Nx,), if given, replaces s_bottom by a sign per grid column
    (a wall made of parts of different kinds).
    Returns the spread density (the kernel carries the 1/Delta V factor).
    """
    Nz, Nyg, Nx = shape
    Ny = Nyg if ytype == CELL else Nyg - 1
    grid = np.zeros(shape)
    pos = np.asarray(pos, dtype=np.float64)
    vals = np.asarray(vals, dtype=np.float64)
    images = [(pos[1], 1.0), (-pos[1], signs[0]), (2.0 * Ny - pos[1], signs[1])]
    ix, wx = kernel.stencil(pos[0] - offs[0])
    iz, wz = kernel.stencil(pos[2] - offs[2])
    ix %= Nx
    iz %= Nz
    w = kernel.w
    for m, (ypos, sgn) in enumerate(images):
        iy, wy = kernel.stencil(ypos - offs[1])
        valid = (iy >= 0) & (iy < Nyg)
        wyv = np.where(valid, wy, 0.0)
        iyc = np.clip(iy, 0, Nyg - 1)
        # (n, w, w, w) contributions, axes (z, y, x)
        contrib = (sgn * vals)[:, None, None, None] * wz[:, :, None, None] \
            * wyv[:, None, :, None] * wx[:, None, None, :]
        if m == 1 and bottom_cols is not None:
            contrib = contrib / sgn * np.asarray(bottom_cols)[ix][:, None, None, :]
        K = np.broadcast_to(iz[:, :, None, None], contrib.shape)
        J = np.broadcast_to(iyc[:, None, :, None], contrib.shape)
        I = np.broadcast_to(ix[:, None, None, :], contrib.shape)
        np.add.at(grid, (K.ravel(), J.ravel(), I.ravel()), contrib.ravel())
    return grid


def extend_y(grid, ytype, ghost, bottom, top):
    """Add `ghost` layers on both y sides, filled by affine reflection rules.

    bottom/top: (sign, offset_fn) where the ghost value is
        sign * grid[mirror] + offset_fn(m)
    and m = 0, 1, ... counts ghost layers away from the wall.  Mirrors: for
    CELL, ghost cell -1-m <-> cell m (top: Ny+m <-> Ny-1-m); for FACE, ghost
    face -m-1 <-> face m+1 (top: Ny+1+m <-> Ny-1-m), the wall faces being
    grid points.
    Returns the extended array and the index of original point 0 in it.
    """
    Nz, Nyg, Nx = grid.shape
    ext = np.zeros((Nz, Nyg + 2 * ghost, Nx))
    ext[:, ghost:ghost + Nyg, :] = grid
    sb, ob = bottom
    st, ot = top
    for m in range(ghost):
        if ytype == CELL:
            mb, mt = m, Nyg - 1 - m
        else:
            mb, mt = m + 1, Nyg - 2 - m
        ext[:, ghost - 1 - m, :] = sb * grid[:, mb, :] + ob(m)
        ext[:, ghost + Nyg + m, :] = st * grid[:, mt, :] + ot(m)
    return ext, ghost


def interpolate(kernel, pos, grid_ext, y0, offs):
    """Interpolate an already ghost-extended grid at positions pos.

    grid_ext has its original y-point 0 at extended index y0.  Returns the
    values Delta V * sum_j delta(x - r_j) g_j (Delta V = 1).
    """
    Nz, Nye, Nx = grid_ext.shape
    pos = np.asarray(pos, dtype=np.float64)
    ix, wx = kernel.stencil(pos[0] - offs[0])
    iy, wy = kernel.stencil(pos[1] - offs[1])
    iz, wz = kernel.stencil(pos[2] - offs[2])
    ix %= Nx
    iz %= Nz
    iy = iy + y0
    if iy.min() < 0 or iy.max() >= Nye:
        raise ValueError("interpolation stencil leaves the ghost layers")
    g = grid_ext[iz[:, :, None, None], iy[:, None, :, None], ix[:, None, None, :]]
    return np.einsum('nk,nj,ni,nkji->n', wz, wy, wx, g)


# ---------------------------------------------------------------- electrostatics
DIRICHLET, NEUMANN = 0, 1


def charge_signs(bc):
    """Image charge sign per wall (Sec. II.B.1): opposite at a Dirichlet wall,
    like at a Neumann wall."""
    return tuple(-1.0 if b == DIRICHLET else 1.0 for b in bc)


def strip_cols(dims, strip):
    """Bool (Nx,): the bottom cell columns under a metal strip (centre in [x0, x1))."""
    xc = np.arange(dims[0]) + 0.5
    return (xc >= strip[0]) & (xc < strip[1])


def spread_charge(kernel, pos, q, dims, bc, strip=None):
    """Charge density rho = S^es q on cell centres with wall images.  With a
    metal strip (x0, x1, phi) in the dielectric bottom wall, the bottom image
    takes the conducting wall's sign (-1) in the strip's columns (reading:
    the image follows the kind of wall under each grid column)."""
    Nx, Ny, Nz = dims
    cols = None
    if strip is not None:
        cols = np.where(strip_cols(dims, strip), -1.0, 1.0)
    return spread(kernel, pos, q, (Nz, Ny, Nx), (0.5, 0.5, 0.5), CELL, charge_signs(bc), cols)


def phi_ghost_rules(bc, phi_b, dphidy):
    """Ghost-cell rules for phi that satisfy Eqs. esbc1/esbc3.

    Dirichlet: phi(-1-m) = 2 phi_b - phi(m) (odd about phi_b on the wall face).
    Neumann:   phi(-1-m) = phi(m) - g (2m + 1), g = dphi/dy on the wall, i.e.
    the reflection of phi - g y; at the top wall phi(Ny+m) = phi(Ny-1-m) +
    g_top (2m + 1).
    """
    rules = []
    for w in range(2):
        if bc[w] == DIRICHLET:
            pb = phi_b[w]
            rules.append((-1.0, (lambda m, pb=pb: 2.0 * pb)))
        else:
            g = dphidy[w]
            if w == 0:
                rules.append((1.0, (lambda m, g=g: -g * (2 * m + 1))))
            else:
                rules.append((1.0, (lambda m, g=g: g * (2 * m + 1))))
    return rules


def efield_at_ions(kernel, pos, phi, bc, phi_b, dphidy, strip=None, E_x=0.0):
    """E^P = J^es(-grad_h phi) (Eq. efieldop) with E on cell faces.

    phi is extended with ghost cells (phi_ghost_rules), E = -(phi_i - phi_{i-1})
    is formed on every face of the extended grid, and each component is
    interpolated with the kernel centred at its own face positions.  With a
    metal strip (x0, x1, phi_total) in the bottom wall, the ghost cells below
    the strip's columns follow the Dirichlet rule with phi_m(x) = phi_total +
    E_x (x - x_c) (see poisson.strip_potential).
    Returns E, shape (3, N).
    """
    Nz, Ny, Nx = phi.shape
    ghost = kernel.w // 2 + 3
    rb, rt = phi_ghost_rules(bc, phi_b, dphidy)
    ext, y0 = extend_y(phi, CELL, ghost, rb, rt)
    if strip is not None:
        on = strip_cols((Nx, Ny, Nz), strip)
        xc = np.arange(Nx) + 0.5
        pm = strip[2] + E_x * (xc - 0.5 * (strip[0] + strip[1]))
        for m in range(ghost):
            ext[:, ghost - 1 - m, on] = 2.0 * pm[on][None, :] - phi[:, m, :][:, on]
    Ex = -(ext - np.roll(ext, 1, axis=2))          # x-face i: phi_i - phi_{i-1}
    Ez = -(ext - np.roll(ext, 1, axis=0))
    Ey = np.zeros_like(ext)                          # y-face at ext index j: phi_j - phi_{j-1}
    Ey[:, 1:, :] = -(ext[:, 1:, :] - ext[:, :-1, :])
    ex = interpolate(kernel, pos, Ex, y0, (0.0, 0.5, 0.5))
    ez = interpolate(kernel, pos, Ez, y0, (0.5, 0.5, 0.0))
    # extended index j of Ey is the face at y = j - y0
    ey = interpolate(kernel, pos, Ey, y0, (0.5, 0.0, 0.5))
    return np.stack([ex, ey, ez])


# ---------------------------------------------------------------- hydrodynamics
NOSLIP = 0


def spread_force(kernel, pos, F, dims, slip=(False, False)):
    """Hydrodynamic spreading S^hy F (Eq. kernel2) per MAC component with the
    image construction of Sec. II.A: opposite normal force at every wall;
    opposite tangential force at a no-slip wall, the same at a slip wall.
    Returns (fx on x-faces, fy on y-faces incl. walls, fz on z-faces)."""
    Nx, Ny, Nz = dims
    s = (-1.0, -1.0)
    st = tuple(1.0 if sl else -1.0 for sl in slip)
    fx = spread(kernel, pos, F[0], (Nz, Ny, Nx), (0.0, 0.5, 0.5), CELL, st)
    fy = spread(kernel, pos, F[1], (Nz, Ny + 1, Nx), (0.5, 0.0, 0.5), FACE, s)
    fz = spread(kernel, pos, F[2], (Nz, Ny, Nx), (0.5, 0.5, 0.0), CELL, st)
    return fx, fy, fz


def spread_force_species(kernels, species, pos, F, dims, slip=(False, False)):
    """S^hy F with a hydrodynamic kernel per species (App. B: one kernel for
    the cations, another for the anions, on one grid): every ion spreads with
    its own species' kernel, and the grid holds the sum."""
    Nx, Ny, Nz = dims
    species = np.asarray(species)
    out = (np.zeros((Nz, Ny, Nx)), np.zeros((Nz, Ny + 1, Nx)), np.zeros((Nz, Ny, Nx)))
    for s, kernel in enumerate(kernels):
        m = species == s
        if m.any():
            part = spread_force(kernel, pos[:, m], F[:, m], dims, slip)
            out = tuple(a + b for a, b in zip(out, part))
    return out


def interp_velocity(kernel, pos, u, v, w, slip=(False, False)):
    """V = J^hy v (Eq. kernel1) with ghost fill from the wall conditions:
    tangential ghosts are the negated mirror values at a no-slip wall and the
    mirror values at a slip wall, normal ghosts the negated mirror values;
    the wall faces carry v = 0."""
    ghost = kernel.w // 2 + 3
    zero = (lambda m: 0.0)
    tb, tt = (1.0 if slip[0] else -1.0), (1.0 if slip[1] else -1.0)
    ue, y0 = extend_y(u, CELL, ghost, (tb, zero), (tt, zero))
    we, _ = extend_y(w, CELL, ghost, (tb, zero), (tt, zero))
    ve, y0v = extend_y(v, FACE, ghost, (-1.0, zero), (-1.0, zero))
    Vx = interpolate(kernel, pos, ue, y0, (0.0, 0.5, 0.5))
    Vy = interpolate(kernel, pos, ve, y0v, (0.5, 0.0, 0.5))
    Vz = interpolate(kernel, pos, we, y0, (0.5, 0.5, 0.0))
    return np.stack([Vx, Vy, Vz])


def interp_velocity_species(kernels, species, pos, u, v, w, slip=(False, False)):
    """J^hy v with a hydrodynamic kernel per species (App. B): every ion
    interpolates with its own species' kernel."""
    species = np.asarray(species)
    V = np.zeros((3, pos.shape[1]))
    for s, kernel in enumerate(kernels):
        m = species == s
        if m.any():
            V[:, m] = interp_velocity(kernel, pos[:, m], u, v, w, slip)
    return V
