"""Forces and the four-stage time step (Sec. II.D).

Test infrastructure only (see ``oracle/__init__``).

Parameters come in a plain dict `p` (reduced units: Delta r = 1, kT given,
eps = 1/(4 pi l_B)):
  dims (Nx, Ny, Nz); bc (bottom, top) 0 = Dirichlet, 1 = Neumann; phi_b;
  surf_charge; kernel_es, kernel_hy (kernels.Kernel); lB; eta; kT; dt; psi;
  fp_table; lj_sigma/lj_xi/lj_rc [ns][ns]; wall_sigma/wall_xi/wall_rc [ns];
  wall_type; E_ext (3,); gamma_coef [ns][2][2][7]; D_tot, D_wet [ns];
  wet, drift (bools); seed; slip (bottom, top) hydrodynamic slip walls;
  kernel_hy_species: None, or a list of per-species hydrodynamic kernels
  that replaces kernel_hy (App. B);
  strip (x0, x1, phi_total) or None.

Stage 1: rho = S^es q, Poisson (Eq. poisson).  Stage 2: E^P = J^es(-grad phi)
(Eq. efieldop), F = q E^P + near field (Eqs. fullElectro, LC) + LJ
(Eq. closerange) + wall + q E_ext (Eq. totalforce).  Stage 3: f = S^hy F +
f_th + stochastic stress, Stokes solve.  Stage 4: midpoint update
(Eqs. step1-step2) with the dry tensor of Eqs. diff1-diff2 and its Ito drift
(Eq. ions3).  A dry-only step (no hydrodynamic grid) is Euler-Maruyama on
Eq. ions3 with V = 0.
"""
import numpy as np

from . import gridops, poisson, particles, mobility, stokes, philox


def electrostatic_field(p, pos, q):
    """(rho, phi, E^P at the ions).  p['strip'] = (x0, x1, phi_total) puts a
    metal strip into the dielectric bottom wall (Sec. IV.B)."""
    dims = p['dims']
    strip = p.get('strip')
    rho = gridops.spread_charge(p['kernel_es'], pos, q, dims, p['bc'], strip)
    slopes = poisson.wall_slopes(p['bc'], p['surf_charge'], p['lB'])
    E_x = float(p['E_ext'][0])
    if strip is None:
        phi = poisson.solve(rho, p['bc'], p['lB'], p['phi_b'], p['surf_charge'])
    else:
        mask = poisson.strip_columns(dims, strip[0], strip[1])
        pm = poisson.strip_potential(dims, strip[0], strip[1], strip[2], E_x)
        phi = poisson.solve_strip(rho, p['lB'], mask, pm, p['bc'][1], p['phi_b'][1], p['surf_charge'])
    E = gridops.efield_at_ions(p['kernel_es'], pos, phi, p['bc'], p['phi_b'], slopes, strip, E_x)
    return rho, phi, E


def forces(p, pos, q, species, pair_dtype=np.float64):
    """Total force, Eq. totalforce.  Returns (F (3,N), counts, parts dict)."""
    rho, phi, E = electrostatic_field(p, pos, q)
    Fp = q[None, :] * E
    Fn, counts = particles.near_field(pos, q, species, p, p['fp_table'], pair_dtype)
    Fw = particles.wall_force(pos, species, p)
    F = Fp + Fn
    F[1] += Fw
    F += q[None, :] * np.asarray(p['E_ext'], dtype=np.float64)[:, None]
    return F, counts, dict(rho=rho, phi=phi, E=E, Fp=Fp, Fn=Fn, Fw=Fw)


def wrap_reflect(pos, dims):
    """Periodic wrap in x, z (one shift) and specular reflection at the walls."""
    Nx, Ny, Nz = dims
    x = pos.copy()
    for d, L in ((0, Nx), (2, Nz)):
        x[d] = np.where(x[d] < 0, x[d] + L, np.where(x[d] >= L, x[d] - L, x[d]))
    y = x[1]
    x[1] = np.where(y < 0, -y, np.where(y > Ny, 2.0 * Ny - y, y))
    return x


def dry_increment(p, pos, species, F, step, replica=0, first_index=0):
    """Dry part of Eq. ions3 over one step: dt (D Gamma F / kT + div D) +
    sqrt(2 dt D Gamma) W, W from Philox tag 1."""
    Ny = p['dims'][1]
    sp_ = np.asarray(species)
    Dd = (np.asarray(p['D_tot']) - np.asarray(p['D_wet']))[sp_]
    G, dGp = mobility.dry_tensor(pos[1], Ny, species, p)
    W = philox.ion_normals(pos.shape[1], step, replica, philox.TAG_DRY, p['seed'], first_index)
    inc = p['dt'] * (Dd[None, :] * G * F / p['kT'])
    if p.get('drift', True):
        inc[1] += p['dt'] * Dd * dGp
    inc += np.sqrt(2.0 * p['dt'] * Dd[None, :] * np.maximum(G, 0.0)) * W
    return inc


def dry_step(p, pos, q, species, step, pair_dtype=np.float64, replica=0):
    """One Euler-Maruyama step of the dry-diffusion dynamics (noise of the
    given replica's Philox stream)."""
    F, counts, parts = forces(p, pos, q, species, pair_dtype)
    new = wrap_reflect(pos + dry_increment(p, pos, species, F, step, replica), p['dims'])
    return new, F, counts


def spread_hy(p, pos, F, species):
    """S^hy F with the run's hydrodynamic kernel, or each species' own."""
    slip = p.get('slip', (False, False))
    ks = p.get('kernel_hy_species')
    if ks is None:
        return gridops.spread_force(p['kernel_hy'], pos, F, p['dims'], slip)
    return gridops.spread_force_species(ks, species, pos, F, p['dims'], slip)


def interp_hy(p, pos, u, v, w, species):
    """J^hy v with the run's hydrodynamic kernel, or each species' own."""
    slip = p.get('slip', (False, False))
    ks = p.get('kernel_hy_species')
    if ks is None:
        return gridops.interp_velocity(p['kernel_hy'], pos, u, v, w, slip)
    return gridops.interp_velocity_species(ks, species, pos, u, v, w, slip)


def fluid_forcing(p, pos, F, step, species=None):
    """f = S^hy F + f_th + stochastic stress (each optional by flags)."""
    dims = p['dims']
    slip = p.get('slip', (False, False))
    fx, fy, fz = spread_hy(p, pos, F, species)
    if p.get('drift', True) and p['kT'] > 0:
        ks = p.get('kernel_hy_species')
        tx, ty, tz = stokes.rfd_forcing(p['kernel_hy'] if ks is None else ks, pos, dims, p['kT'], step, 0,
                                        p['seed'], slip=slip, species=None if ks is None else species)
        fx, fy, fz = fx + tx, fy + ty, fz + tz
    if p['kT'] > 0:
        nx, ny, nz = stokes.noise_forcing(dims, p['eta'], p['kT'], p['dt'], step, 0, p['seed'], slip)
        fx, fy, fz = fx + nx, fy + ny, fz + nz
    fy = fy.copy()
    fy[:, 0, :] = 0.0
    fy[:, -1, :] = 0.0
    return fx, fy, fz


def wet_increment(p, pos, species, F, step):
    """Stages 3 and 4 of Sec. II.D for given forces F: the fluid forcing
    (spread forces, RFD thermal forcing, stochastic stress), the Stokes solve,
    and the midpoint update of Eqs. step1-step2 (V = J(x*) v with
    x* = x + dt/2 J(x) v) plus the dry part of Eq. ions3.  With p['drift']
    false the RFD term is left out and the update is single stage (V = J(x) v).
    Returns (increment (3, N), fluid fields dict)."""
    slip = p.get('slip', (False, False))
    fx, fy, fz = fluid_forcing(p, pos, F, step, species)
    u, v, w, pr = stokes.solve(fx, fy, fz, p['eta'], slip=slip)
    V1 = interp_hy(p, pos, u, v, w, species)
    if p.get('drift', True):
        xs = pos + 0.5 * p['dt'] * V1
        V = interp_hy(p, xs, u, v, w, species)
    else:
        V = V1
    inc = p['dt'] * V + dry_increment(p, pos, species, F, step)
    return inc, dict(u=u, v=v, w=w, p=pr, V1=V1, V=V)


def wet_step(p, pos, q, species, step, pair_dtype=np.float64):
    """One step of the four-stage algorithm with the midpoint scheme."""
    F, counts, parts = forces(p, pos, q, species, pair_dtype)
    inc, fluid = wet_increment(p, pos, species, F, step)
    new = wrap_reflect(pos + inc, p['dims'])
    return new, F, counts, dict(parts, **fluid)
