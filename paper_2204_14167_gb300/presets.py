"""Workload presets: synthetic channels shaped like the paper's runs.

Each preset returns (RunConfig, ion recipe).  Reduced units: grid spacing 1,
kT = 1.  The near-field cutoff psi = 4 is where the grid pair force of the
4- and 6-point kernels has reached Coulomb to within 0.7%.
"""
import math

from . import RunConfig, BC_DIRICHLET, BC_NEUMANN, KERNEL_PESKIN4, KERNEL_PESKIN6, KERNEL_ES, FP64, MIXED
from . import mobility

WCA = 2.0 ** (1.0 / 6.0)
# Hydrodynamic radii in grid units of the 4-point kernel and of the two ES
# kernels of App. B (cations: w = 7, beta = 7; anions: w = 4, beta = 8),
# measured with this library's own Stokes solver (Sec. III.A): the
# mid-channel perpendicular mobility of one particle (8 sub-cell offsets,
# FP64) in a 128^3 no-slip channel, matched to Eq. mob_analytic by
# calibrate.hydrodynamic_radius (64^3 gives the same to 0.2 %).
A_WET_PESKIN4 = 1.25
A_WET_ES77 = 2.08
A_WET_ES48 = 1.08


def _wca(sigma):
    return dict(lj_sigma=[[sigma]], lj_xi=[[1.0]], lj_rc=[[WCA * sigma]])


def _wall():
    # repulsive 12-6 wall cut at 1 cell (sigma = 2^-1/6)
    return dict(wall_sigma=[2.0 ** (-1.0 / 6.0)], wall_xi=[1.0], wall_rc=[1.0])


def dry_channel_32(precision=FP64):
    """32^3 channel, Dirichlet phi = 0 walls, 128 + 128 ions, l_B = 7,
    6-point kernel, dry diffusion (D = 1).  dt = 0.001: explicit
    Euler-Maruyama needs dt D U''(r) < 1 at WCA contact, U''(0.9 sigma) ~ 560
    kT per cell^2 for sigma = 3; at dt = 0.01 a 512-ion channel of this kind
    blows up within a few steps (the oracle does the same)."""
    gam = mobility.gamma_table(1.0, 1.0, 32.0)
    cfg = RunConfig(Nx=32, Ny=32, Nz=32, bc=(BC_DIRICHLET, BC_DIRICHLET), kernel_es=KERNEL_PESKIN6,
                    kernel_hy=KERNEL_PESKIN6, lB=7.0, dt=0.001, psi=4.0, n_tab=64, D_tot=[1.0], D_wet=[0.0],
                    gamma_coef=[gam], wet=False, precision=precision, max_ions=256, **_wca(3.0), **_wall())
    return cfg, dict(n_pos=128, n_neg=128, ymargin=1.0, min_sep=0.9 * 3.0, seed=20220429)


def wet_channel_128x64x128(precision=MIXED):
    """128 x 64 x 128 channel with dielectric (Neumann) walls, 10k + 10k ions,
    Debye length ~4 cells (l_B = 0.261), E_x = 0.05, fluctuating Stokes with
    no-slip walls, 50% wet (4-point kernel, a_w = 1.25, a_t = a_w / 2).
    dt = 0.001 keeps D_tot dt / a_t^2 ~ 0.01, the paper's ratio of time step
    to diffusive time (Sec. III.C)."""
    Ny = 64
    eta = 1.0 / (6.0 * math.pi)
    D_wet = 1.0 / A_WET_PESKIN4            # kT / (6 pi eta a_w)
    D_tot = 2.0 * D_wet                    # a_t = a_w / 2
    gam = mobility.gamma_table(0.5 * A_WET_PESKIN4, A_WET_PESKIN4, float(Ny))
    cfg = RunConfig(Nx=128, Ny=Ny, Nz=128, bc=(BC_NEUMANN, BC_NEUMANN), kernel_es=KERNEL_PESKIN4,
                    kernel_hy=KERNEL_PESKIN4, lB=0.261, eta=eta, kT=1.0, dt=0.001, psi=4.0, n_tab=64,
                    D_tot=[D_tot], D_wet=[D_wet], gamma_coef=[gam], E_ext=(0.05, 0.0, 0.0), wet=True,
                    precision=precision, max_ions=20000, **_wca(1.0), **_wall())
    return cfg, dict(n_pos=10000, n_neg=10000, ymargin=1.0, min_sep=0.9, seed=20220430)


def wet_channel_small(precision=MIXED, Nx=32, Ny=16, Nz=16, n=300):
    """Small wet channel with the same physics as wet_channel_128x64x128, for
    tests the oracle finishes in seconds."""
    cfg, rec = wet_channel_128x64x128(precision)
    cfg.Nx, cfg.Ny, cfg.Nz = Nx, Ny, Nz
    cfg.gamma_coef = [mobility.gamma_table(0.5 * A_WET_PESKIN4, A_WET_PESKIN4, float(Ny))]
    cfg.max_ions = max(n, 1)
    rec = dict(rec, n_pos=n // 2, n_neg=n - n // 2)
    return cfg, rec


def energy_channel_64(precision=FP64):
    """64^3 channel between Dirichlet walls at phi = +0.5 and -0.5, 2048 +
    2048 ions placed uniformly in y in [1, 63], l_B = 7, 6-point kernel:
    the workload of the differentiable energy (forward U and its adjoint)."""
    cfg = RunConfig(Nx=64, Ny=64, Nz=64, bc=(BC_DIRICHLET, BC_DIRICHLET), phi_b=(0.5, -0.5),
                    kernel_es=KERNEL_PESKIN6, kernel_hy=KERNEL_PESKIN6, lB=7.0, dt=0.01, psi=4.0, n_tab=64,
                    D_tot=[1.0], D_wet=[0.0], gamma_coef=[mobility.gamma_table(1.0, 1.0, 64.0)], wet=False,
                    precision=precision, max_ions=4096, **_wca(1.0), **_wall())
    return cfg, dict(n_pos=2048, n_neg=2048, ymargin=1.0, min_sep=0.0, seed=20220501)


def iceo_channel_256x128x256(precision=MIXED):
    """256 x 128 x 256 channel, conducting (Dirichlet phi = 0) bottom wall and
    dielectric (Neumann, no surface charge) top wall, 200k + 200k ions
    uniform in y in [1, 127] and at least 0.9 sigma apart, l_B = 0.96, ion
    WCA sigma = 0.6, E_x = 0.02, dt = 5e-5 (stable at WCA contact),
    the full wet step of the 128 x 64 x 128 channel (fluctuating Stokes,
    thermal drift, near-wall mobility)."""
    cfg, rec = wet_channel_128x64x128(precision)
    Ny = 128
    cfg.Nx, cfg.Ny, cfg.Nz = 256, Ny, 256
    cfg.bc = (BC_DIRICHLET, BC_NEUMANN)
    cfg.phi_b = (0.0, 0.0)
    cfg.surf_charge = (0.0, 0.0)
    cfg.lB = 0.96
    cfg.E_ext = (0.02, 0.0, 0.0)
    cfg.gamma_coef = [mobility.gamma_table(0.5 * A_WET_PESKIN4, A_WET_PESKIN4, float(Ny))]
    cfg.max_ions = 400000
    # explicit Euler-Maruyama is stable near WCA contact for dt D_tot U''(r) < 1;
    # at the placement minimum r = 0.9 sigma = 0.54, U'' ~ 6500 kT per cell^2,
    # and with D_tot = 2 / a_w = 1.6 this gives dt = 5e-5 (0.5)
    cfg.dt = 5e-5
    for k, v in _wca(0.6).items():
        setattr(cfg, k, v)
    return cfg, dict(n_pos=200000, n_neg=200000, ymargin=1.0, min_sep=0.9 * 0.6, seed=20220503)


def iceo_strip_256x128x256(precision=MIXED):
    """The 256 x 128 x 256 channel in the paper's ICEO geometry (Sec. IV.B,
    Fig. EOgeometry): both walls dielectric (Neumann, no surface charge) and a
    metal strip centred in the bottom wall, its width the paper's ratio
    L_m / P_x = 5.272 / 26.36 = 0.2 of the box (51.2 cells), held at total
    potential 0 (phi + phi_E constant on the metal under E_x = 0.02); ions,
    physics and time step as iceo_channel_256x128x256."""
    cfg, rec = iceo_channel_256x128x256(precision)
    cfg.bc = (BC_NEUMANN, BC_NEUMANN)
    cfg.strip = True
    w = 0.2 * cfg.Nx
    cfg.strip_x = (0.5 * (cfg.Nx - w), 0.5 * (cfg.Nx + w))
    cfg.strip_phi = 0.0
    return cfg, dict(rec, seed=rec["seed"] + 7)


def batched_channels_32(R=512, precision=MIXED, seed=20220502):
    """R independent replicas of dry_channel_32's channel (Dirichlet phi = 0
    walls, l_B = 7, 6-point kernel, dt = 0.001), replica r holding an even,
    charge-neutral number of ions drawn uniformly in [64, 512]."""
    import numpy as np
    cfg, rec = dry_channel_32(precision)
    cfg.max_ions = 512
    counts = 2 * np.random.default_rng(seed).integers(32, 257, size=R)
    return cfg, dict(rec, counts=[int(c) for c in counts], seed=seed)


def batched_ions(cfg, rec):
    """Packed ions of a batched preset: (pos (3, Ntot), q, species, offsets)."""
    import numpy as np
    from . import synth
    pos, q, sp, off = [], [], [], [0]
    for r, n in enumerate(rec["counts"]):
        p_, q_, s_ = synth.ions(cfg.dims, n // 2, n - n // 2, rec["seed"] + 1 + r, rec["ymargin"], rec["min_sep"])
        pos.append(p_); q.append(q_); sp.append(s_)
        off.append(off[-1] + n)
    return np.concatenate(pos, axis=1), np.concatenate(q), np.concatenate(sp), off


def eo_two_species(precision=MIXED, Nx=64, Ny=56, Nz=64, n_pos=6400, n_neg=5600):
    """Electro-osmotic channel of Sec. IV.A with a hydrodynamic kernel per
    species (App. B): cations spread and interpolate with the ES kernel of
    w = 7, beta = 7, anions with w = 4, beta = 8, on one hydrodynamic grid;
    the 4-point kernel for the electrostatics.  Dielectric walls carry the
    same surface charge, which balances the excess of cations (the channel
    is neutral); E_x = 0.05; 85 % wet (Sec. IV.A runs 85 % wet on a coarser
    grid); no-slip fluctuating Stokes with the midpoint scheme.  The paper's
    grid is 56^3; x and z are powers of two here (64)."""
    eta = 1.0 / (6.0 * math.pi)
    radii = (A_WET_ES77, A_WET_ES48)
    D_wet = [1.0 / a for a in radii]              # kT / (6 pi eta a_w)
    D_tot = [d / 0.85 for d in D_wet]
    gam = [mobility.gamma_table(0.85 * a, a, float(Ny)) for a in radii]
    net = n_pos - n_neg
    sigma_s = -net / (2.0 * Nx * Nz)
    cfg = RunConfig(Nx=Nx, Ny=Ny, Nz=Nz, bc=(BC_NEUMANN, BC_NEUMANN), surf_charge=(sigma_s, sigma_s),
                    kernel_es=KERNEL_PESKIN4, kernel_hy=KERNEL_ES, es_w=(6, 7), es_beta=(8.0, 7.0),
                    lB=0.5, eta=eta, kT=1.0, dt=0.001, psi=4.0, n_tab=64, nspecies=2, D_tot=D_tot, D_wet=D_wet,
                    gamma_coef=gam, E_ext=(0.05, 0.0, 0.0), wet=True, precision=precision,
                    max_ions=n_pos + n_neg, hy_species=True, kernel_hy_s=[KERNEL_ES, KERNEL_ES], hy_w_s=[7, 4],
                    hy_beta_s=[7.0, 8.0], lj_sigma=[[1.0, 1.0], [1.0, 1.0]], lj_xi=[[1.0, 1.0], [1.0, 1.0]],
                    lj_rc=[[WCA, WCA], [WCA, WCA]], wall_sigma=[2.0 ** (-1.0 / 6.0)] * 2, wall_xi=[1.0, 1.0],
                    wall_rc=[1.0, 1.0])
    return cfg, dict(n_pos=n_pos, n_neg=n_neg, ymargin=1.0, min_sep=0.9, seed=20220504)


def eo_two_species_small(precision=MIXED, Nx=32, Ny=16, Nz=32, n=300):
    """eo_two_species on a grid the oracle finishes in seconds (n ions, a
    cation excess of n / 15 balanced by the walls' surface charge)."""
    n_neg = (n - n // 15) // 2
    return eo_two_species(precision, Nx, Ny, Nz, n - n_neg, n_neg)


def species_by_charge(q):
    """Species of each ion for the two-species presets: 0 cation, 1 anion."""
    import numpy as np
    return (np.asarray(q) < 0).astype(np.int32)


PRESETS = {
    "dry_channel_32": dry_channel_32,
    "wet_channel_128x64x128": wet_channel_128x64x128,
    "energy_channel_64": energy_channel_64,
    "iceo_channel_256x128x256": iceo_channel_256x128x256,
    "iceo_strip_256x128x256": iceo_strip_256x128x256,
    "eo_two_species": eo_two_species,
}
