"""Test-side glue: the same run parameters handed to the CUDA path (RunConfig)
and to the oracle (a plain dict), plus comparison helpers."""
import numpy as np

from oracle import kernels as okernels, greens as ogreens


def oracle_params(cfg):
    return dict(
        dims=cfg.dims, bc=tuple(cfg.bc), phi_b=tuple(cfg.phi_b), surf_charge=tuple(cfg.surf_charge),
        kernel_es=okernels.Kernel(cfg.kernel_es, cfg.es_w[0], cfg.es_beta[0]),
        kernel_hy=okernels.Kernel(cfg.kernel_hy, cfg.es_w[1], cfg.es_beta[1]),
        lB=cfg.lB, eta=cfg.eta, kT=cfg.kT, dt=cfg.dt, psi=cfg.psi,
        fp_table=ogreens.fp_table(cfg.kernel_es, cfg.psi, cfg.n_tab, cfg.es_w[0], cfg.es_beta[0]),
        lj_sigma=cfg.lj_sigma, lj_xi=cfg.lj_xi, lj_rc=cfg.lj_rc,
        wall_sigma=cfg.wall_sigma, wall_xi=cfg.wall_xi, wall_rc=cfg.wall_rc, wall_type=cfg.wall_type,
        E_ext=tuple(cfg.E_ext), gamma_coef=cfg.gamma_coef, D_tot=cfg.D_tot, D_wet=cfg.D_wet,
        wet=bool(cfg.wet), drift=bool(cfg.drift), seed=cfg.seed,
        strip=(float(cfg.strip_x[0]), float(cfg.strip_x[1]), float(cfg.strip_phi)) if cfg.strip else None,
        slip=(bool(cfg.bc_hy[0]), bool(cfg.bc_hy[1])),
        kernel_hy_species=([okernels.Kernel(cfg.kernel_hy_s[s], cfg.hy_w_s[s], cfg.hy_beta_s[s])
                            for s in range(cfg.nspecies)] if cfg.hy_species else None))


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def min_image_disp(new, old, dims):
    """Displacement new - old with periodic wrap undone in x and z."""
    d = np.asarray(new, dtype=np.float64) - np.asarray(old, dtype=np.float64)
    for ax, L in ((0, dims[0]), (2, dims[2])):
        d[ax] = d[ax] - L * np.round(d[ax] / L)
    return d


def mac_split(flat, dims):
    """Split a flat u|v|w face buffer into (u, v, w) arrays."""
    Nx, Ny, Nz = dims
    G = Nx * Ny * Nz
    Gv = Nx * (Ny + 1) * Nz
    f = np.asarray(flat, dtype=np.float64)
    return f[:G].reshape(Nz, Ny, Nx), f[G:G + Gv].reshape(Nz, Ny + 1, Nx), f[G + Gv:].reshape(Nz, Ny, Nx)


def mac_join(u, v, w):
    return np.concatenate([np.ravel(u), np.ravel(v), np.ravel(w)])
