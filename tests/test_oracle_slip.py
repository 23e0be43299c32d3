"""Pins of the oracle's slip walls (Eq. fluidbc with a slip condition:
zero normal velocity and zero shear stress; Sec. II.A's images with a like
tangential image), each against what the mathematics fixes:

* discrete fluctuation-dissipation: the stochastic stress divergence D with
  the wall-edge stress switched off at a slip wall satisfies
  D D^T = L + Div^T Div exactly, L the viscous operator with the slip rows;
* a uniform body force between a slip wall (y = 0) and a no-slip wall
  (y = L) gives the half-Poiseuille profile f (L^2 - y^2) / (2 eta), reached
  at second order;
* the spreading and interpolation with slip images are adjoint
  (Eq. adjoint: <S F, v> = <F, J v>);
* the solve is divergence free and self-adjoint with a slip wall.
"""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import gridops, kernels, stokes


def test_fdt_with_a_slip_wall():
    Nx, Ny, Nz = 4, 4, 3
    shapes = [(Nz, Ny, Nx)] * 3 + [(Nz, Ny + 1, Nx), (Nz, Ny, Nx), (Nz, Ny + 1, Nx)]
    for slip in ((True, False), (False, True)):
        cols = []
        for c, shp in enumerate(shapes):
            for e in range(int(np.prod(shp))):
                Z = [np.zeros(s) for s in shapes]
                Z[c].flat[e] = 1.0
                if c < 3:
                    Z[c] *= np.sqrt(2)
                if c in (3, 5):
                    Z[c][:, 0, :] *= 0.0 if slip[0] else np.sqrt(2)
                    Z[c][:, Ny, :] *= 0.0 if slip[1] else np.sqrt(2)
                dx, dy, dz = stokes.stress_divergence(*Z)
                cols.append(np.concatenate([dx.ravel(), dy[:, 1:Ny, :].ravel(), dz.ravel()]))
        D = np.array(cols).T
        Lu, Lv, Lw, Gx, Gy, Gz = stokes._ops((Nx, Ny, Nz), slip)
        L = sp.block_diag([Lu, Lv, Lw]).toarray()
        G = sp.vstack([Gx, Gy, Gz]).toarray()
        assert np.abs(D @ D.T - (L + G @ G.T)).max() < 1e-13
        # the drawn stress has no shear on the slip wall's edges
        Zs = stokes.stress_fields((Nx, Ny, Nz), 2, 0, 5, slip)
        w = 0 if slip[0] else Ny
        assert np.all(Zs[3][:, w, :] == 0.0) and np.all(Zs[5][:, w, :] == 0.0)


def test_half_poiseuille_second_order():
    errs = []
    for Ny in (8, 16):
        Nx = Nz = 4
        h = 1.0 / Ny
        fx = np.ones((Nz, Ny, Nx)) * h ** 2
        u, v, w, pr = stokes.solve(fx, np.zeros((Nz, Ny + 1, Nx)), np.zeros((Nz, Ny, Nx)), 1.0, slip=(True, False))
        y = (np.arange(Ny) + 0.5) * h
        exact = (1.0 - y ** 2) / 2.0
        errs.append(np.abs(u[0, :, 0] - exact).max())
        assert np.abs(v).max() < 1e-12 and np.abs(w).max() < 1e-12
    assert errs[0] < 1e-2 and 3.5 < errs[0] / errs[1] < 4.5


@pytest.mark.parametrize("kind", [kernels.PESKIN4, kernels.PESKIN6])
def test_slip_images_adjoint(kind):
    dims = (8, 8, 8)
    Nx, Ny, Nz = dims
    rng = np.random.default_rng(11)
    N = 30
    pos = np.stack([rng.uniform(0, Nx, N), rng.uniform(0, Ny, N), rng.uniform(0, Nz, N)])
    pos[1, :6] = rng.uniform(0, 1.2, 6)
    F = rng.normal(size=(3, N))
    u, w = rng.normal(size=(Nz, Ny, Nx)), rng.normal(size=(Nz, Ny, Nx))
    v = rng.normal(size=(Nz, Ny + 1, Nx))
    v[:, 0] = v[:, Ny] = 0.0
    k = kernels.Kernel(kind)
    for slip in ((True, False), (False, True), (True, True)):
        f = gridops.spread_force(k, pos, F, dims, slip)
        V = gridops.interp_velocity(k, pos, u, v, w, slip)
        lhs = sum(np.sum(a * b) for a, b in zip(f, (u, v, w)))
        assert abs(lhs - np.sum(F * V)) < 1e-12 * abs(lhs)
    # like tangential images: the folded kernel keeps its partition of unity,
    # so the spread tangential force is conserved next to slip walls (and is
    # not next to no-slip walls, whose images are opposite)
    fs = gridops.spread_force(k, pos, F, dims, (True, True))
    fn = gridops.spread_force(k, pos, F, dims, (False, False))
    for c in (0, 2):
        assert abs(fs[c].sum() - F[c].sum()) < 1e-12 * np.abs(F[c]).sum()
        assert abs(fn[c].sum() - F[c].sum()) > 1e-3 * np.abs(F[c]).sum()


def test_slip_solve_divergence_free_and_self_adjoint():
    rng = np.random.default_rng(6)
    Nx, Ny, Nz = 6, 8, 4
    f = [rng.normal(size=(Nz, Ny, Nx)), rng.normal(size=(Nz, Ny + 1, Nx)), rng.normal(size=(Nz, Ny, Nx))]
    g = [rng.normal(size=(Nz, Ny, Nx)), rng.normal(size=(Nz, Ny + 1, Nx)), rng.normal(size=(Nz, Ny, Nx))]
    for a in (f, g):
        a[1][:, 0, :] = 0; a[1][:, Ny, :] = 0
    for slip in ((True, False), (False, True)):
        u1 = stokes.solve(*f, eta=0.8, slip=slip)
        u2 = stokes.solve(*g, eta=0.8, slip=slip)
        assert np.abs(stokes.divergence(*u1[:3])).max() < 1e-12
        lhs = sum(np.sum(a * b) for a, b in zip(f, u2[:3]))
        rhs = sum(np.sum(a * b) for a, b in zip(u1[:3], g))
        assert abs(lhs - rhs) < 1e-11 * abs(lhs)
        (rx, ry, rz), div = stokes.residual(*u1, *f, 0.8, slip=slip)
        assert np.sqrt(sum(np.sum(r ** 2) for r in (rx, ry, rz))) < 1e-10 * np.sqrt(sum(np.sum(a ** 2) for a in f))
    with pytest.raises(ValueError):
        stokes.solve(*f, eta=0.8, slip=(True, True))
