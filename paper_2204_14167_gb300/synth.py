"""Seeded synthetic ion configurations (input generation only; none of the
method's arithmetic lives here).

Ions are +1 / -1 point charges placed uniformly at random in the channel
(x, z over the periodic box, y at least `ymargin` from each wall); with
`min_sep` > 0, ions closer than that to another ion are redrawn until no
such pair is left, so the first short-range forces stay finite.
"""
import numpy as np


def ions(dims, n_pos, n_neg, seed, ymargin=1.0, min_sep=0.0, charge_pos=1.0, charge_neg=-1.0):
    """Return (pos (3, N) float64, q (N,) float64, species (N,) int32)."""
    Nx, Ny, Nz = dims
    N = n_pos + n_neg
    rng = np.random.default_rng(seed)

    def draw(n):
        return np.stack([rng.uniform(0.0, Nx, n), rng.uniform(ymargin, Ny - ymargin, n), rng.uniform(0.0, Nz, n)])

    pos = draw(N)
    if min_sep > 0.0 and N > 1:
        from scipy.spatial import cKDTree
        box = np.array([Nx, 4.0 * Ny + 4.0 * min_sep, Nz], dtype=np.float64)
        for _ in range(200):
            pts = np.mod(pos.T, box)
            tree = cKDTree(pts, boxsize=box)
            pairs = tree.query_pairs(min_sep, output_type="ndarray")
            if len(pairs) == 0:
                break
            redo = np.unique(pairs[:, 1])
            pos[:, redo] = draw(len(redo))
        else:
            raise RuntimeError("could not place ions with the requested separation")
    q = np.concatenate([np.full(n_pos, charge_pos), np.full(n_neg, charge_neg)])
    perm = rng.permutation(N)
    q = q[perm]
    species = np.zeros(N, dtype=np.int32)
    return pos, q, species
