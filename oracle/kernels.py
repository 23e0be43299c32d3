"""Immersed-boundary kernels in one dimension (grid spacing 1).

Test infrastructure only (see ``oracle/__init__``).

* 4-point Peskin kernel: App. B, Eq. peskin1d, with Delta r = 1.
* 6-point Peskin kernel: only cited in Sec. II.A.  It is the kernel defined by
  its moment conditions: for a particle at fractional offset r in [0,1) the six
  weights a_m = phi(r - m), m = -2..3, satisfy
      sum_{m even} a_m = sum_{m odd} a_m = 1/2,
      sum (r-m)   a_m = 0,   sum (r-m)^2 a_m = K,   sum (r-m)^3 a_m = 0,
      sum a_m^2 = C,
  with K = 59/60 - sqrt(29)/20 (the value that makes the kernel C^3) and C
  fixed by phi(-3) = 0 at r = 0 (continuity at the edge of the support).
  Here the five linear conditions are solved numerically for the other
  weights as affine functions of a_0 = phi(r); the quadratic condition then
  gives phi(r), taking the root that is continuous with phi(0) = 5/8 - K/4.
* ES ("exponential of a semicircle") kernel: App. B, Eq. eskernel, with the
  normalising integral done by adaptive quadrature.
"""
import numpy as np
from scipy import integrate

PESKIN4, PESKIN6, ES = 0, 1, 2

K6 = 59.0 / 60.0 - np.sqrt(29.0) / 20.0


def peskin4(z):
    """4-point Peskin kernel, App. B Eq. peskin1d (Delta r = 1)."""
    a = np.abs(np.asarray(z, dtype=np.float64))
    out = np.zeros_like(a)
    m1 = a <= 1.0
    m2 = (a > 1.0) & (a <= 2.0)
    out[m1] = (3.0 - 2.0 * a[m1] + np.sqrt(1.0 + 4.0 * a[m1] - 4.0 * a[m1] ** 2)) / 8.0
    out[m2] = (5.0 - 2.0 * a[m2] - np.sqrt(np.maximum(-7.0 + 12.0 * a[m2] - 4.0 * a[m2] ** 2, 0.0))) / 8.0
    return out


def _peskin6_affine(r, K=K6):
    """For offsets r (array), return (U, V), shape (n, 5), with
    a_m = U[:, k] + V[:, k] * a_0 for m = -2, -1, 1, 2, 3 (k = 0..4).

    Solves the five linear moment conditions numerically, one 5x5 system per
    offset (batched).
    """
    r = np.atleast_1d(np.asarray(r, dtype=np.float64))
    ms = np.array([-2, -1, 1, 2, 3], dtype=np.float64)
    d = r[:, None] - ms[None, :]                              # (n, 5)
    n = r.shape[0]
    A = np.empty((n, 5, 5))
    A[:, 0, :] = (np.array([-2, -1, 1, 2, 3]) % 2 == 0)       # even sum
    A[:, 1, :] = (np.array([-2, -1, 1, 2, 3]) % 2 != 0)       # odd sum
    A[:, 2, :] = d
    A[:, 3, :] = d ** 2
    A[:, 4, :] = d ** 3
    # a_0 sits at offset r; move its terms to the right-hand side
    rhs_const = np.tile(np.array([0.5, 0.5, 0.0, K, 0.0]), (n, 1))
    rhs_p = -np.stack([np.ones(n), np.zeros(n), r, r ** 2, r ** 3], axis=1)
    U = np.linalg.solve(A, rhs_const[..., None])[..., 0]
    V = np.linalg.solve(A, rhs_p[..., None])[..., 0]
    return U, V


def _peskin6_C(K=K6):
    """Sum-of-squares constant: impose a_3 = phi(-3) = 0 at r = 0."""
    U, V = _peskin6_affine(np.array([0.0]), K)
    p = -U[0, 4] / V[0, 4]
    a = U[0] + V[0] * p
    return float(np.sum(a ** 2) + p ** 2)


def peskin6_weights(r, K=K6):
    """Weights (phi(r+2), phi(r+1), phi(r), phi(r-1), phi(r-2), phi(r-3))
    for offsets r in [0, 1); r may be an array (result shape (n, 6))."""
    C = _peskin6_C(K)
    U, V = _peskin6_affine(r, K)
    # sum_k (U_k + V_k p)^2 + p^2 = C  ->  A p^2 + B p + c = 0
    A = np.sum(V ** 2, axis=1) + 1.0
    B = 2.0 * np.sum(U * V, axis=1)
    c = np.sum(U ** 2, axis=1) - C
    disc = np.maximum(B * B - 4 * A * c, 0.0)
    sgn = 1.0 if K < 1.5 else -1.0
    p = (-B + sgn * np.sqrt(disc)) / (2 * A)
    a = U + V * p[:, None]
    return np.stack([a[:, 0], a[:, 1], p, a[:, 2], a[:, 3], a[:, 4]], axis=1)


def peskin6(z, K=K6):
    """6-point Peskin kernel evaluated at arbitrary offsets z (support |z| < 3)."""
    z = np.asarray(z, dtype=np.float64)
    flat = z.ravel()
    out = np.zeros_like(flat)
    inside = np.abs(flat) < 3.0
    zz = flat[inside]
    fl = np.floor(zz)
    r = zz - fl
    m = (-fl).astype(np.int64)          # zz = r - m, m in -2..3
    wts = peskin6_weights(r, K)
    out[inside] = wts[np.arange(len(zz)), m + 2]
    return out.reshape(z.shape)


class ESKernel:
    """ES kernel of App. B, Eq. eskernel, alpha = w/2 (Delta r = 1)."""

    def __init__(self, w, beta):
        self.w = int(w)
        self.beta = float(beta)
        self.alpha = self.w / 2.0
        f = lambda z: np.exp(self.beta * (np.sqrt(max(1.0 - (z / self.alpha) ** 2, 0.0)) - 1.0))
        val, _ = integrate.quad(f, -self.alpha, self.alpha, epsabs=1e-14, epsrel=1e-13, limit=200)
        self.norm = val

    def __call__(self, z):
        z = np.asarray(z, dtype=np.float64)
        t = 1.0 - (z / self.alpha) ** 2
        out = np.where(t >= 0.0, np.exp(self.beta * (np.sqrt(np.maximum(t, 0.0)) - 1.0)), 0.0)
        return out / self.norm


class Kernel:
    """A 1-D kernel phi with support width w (number of grid points)."""

    def __init__(self, kind, es_w=6, es_beta=8.0):
        self.kind = kind
        if kind == PESKIN4:
            self.w = 4
            self._f = peskin4
        elif kind == PESKIN6:
            self.w = 6
            self._f = None
        elif kind == ES:
            self._es = ESKernel(es_w, es_beta)
            self.w = self._es.w
            self._f = self._es
        else:
            raise ValueError("unknown kernel kind")

    def __call__(self, z):
        if self.kind == PESKIN6:
            return peskin6(z)
        return self._f(z)

    def stencil(self, s):
        """Grid points and weights for coordinates s (grid points at integers).

        Returns (idx, wts) of shape (len(s), w): idx = floor(s - w/2) + 1 + l.
        """
        s = np.asarray(s, dtype=np.float64)
        start = np.floor(s - self.w / 2.0).astype(np.int64) + 1
        idx = start[:, None] + np.arange(self.w)[None, :]
        z = s[:, None] - idx
        if self.kind == PESKIN6:
            # the six points are floor(s)-2 .. floor(s)+3: offsets r+2 .. r-3
            wts = peskin6_weights(s - np.floor(s))
        else:
            wts = self._f(z)
        return idx, wts
