"""GB300-native DISCOS hot path (wall-bounded channel) behind the libdiscos C ABI.

Python side: a thin binding (`Discos`) over include/discos.h that passes
torch device tensors and the current CUDA stream to the library, a run
configuration (`RunConfig`), workload presets and seeded synthetic inputs.
All numerical work happens in the CUDA kernels of libdiscos.
"""
from dataclasses import dataclass, field
import ctypes

from . import _lib
from ._lib import (BC_DIRICHLET, BC_NEUMANN, HY_NOSLIP, HY_SLIP, KERNEL_PESKIN4, KERNEL_PESKIN6, KERNEL_ES, FP64, MIXED,
                   WALL_WCA, WALL_LJ93, SPREAD_CHARGE, SPREAD_FORCE, INTERP_EFIELD, INTERP_VELOCITY,
                   DiscosError)

__all__ = ["RunConfig", "Discos", "DiscosError", "fp_table", "BC_DIRICHLET", "BC_NEUMANN", "HY_NOSLIP", "HY_SLIP",
           "KERNEL_PESKIN4",
           "KERNEL_PESKIN6", "KERNEL_ES", "FP64", "MIXED", "WALL_WCA", "WALL_LJ93"]


def _unit_gamma():
    # gamma_hat = 1 everywhere: c1 = 1, all other terms zero (c3, c5, c7 = 1 keep it finite)
    return [1.0, 0.0, 1.0, 0.0, 1.0, 0.0, 1.0]


@dataclass
class RunConfig:
    """Reduced units: grid spacing 1, eps = 1/(4 pi lB).  Mirrors discos_config."""
    Nx: int = 32
    Ny: int = 32
    Nz: int = 32
    bc: tuple = (BC_DIRICHLET, BC_DIRICHLET)
    phi_b: tuple = (0.0, 0.0)
    surf_charge: tuple = (0.0, 0.0)
    kernel_es: int = KERNEL_PESKIN6
    kernel_hy: int = KERNEL_PESKIN4
    es_w: tuple = (6, 6)
    es_beta: tuple = (8.0, 8.0)
    lB: float = 7.0
    eta: float = 1.0
    kT: float = 1.0
    dt: float = 0.01
    psi: float = 4.0
    n_tab: int = 64
    nspecies: int = 1
    D_tot: list = field(default_factory=lambda: [1.0])
    D_wet: list = field(default_factory=lambda: [0.0])
    # [species][direction: 0 parallel, 1 perpendicular][0 tot, 1 wet][7]
    gamma_coef: list = field(default_factory=lambda: [[[_unit_gamma(), _unit_gamma()]] * 2])
    lj_sigma: list = field(default_factory=lambda: [[1.0]])
    lj_xi: list = field(default_factory=lambda: [[1.0]])
    lj_rc: list = field(default_factory=lambda: [[2.0 ** (1.0 / 6.0)]])
    wall_type: int = WALL_WCA
    wall_sigma: list = field(default_factory=lambda: [2.0 ** (-1.0 / 6.0)])
    wall_xi: list = field(default_factory=lambda: [1.0])
    wall_rc: list = field(default_factory=lambda: [1.0])
    E_ext: tuple = (0.0, 0.0, 0.0)
    precision: int = FP64
    max_refine: int = 0
    wet: bool = False
    drift: bool = True
    max_ions: int = 1024
    seed: int = 20220428
    # metal strip in the (dielectric) bottom wall: cells with centre in [x0, x1)
    strip: bool = False
    strip_x: tuple = (0.0, 0.0)
    strip_phi: float = 0.0
    # hydrodynamic wall conditions (bottom, top): HY_NOSLIP or HY_SLIP
    bc_hy: tuple = (0, 0)
    # hydrodynamic kernel per species (App. B): with hy_species, species s
    # spreads and interpolates with (kernel_hy_s[s], hy_w_s[s], hy_beta_s[s])
    hy_species: bool = False
    kernel_hy_s: list = field(default_factory=lambda: [KERNEL_PESKIN4])
    hy_w_s: list = field(default_factory=lambda: [4])
    hy_beta_s: list = field(default_factory=lambda: [0.0])

    @property
    def dims(self):
        return (self.Nx, self.Ny, self.Nz)

    def to_c(self):
        c = _lib.Config()
        c.Nx, c.Ny, c.Nz = self.Nx, self.Ny, self.Nz
        for w in range(2):
            c.bc[w] = int(self.bc[w])
            c.phi_b[w] = float(self.phi_b[w])
            c.surf_charge[w] = float(self.surf_charge[w])
            c.es_w[w] = int(self.es_w[w])
            c.es_beta[w] = float(self.es_beta[w])
        c.kernel_es, c.kernel_hy = int(self.kernel_es), int(self.kernel_hy)
        c.lB, c.eta, c.kT, c.dt, c.psi = self.lB, self.eta, self.kT, self.dt, self.psi
        c.n_tab = self.n_tab
        c.nspecies = self.nspecies
        for a in range(self.nspecies):
            c.D_tot[a] = float(self.D_tot[a])
            c.D_wet[a] = float(self.D_wet[a])
            for d in range(2):
                for t in range(2):
                    for k in range(7):
                        c.gamma_coef[a][d][t][k] = float(self.gamma_coef[a][d][t][k])
            for b in range(self.nspecies):
                c.lj_sigma[a][b] = float(self.lj_sigma[a][b])
                c.lj_xi[a][b] = float(self.lj_xi[a][b])
                c.lj_rc[a][b] = float(self.lj_rc[a][b])
            c.wall_sigma[a] = float(self.wall_sigma[a])
            c.wall_xi[a] = float(self.wall_xi[a])
            c.wall_rc[a] = float(self.wall_rc[a])
        c.wall_type = int(self.wall_type)
        for d in range(3):
            c.E_ext[d] = float(self.E_ext[d])
        c.precision = int(self.precision)
        c.max_refine = int(self.max_refine)
        c.wet = int(bool(self.wet))
        c.drift = int(bool(self.drift))
        c.max_ions = int(self.max_ions)
        c.seed = int(self.seed)
        c.strip = int(bool(self.strip))
        c.strip_x[0], c.strip_x[1] = float(self.strip_x[0]), float(self.strip_x[1])
        c.strip_phi = float(self.strip_phi)
        c.bc_hy[0], c.bc_hy[1] = int(self.bc_hy[0]), int(self.bc_hy[1])
        c.hy_species = int(bool(self.hy_species))
        if self.hy_species:
            for a in range(self.nspecies):
                c.kernel_hy_s[a] = int(self.kernel_hy_s[a])
                c.hy_w_s[a] = int(self.hy_w_s[a])
                c.hy_beta_s[a] = float(self.hy_beta_s[a])
        return c


def _need(t, n, dtype, name, dtypes=None, device=None):
    """Reject a device array that the library would read or write past, or
    misread: it must be a contiguous CUDA tensor of the handle's type with at
    least n elements, on the handle's GPU (None passes: the argument is
    optional)."""
    if t is None:
        return
    ok_type = t.dtype in dtypes if dtypes else t.dtype == dtype
    if not (getattr(t, "is_cuda", False) and ok_type and t.is_contiguous() and t.numel() >= n):
        where = "" if getattr(t, "is_cuda", False) else " on the host"
        raise ValueError(f"{name}: need a contiguous CUDA tensor of {dtype} with at least {n} elements, "
                         f"got shape {tuple(t.shape)} {t.dtype}{where}")
    if device is not None and t.device != device:
        raise ValueError(f"{name}: on {t.device}, but the handle lives on {device}")


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


class Discos:
    """A libdiscos handle.  Tensors are CUDA tensors of the handle's real type
    (float64 for FP64, float32 for MIXED); positions are (3, N), contiguous."""

    def __init__(self, cfg: RunConfig):
        import torch
        lib = _lib.load()
        if not torch.cuda.is_available():
            raise RuntimeError("libdiscos needs a CUDA device")
        torch.cuda.init()
        # the library launches on the current device; the handle's workspace
        # lives on the device current at creation, and every tensor must too
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.cfg = cfg
        self._c = cfg.to_c()
        h = ctypes.c_void_p()
        _lib.check(lib.discos_create(ctypes.byref(self._c), None, None, None, ctypes.byref(h)))
        self._h = h
        self._lib = lib
        self.dtype = torch.float64 if cfg.precision == FP64 else torch.float32

    def close(self):
        if getattr(self, "_h", None):
            self._lib.discos_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- helpers
    def _need(self, t, n, dtype, name, dtypes=None):
        _need(t, n, dtype, name, dtypes, self.device)

    def _check_ions(self, x):
        if not (getattr(x, "is_cuda", False) and x.dtype == self.dtype and x.is_contiguous() and x.dim() == 2
                and x.shape[0] == 3):
            raise ValueError(f"positions: need a contiguous (3, N) CUDA tensor of {self.dtype}")
        if x.device != self.device:
            raise ValueError(f"positions: on {x.device}, but the handle lives on {self.device}")
        return x.shape[1]

    def _G(self):
        Nx, Ny, Nz = self.cfg.dims
        return Nx * Ny * Nz

    def _Gf(self):
        Nx, Ny, Nz = self.cfg.dims
        return Nx * Nz * (3 * Ny + 1)

    def _ions_q(self, x, q, species=None):
        import torch
        N = self._check_ions(x)
        self._need(q, N, self.dtype, "q")
        self._need(species, N, torch.int32, "species")
        return N

    def empty_grid(self, kind="cell"):
        import torch
        Nx, Ny, Nz = self.cfg.dims
        if kind == "cell":
            return torch.empty((Nz, Ny, Nx), dtype=self.dtype, device=self.device)
        n = Nx * Nz * (3 * Ny + 1)
        return torch.empty(n, dtype=self.dtype, device=self.device)

    # -- entry points
    def spread_charge(self, x, q, out=None, stream=None):
        N = self._ions_q(x, q)
        self._need(out, self._G(), self.dtype, "out")
        rho = self.empty_grid("cell") if out is None else out
        _lib.check(self._lib.discos_spread(self._h, _ptr(x), _ptr(q), N, SPREAD_CHARGE, _ptr(rho), _stream(stream)))
        return rho

    def spread_force(self, x, F, out=None, stream=None, species=None):
        """S^hy F; with species (int32 (N,)) and a per-species kernel run,
        each ion spreads with its own species' kernel."""
        import torch
        N = self._check_ions(x)
        self._need(F, 3 * N, self.dtype, "F")
        self._need(out, self._Gf(), self.dtype, "out")
        self._need(species, N, torch.int32, "species")
        f = self.empty_grid("mac") if out is None else out
        _lib.check(self._lib.discos_spread_species(self._h, _ptr(x), _ptr(F), _ptr(species), N, SPREAD_FORCE,
                                                   _ptr(f), _stream(stream)))
        return f

    def solve_poisson(self, rho, out=None, stream=None):
        self._need(rho, self._G(), self.dtype, "rho")
        self._need(out, self._G(), self.dtype, "out")
        phi = self.empty_grid("cell") if out is None else out
        _lib.check(self._lib.discos_solve_poisson(self._h, _ptr(rho), _ptr(phi), _stream(stream)))
        return phi

    def solve_stokes(self, f, out=None, pressure=False, stream=None):
        self._need(f, self._Gf(), self.dtype, "f")
        self._need(out, self._Gf(), self.dtype, "out")
        v = self.empty_grid("mac") if out is None else out
        p = self.empty_grid("cell") if pressure else None
        _lib.check(self._lib.discos_solve_stokes(self._h, _ptr(f), _ptr(v), _ptr(p), _stream(stream)))
        return (v, p) if pressure else v

    def interpolate_efield(self, x, phi, stream=None):
        import torch
        N = self._check_ions(x)
        self._need(phi, self._G(), self.dtype, "phi")
        out = torch.empty((3, N), dtype=self.dtype, device=self.device)
        _lib.check(self._lib.discos_interpolate(self._h, _ptr(x), N, INTERP_EFIELD, _ptr(phi), _ptr(out),
                                                _stream(stream)))
        return out

    def interpolate_velocity(self, x, v, stream=None, species=None):
        """J^hy v; with species (int32 (N,)) and a per-species kernel run,
        each ion interpolates with its own species' kernel."""
        import torch
        N = self._check_ions(x)
        self._need(v, self._Gf(), self.dtype, "v")
        self._need(species, N, torch.int32, "species")
        out = torch.zeros((3, N), dtype=self.dtype, device=self.device)
        _lib.check(self._lib.discos_interpolate_species(self._h, _ptr(x), _ptr(species), N, INTERP_VELOCITY,
                                                        _ptr(v), _ptr(out), _stream(stream)))
        return out

    def cell_list(self, x, stream=None):
        import torch
        N = self._check_ions(x)
        n = ctypes.c_int()
        _lib.check(self._lib.discos_cell_list(self._h, _ptr(x), 0, None, None, ctypes.byref(n), _stream(stream)))
        start = torch.empty(n.value + 1, dtype=torch.int32, device=self.device)
        perm = torch.empty(max(N, 1), dtype=torch.int32, device=self.device)
        _lib.check(self._lib.discos_cell_list(self._h, _ptr(x), N, _ptr(start), _ptr(perm), None, _stream(stream)))
        return start, perm[:N]

    def near_field(self, x, q, species=None, F=None, counts=True, stream=None):
        import torch
        N = self._ions_q(x, q, species)
        self._need(F, 3 * N, self.dtype, "F")
        if F is None:
            F = torch.zeros((3, N), dtype=self.dtype, device=self.device)
        nbr = torch.empty(max(N, 1), dtype=torch.int32, device=self.device) if counts else None
        _lib.check(self._lib.discos_near_field(self._h, _ptr(x), _ptr(q), _ptr(species), N, _ptr(F), _ptr(nbr),
                                               _stream(stream)))
        return (F, nbr[:N]) if counts else F

    def forces(self, x, q, species=None, counts=False, stream=None):
        import torch
        N = self._ions_q(x, q, species)
        F = torch.empty((3, N), dtype=self.dtype, device=self.device)
        nbr = torch.empty(max(N, 1), dtype=torch.int32, device=self.device) if counts else None
        _lib.check(self._lib.discos_forces(self._h, _ptr(x), _ptr(q), _ptr(species), N, _ptr(F), _ptr(nbr),
                                           _stream(stream)))
        return (F, nbr[:N]) if counts else F

    def step(self, x, q, species=None, step0=0, nsteps=1, F_out=None, stream=None):
        """Advance x in place by nsteps steps; returns x."""
        N = self._ions_q(x, q, species)
        self._need(F_out, 3 * N, self.dtype, "F_out")
        _lib.check(self._lib.discos_step(self._h, _ptr(x), _ptr(q), _ptr(species), N, int(step0), int(nsteps),
                                         _ptr(F_out), _stream(stream)))
        return x

    def tune_transforms(self, stream=None):
        """Pick the fastest transform launch shape; returns (pairs, threads, tile, (ms_x, ms_z))."""
        a, b, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        ms = (ctypes.c_float * 2)()
        _lib.check(self._lib.discos_tune_transforms(self._h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), ms,
                                                    _stream(stream)))
        return a.value, b.value, c.value, (ms[0], ms[1])

    def set_transform_shape(self, fx_pairs, fx_threads, fz_tile):
        _lib.check(self._lib.discos_set_transform_shape(self._h, int(fx_pairs), int(fx_threads), int(fz_tile)))

    def fault(self, sync=True, clear=False, stream=None):
        """The device fault word (bit 0 non-finite position, bit 1 escaped ion)."""
        w = ctypes.c_uint()
        _lib.check(self._lib.discos_fault(self._h, int(sync), int(clear), ctypes.byref(w), _stream(stream)))
        return w.value

    def diagnostics(self, x, q, F=None, with_rho=True, stream=None):
        """Double-precision sums: dict(sum_q, sum_rho, sum_F, nonfinite, escaped)."""
        import torch
        N = self._ions_q(x, q)
        self._need(F, 3 * N, self.dtype, "F")
        out = torch.zeros(8, dtype=torch.float64, device=self.device)
        _lib.check(self._lib.discos_diagnostics(self._h, _ptr(x), _ptr(q), _ptr(F), N, int(bool(with_rho)),
                                                _ptr(out), _stream(stream)))
        o = out.cpu().tolist()
        return dict(sum_q=o[0], sum_rho=o[1], sum_F=o[2:5], nonfinite=int(o[5]), escaped=int(o[6]))

    def refine_history(self, stream=None):
        """Relative residuals of the last Poisson solve: [after the solve, after sweep 1, ...]."""
        buf = (ctypes.c_double * 8)()
        n = ctypes.c_int()
        _lib.check(self._lib.discos_refine_history(self._h, buf, ctypes.byref(n), _stream(stream)))
        return [buf[i] for i in range(n.value)]

    def refine_history_stokes(self, stream=None):
        """Relative residuals of the last Stokes solve: [after the solve, after sweep 1, ...]."""
        buf = (ctypes.c_double * 8)()
        n = ctypes.c_int()
        _lib.check(self._lib.discos_refine_history_stokes(self._h, buf, ctypes.byref(n), _stream(stream)))
        return [buf[i] for i in range(n.value)]

    # -- batched replicas
    def make_batch(self, x, q, offsets, species=None, phi_b=None, hist=None, sums=None, F_out=None,
                   nbr=None):
        """A discos_batch over packed replicas: x (3, Ntot) float32, q (Ntot,),
        offsets a host sequence of R + 1 ints.  The returned object keeps the
        tensors it references alive."""
        import torch
        off = [int(v) for v in offsets]
        R = len(off) - 1
        Ntot = off[-1] if off else 0
        ints = (torch.int32, getattr(torch, "uint32", torch.int32))
        self._need(x, 3 * Ntot, self.dtype, "x")          # the library itself requires a MIXED handle
        self._need(q, Ntot, self.dtype, "q")
        self._need(species, Ntot, torch.int32, "species")
        self._need(phi_b, 2 * R, torch.float64, "phi_b")
        self._need(hist, R * self.cfg.nspecies * self.cfg.Ny, torch.int32, "hist", ints)
        self._need(sums, 4 * R, torch.float64, "sums")
        self._need(F_out, 3 * Ntot, self.dtype, "F_out")
        self._need(nbr, Ntot, torch.int32, "nbr")
        b = _lib.Batch()
        b.R = R
        b._off_host = (ctypes.c_int * (R + 1))(*off)
        b._off_dev = torch.tensor(off, dtype=torch.int32, device=self.device)
        b.offsets_host = ctypes.cast(b._off_host, ctypes.POINTER(ctypes.c_int))
        b.offsets = b._off_dev.data_ptr()
        b._keep = (x, q, species, phi_b, hist, sums, F_out, nbr)
        for name, t in (("x", x), ("q", q), ("species", species), ("phi_b", phi_b), ("hist", hist),
                        ("sums", sums), ("F_out", F_out), ("nbr_count", nbr)):
            setattr(b, name, None if t is None else t.data_ptr())
        return b

    def step_batched(self, batch, step0=0, nsteps=1, stream=None):
        _lib.check(self._lib.discos_step_batched(self._h, ctypes.byref(batch), int(step0), int(nsteps),
                                                 _stream(stream)))

    def tune_batched(self, batch, trial_steps=32, stream=None):
        """Pick the fastest steps per launch; returns (steps_per_launch, ms_per_step)."""
        s, ms = ctypes.c_int(), ctypes.c_double()
        _lib.check(self._lib.discos_tune_batched(self._h, ctypes.byref(batch), int(trial_steps), ctypes.byref(s),
                                                 ctypes.byref(ms), _stream(stream)))
        return s.value, ms.value

    def set_batched_shape(self, steps_per_launch):
        _lib.check(self._lib.discos_set_batched_shape(self._h, int(steps_per_launch)))

    def _phi_b(self, phi_b):
        if phi_b is None:
            return None
        vals = [float(v) for v in (phi_b.tolist() if hasattr(phi_b, "tolist") else phi_b)]
        assert len(vals) == 2, "phi_b holds the two wall potentials"
        return (ctypes.c_double * 2)(*vals)

    def energy(self, x, q, phi_b=None, out=None, stream=None):
        """Discrete electrostatic energy U as a float64 CUDA scalar."""
        import torch
        N = self._check_ions(x)
        self._need(q, N, self.dtype, "q")
        U = torch.empty((), dtype=torch.float64, device=self.device) if out is None else out
        _lib.check(self._lib.discos_energy(self._h, _ptr(x), _ptr(q), N, self._phi_b(phi_b), _ptr(U),
                                           _stream(stream)))
        return U

    def energy_backward(self, x, q, dU, phi_b=None, need=(True, True, True), stream=None):
        """(dx, dq, dphi_b) = dU * gradients of U; entries not in `need` are None."""
        import torch
        N = self._check_ions(x)
        self._need(q, N, self.dtype, "q")
        dU = dU.to(device=self.device, dtype=torch.float64).contiguous()
        dx = torch.empty((3, N), dtype=self.dtype, device=self.device) if need[0] else None
        dq = torch.empty(N, dtype=self.dtype, device=self.device) if need[1] else None
        db = torch.empty(2, dtype=torch.float64, device=self.device) if need[2] else None
        _lib.check(self._lib.discos_energy_backward(self._h, _ptr(x), _ptr(q), N, self._phi_b(phi_b), _ptr(dU),
                                                    _ptr(dx), _ptr(dq), _ptr(db), _stream(stream)))
        return dx, dq, db


def probe(handle, family):
    """Time every launch of one kernel family ('stokes_y', 'fft_z', ...) with
    CUDA events on its stream; None switches the probe off."""
    fam = -1 if family is None else _lib.PROBE_FAMILIES.index(family)
    _lib.check(handle._lib.discos_probe(handle._h, fam))


def probe_read(handle):
    """(summed milliseconds, number of launches) since the probe was set."""
    t = ctypes.c_double()
    n = ctypes.c_int()
    _lib.check(handle._lib.discos_probe_read(handle._h, ctypes.byref(t), ctypes.byref(n)))
    return t.value, n.value


def fp_table(kernel, psi, n_tab, es_w=6, es_beta=8.0):
    """The library's F^P table (host computation, no GPU needed)."""
    lib = _lib.load()
    out = (ctypes.c_double * (n_tab + 1))()
    _lib.check(lib.discos_fp_table(int(kernel), int(es_w), float(es_beta), float(psi), int(n_tab), out))
    return list(out)


def launch_count():
    """Kernels the library has enqueued since it was loaded."""
    return int(_lib.load().discos_launch_count())
