"""ctypes binding of libdiscos (include/discos.h): argument marshalling only.

Every computation runs in the CUDA library; this module converts torch
tensors to device pointers and a Python configuration to the C struct.  If
the shared library is missing it raises instead of falling back to anything.
"""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libdiscos.so")

MAX_SPECIES = 4
OK, ERR_INVALID_ARG, ERR_OOM, ERR_NOT_NEUTRAL, ERR_NOT_CONVERGED, ERR_DEVICE_FAULT, ERR_TIMEOUT, ERR_CUDA = range(8)
BC_DIRICHLET, BC_NEUMANN = 0, 1
HY_NOSLIP, HY_SLIP = 0, 1
KERNEL_PESKIN4, KERNEL_PESKIN6, KERNEL_ES = 0, 1, 2
FP64, MIXED = 0, 1
WALL_WCA, WALL_LJ93 = 0, 1
SPREAD_CHARGE, SPREAD_FORCE = 0, 1
INTERP_EFIELD, INTERP_VELOCITY = 0, 1

D = ctypes.c_double
NS = MAX_SPECIES


class Config(ctypes.Structure):
    _fields_ = [
        ("Nx", ctypes.c_int), ("Ny", ctypes.c_int), ("Nz", ctypes.c_int),
        ("bc", ctypes.c_int * 2),
        ("phi_b", D * 2),
        ("surf_charge", D * 2),
        ("kernel_es", ctypes.c_int),
        ("kernel_hy", ctypes.c_int),
        ("es_w", ctypes.c_int * 2),
        ("es_beta", D * 2),
        ("lB", D), ("eta", D), ("kT", D), ("dt", D), ("psi", D),
        ("n_tab", ctypes.c_int),
        ("nspecies", ctypes.c_int),
        ("D_tot", D * NS), ("D_wet", D * NS),
        ("gamma_coef", D * 7 * 2 * 2 * NS),
        ("lj_sigma", D * NS * NS), ("lj_xi", D * NS * NS), ("lj_rc", D * NS * NS),
        ("wall_type", ctypes.c_int),
        ("wall_sigma", D * NS), ("wall_xi", D * NS), ("wall_rc", D * NS),
        ("E_ext", D * 3),
        ("precision", ctypes.c_int),
        ("max_refine", ctypes.c_int),
        ("wet", ctypes.c_int),
        ("drift", ctypes.c_int),
        ("max_ions", ctypes.c_int),
        ("seed", ctypes.c_uint64),
        ("strip", ctypes.c_int),
        ("strip_x", D * 2),
        ("strip_phi", D),
        ("bc_hy", ctypes.c_int * 2),
        ("hy_species", ctypes.c_int),
        ("kernel_hy_s", ctypes.c_int * MAX_SPECIES),
        ("hy_w_s", ctypes.c_int * MAX_SPECIES),
        ("hy_beta_s", D * MAX_SPECIES),
    ]


class Batch(ctypes.Structure):
    """discos_batch (include/discos.h)."""
    _fields_ = [
        ("R", ctypes.c_int),
        ("offsets_host", ctypes.POINTER(ctypes.c_int)),
        ("offsets", ctypes.c_void_p),
        ("x", ctypes.c_void_p),
        ("q", ctypes.c_void_p),
        ("species", ctypes.c_void_p),
        ("phi_b", ctypes.c_void_p),
        ("hist", ctypes.c_void_p),
        ("sums", ctypes.c_void_p),
        ("F_out", ctypes.c_void_p),
        ("nbr_count", ctypes.c_void_p),
    ]


EXPORTS = [
    "discos_create", "discos_destroy", "discos_last_error", "discos_spread", "discos_solve_poisson",
    "discos_solve_stokes", "discos_interpolate", "discos_cell_list", "discos_near_field", "discos_forces",
    "discos_step", "discos_fp_table", "discos_launch_count", "discos_cell_list_noalloc",
    "discos_probe", "discos_probe_read", "discos_energy", "discos_energy_backward",
    "discos_step_batched", "discos_tune_batched", "discos_set_batched_shape", "discos_refine_history",
    "discos_fault", "discos_diagnostics", "discos_tune_transforms", "discos_set_transform_shape",
    "discos_refine_history_stokes", "discos_spread_species", "discos_interpolate_species",
]
PROBE_FAMILIES = ["cell_list", "near_field", "noise", "spread_charge", "fft_x", "fft_z", "poisson_y", "interp_e",
                  "spread_force", "stokes_y", "interp_v", "update"]

_lib = None


def load():
    """Load libdiscos.so (built in-tree by build.py); raise if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libdiscos.so not found at {LIB_PATH}: run paper_2204_14167_gb300/build.py "
                           "(or __graft_entry__.build()) first")
    lib = ctypes.CDLL(LIB_PATH)
    vp, i32, i64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64
    lib.discos_create.argtypes = [ctypes.POINTER(Config), vp, vp, vp, ctypes.POINTER(vp)]
    lib.discos_destroy.argtypes = [vp]
    lib.discos_last_error.restype = ctypes.c_char_p
    lib.discos_spread.argtypes = [vp, vp, vp, i32, i32, vp, vp]
    lib.discos_spread_species.argtypes = [vp, vp, vp, vp, i32, i32, vp, vp]
    lib.discos_solve_poisson.argtypes = [vp, vp, vp, vp]
    lib.discos_solve_stokes.argtypes = [vp, vp, vp, vp, vp]
    lib.discos_interpolate.argtypes = [vp, vp, i32, i32, vp, vp, vp]
    lib.discos_interpolate_species.argtypes = [vp, vp, vp, i32, i32, vp, vp, vp]
    lib.discos_cell_list.argtypes = [vp, vp, i32, vp, vp, ctypes.POINTER(i32), vp]
    lib.discos_near_field.argtypes = [vp, vp, vp, vp, i32, vp, vp, vp]
    lib.discos_forces.argtypes = [vp, vp, vp, vp, i32, vp, vp, vp]
    lib.discos_step.argtypes = [vp, vp, vp, vp, i32, i64, i32, vp, vp]
    lib.discos_fp_table.argtypes = [i32, i32, D, D, i32, ctypes.POINTER(D)]
    lib.discos_probe.argtypes = [vp, i32]
    lib.discos_probe_read.argtypes = [vp, ctypes.POINTER(D), ctypes.POINTER(i32)]
    lib.discos_energy.argtypes = [vp, vp, vp, i32, ctypes.POINTER(D), vp, vp]
    lib.discos_energy_backward.argtypes = [vp, vp, vp, i32, ctypes.POINTER(D), vp, vp, vp, vp, vp]
    lib.discos_step_batched.argtypes = [vp, ctypes.POINTER(Batch), i64, i32, vp]
    lib.discos_tune_batched.argtypes = [vp, ctypes.POINTER(Batch), i32, ctypes.POINTER(i32), ctypes.POINTER(D), vp]
    lib.discos_set_batched_shape.argtypes = [vp, i32]
    lib.discos_tune_transforms.argtypes = [vp, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(i32),
                                           ctypes.POINTER(ctypes.c_float), vp]
    lib.discos_set_transform_shape.argtypes = [vp, i32, i32, i32]
    lib.discos_fault.argtypes = [vp, i32, i32, ctypes.POINTER(ctypes.c_uint), vp]
    lib.discos_diagnostics.argtypes = [vp, vp, vp, vp, i32, i32, vp, vp]
    lib.discos_refine_history.argtypes = [vp, ctypes.POINTER(D), ctypes.POINTER(i32), vp]
    lib.discos_refine_history_stokes.argtypes = [vp, ctypes.POINTER(D), ctypes.POINTER(i32), vp]
    lib.discos_cell_list_noalloc.argtypes = [ctypes.POINTER(Config), vp, i32, vp, vp, ctypes.POINTER(i32), vp]
    for name in EXPORTS:
        getattr(lib, name).restype = ctypes.c_int
    lib.discos_last_error.restype = ctypes.c_char_p
    lib.discos_launch_count.restype = ctypes.c_longlong
    _lib = lib
    return lib


class DiscosError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"discos status {status}: {msg}")
        self.status = status


def check(status):
    if status != OK:
        raise DiscosError(status, load().discos_last_error().decode())
