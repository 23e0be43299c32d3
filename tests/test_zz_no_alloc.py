"""The allocation-free cell list (discos_cell_list_noalloc) against the
handle-based discos_cell_list, through the C ABI, on two calls in a row.

The allocation-free entry point serves callers that cannot allocate device
memory when they build a cell list (stream capture, a framework that owns the
device memory, fixed-latency loops); its scratch is a static device array
that keeps the previous call's contents, so the second call here checks that
nothing leaks from the first.  Cell lists are integer outputs: the tolerance
is bit-exact equality.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def _noalloc(lib, cfg, x):
    from paper_2204_14167_gb300 import _lib
    c = cfg.to_c()
    n = ctypes.c_int()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    # size query: N = 0 enqueues the (empty) list and reports n_cells
    probe = torch.empty(1 << 18 | 1, dtype=torch.int32, device="cuda")
    _lib.check(lib.discos_cell_list_noalloc(ctypes.byref(c), None, 0, ctypes.c_void_p(probe.data_ptr()), None,
                                            ctypes.byref(n), stream))
    N = x.shape[1]
    start = torch.full((n.value + 1,), -7, dtype=torch.int32, device="cuda")
    perm = torch.full((max(N, 1),), -7, dtype=torch.int32, device="cuda")
    _lib.check(lib.discos_cell_list_noalloc(ctypes.byref(c), ctypes.c_void_p(x.data_ptr()), N,
                                            ctypes.c_void_p(start.data_ptr()), ctypes.c_void_p(perm.data_ptr()),
                                            None, stream))
    torch.cuda.synchronize()
    return start.cpu().numpy(), perm[:N].cpu().numpy()


@pytest.mark.parametrize("prec", [0, 1])
def test_noalloc_cell_list_matches_handle_version(prec):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2204_14167_gb300 as dg
    from paper_2204_14167_gb300 import presets, synth, _lib
    lib = _lib.load()
    cfg, rec = presets.dry_channel_32()
    cfg.precision = prec
    cfg.max_ions = 700
    dt = torch.float64 if prec == dg.FP64 else torch.float32
    h = dg.Discos(cfg)
    for call, (n, seed) in enumerate(((700, 5), (333, 6))):
        pos, q, sp = synth.ions(cfg.dims, n // 2, n - n // 2, seed, 0.05, 0.0)
        x = torch.tensor(pos, dtype=dt, device="cuda").contiguous()
        ref_start, ref_perm = h.cell_list(x)
        torch.cuda.synchronize()
        start, perm = _noalloc(lib, cfg, x)
        assert np.array_equal(start, ref_start.cpu().numpy()), f"cell starts differ on call {call}"
        assert np.array_equal(perm, ref_perm.cpu().numpy()), f"permutation differs on call {call}"


def test_noalloc_rejects_oversize():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2204_14167_gb300 import presets, _lib
    lib = _lib.load()
    cfg, rec = presets.dry_channel_32()
    c = cfg.to_c()
    st = lib.discos_cell_list_noalloc(ctypes.byref(c), None, (1 << 20) + 1, None, None, None, None)
    assert st == _lib.ERR_INVALID_ARG


@pytest.mark.parametrize("prec", [0, 1])
def test_noalloc_many_scan_tiles_then_fewer_cells(prec):
    """32,768 list cells (a 64^3 channel, cutoff 2): the scan runs over 32
    tiles of 1024 counts, so the tile sums kept in the static array take part;
    then a call with 512 cells must not see the first call's leftovers."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2204_14167_gb300 as dg
    from paper_2204_14167_gb300 import presets, synth, _lib
    lib = _lib.load()
    dt = torch.float64 if prec == dg.FP64 else torch.float32
    for dims, psi, n in (((64, 64, 64), 2.0, 5001), ((32, 32, 32), 4.0, 777)):
        cfg, rec = presets.dry_channel_32()
        cfg.Nx, cfg.Ny, cfg.Nz = dims
        cfg.psi = psi
        cfg.lj_sigma, cfg.lj_rc = [[1.0]], [[1.1]]
        cfg.precision = prec
        cfg.max_ions = n
        h = dg.Discos(cfg)
        pos, q, sp = synth.ions(cfg.dims, n // 2, n - n // 2, 11, 0.05, 0.0)
        x = torch.tensor(pos, dtype=dt, device="cuda").contiguous()
        ref_start, ref_perm = h.cell_list(x)
        torch.cuda.synchronize()
        start, perm = _noalloc(lib, cfg, x)
        assert len(start) - 1 == (dims[0] // int(psi)) * (dims[1] // int(psi)) * (dims[2] // int(psi))
        assert np.array_equal(start, ref_start.cpu().numpy())
        assert np.array_equal(perm, ref_perm.cpu().numpy())


def test_noalloc_nonfinite_positions_return_quickly():
    """Ions at NaN all land in one list cell; the binning flags them and the
    per-cell sort stands down instead of going quadratic.  The call returns
    and the list still holds every ion exactly once."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import time
    from paper_2204_14167_gb300 import presets, _lib
    lib = _lib.load()
    cfg, rec = presets.dry_channel_32()
    cfg.precision = 1
    N = 200000
    x = torch.full((3, N), float("nan"), dtype=torch.float32, device="cuda")
    t0 = time.perf_counter()
    start, perm = _noalloc(lib, cfg, x)
    assert time.perf_counter() - t0 < 30.0
    assert start[-1] == N and np.array_equal(np.sort(perm), np.arange(N))
