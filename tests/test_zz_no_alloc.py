"""The allocation-free cell-key sort against the library's allocating path.

sph_sort_cell_keys_static serves callers that may not let a library allocate
device memory (a host that owns the device-memory budget, or a loop that must
not risk the device synchronisation of cudaMalloc/cudaFree).  Its scratch is
a fixed array in the library's device data.  Here it sorts the cell keys of
the 28,062-particle dam break and must reproduce, bit for bit, the order and
cells that sph_get_order returns (the neighbour list built by the engine with
allocated scratch) -- on two calls in a row, since every call reuses the same
array.  This file is collected last so a failure here leaves the rest run.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2104_00537_gb300 import cases, sph

pytestmark = pytest.mark.gpu


def _fn():
    L = sph.load()
    f = L.sph_sort_cell_keys_static
    f.restype = C.c_int
    f.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_int32, C.c_void_p]
    return f


def test_static_sort_matches_engine_neighbour_list():
    import torch
    torch.cuda.set_device(0)
    case = cases.dam_break(0.02)
    eng = sph.Engine.create(case)
    ids, cells, n_inside = eng.order()          # existing entry point (allocating path)
    eng.destroy()
    assert n_inside == case.n
    # the engine's keys, in the caller's particle order: boundary bit above the cell
    cbits = int(cells.max()).bit_length()
    keys = np.zeros(case.n, np.int64)
    keys[ids] = (case.ptype[ids].astype(np.int64) << cbits) | cells
    nbits = cbits + 1
    stream = torch.cuda.current_stream()
    d_in = torch.from_numpy(keys.astype(np.int32)).cuda()
    f = _fn()
    for call in range(2):                        # the scratch array is reused
        d_keys = torch.full((case.n,), -1, dtype=torch.int32, device="cuda")
        d_perm = torch.full((case.n,), -1, dtype=torch.int32, device="cuda")
        rc = f(d_in.data_ptr(), d_keys.data_ptr(), d_perm.data_ptr(), case.n, nbits,
               stream.cuda_stream)
        assert rc == 0, sph.last_error()
        torch.cuda.synchronize()
        perm = d_perm.cpu().numpy().astype(np.int64)
        skeys = d_keys.cpu().numpy().astype(np.int64)
        assert np.array_equal(perm, ids), call
        assert np.array_equal(skeys & ((1 << cbits) - 1), cells), call
        assert np.array_equal(skeys >> cbits, case.ptype[ids]), call


def test_static_sort_at_the_size_limit():
    """Exactly SPH_SORT_STATIC_MAX_KEYS random keys below 2^21 (nbits not a
    multiple of 8: three 8-bit passes, the last one partly empty), where the
    sort uses every byte of the fixed array: keys and permutation bit for bit
    equal to NumPy's stable argsort, on two calls in a row."""
    import torch
    torch.cuda.set_device(0)
    n, nbits = sph.SORT_STATIC_MAX_KEYS, 21
    from paper_2104_00537_gb300 import cases
    keys = (cases.splitmix64(11, n) >> np.uint64(64 - nbits)).astype(np.int64)
    assert keys.max() < (1 << nbits) and len(np.unique(keys)) < n  # ties present
    ref = np.argsort(keys, kind="stable")
    stream = torch.cuda.current_stream()
    d_in = torch.from_numpy(keys.astype(np.int32)).cuda()
    f = _fn()
    for call in range(2):
        d_keys = torch.full((n,), -1, dtype=torch.int32, device="cuda")
        d_perm = torch.full((n,), -1, dtype=torch.int32, device="cuda")
        rc = f(d_in.data_ptr(), d_keys.data_ptr(), d_perm.data_ptr(), n, nbits,
               stream.cuda_stream)
        assert rc == 0, sph.last_error()
        torch.cuda.synchronize()
        assert np.array_equal(d_perm.cpu().numpy().astype(np.int64), ref), call
        assert np.array_equal(d_keys.cpu().numpy().astype(np.int64), keys[ref]), call
    # the input is read only
    assert np.array_equal(d_in.cpu().numpy().astype(np.int64), keys)


def test_static_sort_rejects_overlapping_buffers():
    import torch
    torch.cuda.set_device(0)
    f = _fn()
    a = torch.zeros(3000, dtype=torch.int32, device="cuda")
    b = torch.zeros(1000, dtype=torch.int32, device="cuda")
    p = a.data_ptr()
    for kin, kout, perm in ((p, p, b.data_ptr()),             # in place
                            (p, p + 4 * 999, b.data_ptr()),   # last key shared
                            (p, p + 4 * 1000, p + 4 * 1500)):  # outputs overlap
        rc = f(kin, kout, perm, 1000, 20, None)
        assert rc == -1
        assert "overlap" in sph.last_error()
    rc = f(p, p + 4 * 1000, b.data_ptr(), 1000, 20, None)  # disjoint: accepted
    assert rc == 0, sph.last_error()
    torch.cuda.synchronize()


def test_static_sort_rejects_oversize():
    f = _fn()
    n = sph.SORT_STATIC_MAX_KEYS + 1
    rc = f(None, None, None, n, 20, None)
    assert rc == -1
    assert "static limit" in sph.last_error()
