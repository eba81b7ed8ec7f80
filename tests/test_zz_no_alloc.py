"""sr_sort_keys_noalloc: the radix sort for callers that cannot allocate
device memory (the library keeps the sort's scratch in a fixed device array).

Checked through the C ABI against the existing entry point: the tile keys
that sr_bin_sort sorted for a frame, put back in the order sr_bin_sort emits
them (by Gaussian record index, then tile), must come out of the no-alloc
sort bit for bit the same.  Two calls in a row, with different key counts
and an odd and an even number of radix passes, show that each call clears
the shared scratch it needs.  This file is collected last on purpose.
"""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_2605_18334_gb300 import native as N
from paper_2605_18334_gb300 import scenes
from paper_2605_18334_gb300.rasterizer import Config, Gaussians, Rasterizer

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU-only container
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

MAX_KEYS = 1 << 20  # SR_NOALLOC_MAX_KEYS


def _lib():
    lib = N.load()
    lib.sr_sort_keys_noalloc.restype = C.c_int
    lib.sr_sort_keys_noalloc.argtypes = [C.c_void_p, C.c_void_p, C.c_int64, C.c_int32, C.c_void_p, C.c_void_p,
                                         C.c_void_p]
    return lib


def _frame_keys(scene, cam):
    g = Gaussians.from_scene(scene)
    r = Rasterizer(g, [cam], Config())
    r.forward(g)
    torch.cuda.synchronize()
    keys, vals = r.sorted_keys()
    return keys.clone(), vals.clone(), int(r.plan.sort_bits)


def _emission_order(keys, vals):
    """The unsorted order of sr_bin_sort's keys: by value (record index),
    then by tile id (row-major tiles of one Gaussian)."""
    k = keys.cpu().numpy().view(np.uint64)
    v = vals.cpu().numpy()
    order = np.lexsort((k >> np.uint64(32), v))
    return (torch.from_numpy(np.ascontiguousarray(k[order]).view(np.int64)).cuda(),
            torch.from_numpy(np.ascontiguousarray(v[order])).cuda())


def test_noalloc_sort_matches_bin_sort_on_two_calls_in_a_row():
    lib = _lib()
    stream = torch.cuda.current_stream().cuda_stream
    cases = [(scenes.cluster(seed=21, n=20_000), scenes.identity_camera(320, 240)),   # 41 sort bits: 6 passes
             (scenes.cube_1k(seed=22, n=3_000), scenes.identity_camera(200, 150))]    # 40 sort bits: 5 passes
    passes = []
    for sc, cam in cases:
        ref_k, ref_v, bits = _frame_keys(sc, cam)
        n = ref_k.numel()
        assert 0 < n <= MAX_KEYS
        in_k, in_v = _emission_order(ref_k, ref_v)
        out_k = torch.full_like(in_k, -1)
        out_v = torch.full_like(in_v, -1)
        s = lib.sr_sort_keys_noalloc(in_k.data_ptr(), in_v.data_ptr(), n, bits, out_k.data_ptr(), out_v.data_ptr(),
                                     stream)
        assert s == N.SR_OK, N.status_string(s)
        torch.cuda.synchronize()
        assert torch.equal(out_k, ref_k)
        assert torch.equal(out_v, ref_v)
        passes.append((bits + 7) // 8)
    assert passes[0] % 2 != passes[1] % 2


def test_noalloc_sort_rejects_oversize_and_bad_arguments():
    lib = _lib()
    a = torch.zeros(4, dtype=torch.int64, device="cuda")
    b = torch.zeros(4, dtype=torch.int32, device="cuda")
    c = torch.zeros(4, dtype=torch.int64, device="cuda")
    d = torch.zeros(4, dtype=torch.int32, device="cuda")
    P = lambda t: t.data_ptr()
    assert lib.sr_sort_keys_noalloc(P(a), P(b), MAX_KEYS + 1, 40, P(c), P(d), None) == N.SR_ERR_CAPACITY
    assert lib.sr_sort_keys_noalloc(P(a), P(b), 4, 0, P(c), P(d), None) == N.SR_ERR_INVALID
    assert lib.sr_sort_keys_noalloc(P(a), P(b), 4, 40, P(a), P(d), None) == N.SR_ERR_INVALID
    assert lib.sr_sort_keys_noalloc(None, P(b), 4, 40, P(c), P(d), None) == N.SR_ERR_INVALID
