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


def _call(lib, in_k, in_v, n, bits):
    out_k = torch.full_like(in_k, -1)
    out_v = torch.full_like(in_v, -1)
    s = lib.sr_sort_keys_noalloc(in_k.data_ptr(), in_v.data_ptr(), n, bits, out_k.data_ptr(), out_v.data_ptr(),
                                 torch.cuda.current_stream().cuda_stream)
    # SR_OK also says that no look-back wait of the sort gave up (the call
    # reads the sort's status word back before it returns)
    assert s == N.SR_OK, N.status_string(s)
    return out_k, out_v


def _stable_sort_reference(k, v, bits):
    """numpy's stable sort by the low ceil(bits / 8) bytes of the keys."""
    kk = k.cpu().numpy().view(np.uint64)
    mask = np.uint64((1 << (8 * ((bits + 7) // 8))) - 1) if bits < 64 else np.uint64(0xFFFFFFFFFFFFFFFF)
    order = np.argsort(kk & mask, kind="stable")
    return kk[order], v.cpu().numpy()[order]


def test_noalloc_sort_matches_bin_sort_on_two_calls_in_a_row():
    lib = _lib()
    cases = [(scenes.cluster(seed=21, n=20_000), scenes.identity_camera(320, 240)),   # 41 sort bits: 6 passes
             (scenes.cube_1k(seed=22, n=3_000), scenes.identity_camera(200, 150))]    # 40 sort bits: 5 passes
    passes = []
    for sc, cam in cases:
        ref_k, ref_v, bits = _frame_keys(sc, cam)
        n = ref_k.numel()
        assert 0 < n <= MAX_KEYS
        in_k, in_v = _emission_order(ref_k, ref_v)
        out_k, out_v = _call(lib, in_k, in_v, n, bits)
        assert torch.equal(out_k, ref_k)
        assert torch.equal(out_v, ref_v)
        passes.append((bits + 7) // 8)
    assert passes[0] % 2 != passes[1] % 2


def test_noalloc_sort_matches_a_stable_sort_with_a_ragged_last_partition():
    """Random 64-bit keys whose bits above sort_bits are zero, n not a
    multiple of the 4096-key partition, against numpy's stable argsort."""
    lib = _lib()
    rng = np.random.default_rng(5)
    for n, bits in ((12_345, 37), (MAX_KEYS - 1, 64), (4095, 9), (1, 8)):
        assert n % 4096 != 0
        raw = rng.integers(0, 2 ** 63, n, dtype=np.int64).view(np.uint64)
        raw[rng.random(n) < 0.3] = raw[0]                     # many equal keys: ties must keep input order
        if bits < 64:
            raw &= np.uint64((1 << bits) - 1)
        k = torch.from_numpy(raw.view(np.int64).copy()).cuda()
        v = torch.from_numpy(np.arange(n, dtype=np.int32)[::-1].copy()).cuda()
        out_k, out_v = _call(lib, k, v, n, bits)
        want_k, want_v = _stable_sort_reference(k, v, bits)
        np.testing.assert_array_equal(out_k.cpu().numpy().view(np.uint64), want_k)
        np.testing.assert_array_equal(out_v.cpu().numpy(), want_v)


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
