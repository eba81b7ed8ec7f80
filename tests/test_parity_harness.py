"""The parity harness's reading of the GPU's blend masks, checked on the CPU
against lists it encodes itself in the documented layout (render.cu: tile
t's word for pixel i of the tile and positions start + 32c .. start + 32c +
31 of its range sits at ((start >> 5) + t + c) * 256 + i; words past the
one holding a pixel's last blend are never written and hold garbage)."""
import types

import numpy as np
import torch

from tests.parity_util import check_key_order, gpu_blend_lists


def _fake(W, H, n, seed):
    rng = np.random.default_rng(seed)
    tx, ty = -(-W // 16), -(-H // 16)
    tiles = tx * ty
    tile_base = 5                      # a view that is not the plan's first
    lens = rng.integers(0, 140, tiles)
    lens[0] = 0
    starts = np.zeros(tiles, np.int64)
    starts[1:] = np.cumsum(lens)[:-1] + 3
    total_keys = int(starts[-1] + lens[-1] + 3)
    vals = rng.integers(0, n, total_keys).astype(np.int32) + n  # view 1 of the plan: values offset by n
    ranges = np.zeros((tile_base + tiles + 2, 2), np.int64)
    ranges[tile_base:tile_base + tiles, 0] = starts
    ranges[tile_base:tile_base + tiles, 1] = starts + lens
    nwords = (total_keys // 32 + tile_base + tiles + 2) * 256
    mask = rng.integers(0, 2 ** 32, nwords, dtype=np.uint64).astype(np.uint32)  # garbage everywhere
    nc = np.zeros((H, W), np.int32)
    truth = []
    for y in range(H):
        for x in range(W):
            t = (y // 16) * tx + x // 16
            L = int(lens[t])
            chosen = np.sort(rng.choice(L, size=rng.integers(0, L + 1) if L else 0, replace=False))
            truth.append(vals[starts[t] + chosen] - n)
            last = int(chosen[-1]) + 1 if chosen.size else 0
            nc[y, x] = last
            pi = (y % 16) * 16 + x % 16
            for c in range((last + 31) // 32):
                w = 0
                for b in chosen[(chosen >= 32 * c) & (chosen < 32 * c + 32)]:
                    w |= 1 << int(b - 32 * c)
                mask[((int(starts[t]) >> 5) + tile_base + t + c) * 256 + pi] = np.uint32(w)
    plan = types.SimpleNamespace(n=n, height=[0, H], width=[0, W], tile_base=[0, tile_base], forward_only=0)
    r = types.SimpleNamespace(
        plan=plan, n_contrib=torch.as_tensor(nc.reshape(-1)),
        ranges=lambda: torch.as_tensor(ranges),
        blend_masks=lambda: torch.as_tensor(mask.view(np.int32)),
        sorted_keys=lambda: (None, torch.as_tensor(vals)),
        view_state=lambda flat, v: flat.view(H, W))
    return r, truth


def test_blend_lists_decode_the_documented_mask_layout():
    for W, H, seed in ((40, 35, 0), (16, 16, 1), (1, 1, 2), (70, 9, 3)):
        r, truth = _fake(W, H, n=1000, seed=seed)
        off, ids = gpu_blend_lists(r, 1, rows_per_block=7)
        assert off.shape == (W * H + 1,)
        for p, want in enumerate(truth):
            np.testing.assert_array_equal(ids[off[p]:off[p + 1]], want)


def test_key_order_check_rejects_out_of_order_ties():
    keys = np.array([(1 << 32) | 5, (1 << 32) | 5, (2 << 32) | 1], np.uint64)
    check_key_order(keys, np.array([3, 7, 0]))
    try:
        check_key_order(keys, np.array([7, 3, 0]))
    except AssertionError:
        return
    raise AssertionError("ties out of index order were accepted")
