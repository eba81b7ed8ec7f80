"""bench.py's reference arm runs on the CPU (it times the oracle): its one
JSON line must carry the keys the benchmark contract names."""
from __future__ import annotations

import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--n", "20000", "--steps", "1",
           "--warmup", "0", "--oracle-threads", "2"]
    out = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1, out.stdout
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] == 2
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
    assert d["config"]["workload"].startswith("unbounded")


def test_end_to_end_buffer_layout_is_aligned_and_disjoint():
    """The end-to-end leg packs every input (and every result) into one flat
    buffer per direction: each field starts on a 256-byte boundary, the
    fields do not overlap, and each view has its field's shape and dtype."""
    import torch

    sys.path.insert(0, ROOT)
    import bench

    specs = [("means", (1001, 3), torch.float32), ("sh", (1001, 16, 3), torch.bfloat16),
             ("quats", (1001, 4), torch.float32), ("upstream", (3 * 7 * 5,), torch.float32)]
    offs, total = bench._layout(specs)
    ends = []
    for (name, shape, dt), (o, n) in zip(specs, offs):
        assert o % 256 == 0
        assert n == torch.empty(shape, dtype=dt).numel() * torch.empty((), dtype=dt).element_size()
        ends.append((o, o + n))
    ends.sort()
    assert all(a[1] <= b[0] for a, b in zip(ends, ends[1:]))
    assert total == ends[-1][1]
    buf = torch.zeros(total, dtype=torch.uint8)
    views = bench._carve(buf, specs)
    for (name, shape, dt) in specs:
        v = views[name]
        assert tuple(v.shape) == shape and v.dtype == dt and v.is_contiguous()
        v.reshape(-1).view(torch.uint8).fill_(0xAB)
    # every field's bytes were written through its own view, nothing else
    covered = torch.zeros(total, dtype=torch.bool)
    for o, e in ends:
        covered[o:e] = True
    assert bool((buf[covered] == 0xAB).all()) and bool((buf[~covered] == 0).all())
