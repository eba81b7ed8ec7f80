"""Scene files: round trips through the PLY layout and the 3DGS field
conventions (channel-major higher SH coefficients, logit opacity, log
scales, w-first quaternions; no skew fields -> zero skew)."""
import numpy as np
import pytest

from paper_2605_18334_gb300 import scenes
from paper_2605_18334_gb300.ply import read_ply, write_ply


@pytest.mark.parametrize("deg,two,split", [(0, False, False), (1, True, False), (2, False, True), (3, True, True)])
def test_round_trip(tmp_path, deg, two, split):
    sc = scenes.cluster(seed=deg, n=257, sh_degree=deg, two_opacities=two, split=split)
    path = tmp_path / "scene.ply"
    write_ply(str(path), sc)
    back = read_ply(str(path))
    assert back.n == sc.n and back.sh_degree == deg and back.two_opacities == two
    for k in ("means", "log_scales", "quats", "opacity_logits", "skew", "sh"):
        np.testing.assert_array_equal(getattr(back, k), np.asarray(getattr(sc, k), np.float32), k)
    if split:
        np.testing.assert_array_equal(back.split_dir, sc.split_dir)
    else:
        assert back.split_dir is None


def test_plain_3dgs_file_reads_with_zero_skew_and_channel_major_sh(tmp_path):
    n, k = 5, 16
    names = ["x", "y", "z", "nx", "ny", "nz", "f_dc_0", "f_dc_1", "f_dc_2"] + [f"f_rest_{i}" for i in range(45)] + \
            ["opacity", "scale_0", "scale_1", "scale_2", "rot_0", "rot_1", "rot_2", "rot_3"]
    a = np.arange(n * len(names), dtype=np.float32).reshape(n, len(names))
    path = tmp_path / "plain.ply"
    with open(path, "wb") as f:
        f.write(("ply\nformat binary_little_endian 1.0\nelement vertex %d\n" % n).encode())
        f.write("".join(f"property float {nm}\n" for nm in names).encode())
        f.write(b"end_header\n")
        f.write(a.astype("<f4").tobytes())
    sc = read_ply(str(path))
    assert sc.sh_degree == 3 and not sc.two_opacities and sc.split_dir is None
    np.testing.assert_array_equal(sc.skew, 0.0)
    col = {nm: i for i, nm in enumerate(names)}
    for c in range(3):
        np.testing.assert_array_equal(sc.sh[:, 0, c], a[:, col[f"f_dc_{c}"]])
        for j in range(1, k):  # f_rest_(c (K-1) + j - 1) is channel c, coefficient j
            np.testing.assert_array_equal(sc.sh[:, j, c], a[:, col[f"f_rest_{c * (k - 1) + j - 1}"]])
    np.testing.assert_array_equal(sc.quats[:, 0], a[:, col["rot_0"]])
    np.testing.assert_array_equal(sc.opacity_logits, a[:, col["opacity"]])


def test_rejects_other_formats(tmp_path):
    p = tmp_path / "ascii.ply"
    p.write_bytes(b"ply\nformat ascii 1.0\nelement vertex 1\nproperty float x\nend_header\n0\n")
    with pytest.raises(ValueError):
        read_ply(str(p))
    q = tmp_path / "not.ply"
    q.write_bytes(b"abc\n")
    with pytest.raises(ValueError):
        read_ply(str(q))
