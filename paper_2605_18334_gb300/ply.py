"""Scene files: the binary PLY layout of 3DGS scenes, extended by the skew
vector (and the second opacity and the split direction of the enhanced
opacity term).

Per vertex (float32, little endian): x y z, nx ny nz (unused, zero), the SH
coefficients f_dc_0..2 (degree 0, one per channel) and f_rest_0.. (the
higher degrees, channel-major: all of red's, then green's, then blue's),
opacity (logit), scale_0..2 (log), rot_0..3 (quaternion w, x, y, z), then
skew_0..2 (the skew vector in the Gaussian's local frame) and, when present,
opacity_1 (second logit) and split_0..2 (split direction).  A file without
skew fields is a plain 3DGS scene: its skew vectors are zero.
"""
from __future__ import annotations

import numpy as np

from .scenes import Scene


def _fields(sh_degree: int, two_opacities: bool, split: bool) -> list:
    k = (sh_degree + 1) ** 2
    names = ["x", "y", "z", "nx", "ny", "nz", "f_dc_0", "f_dc_1", "f_dc_2"]
    names += [f"f_rest_{i}" for i in range(3 * (k - 1))]
    names += ["opacity", "scale_0", "scale_1", "scale_2", "rot_0", "rot_1", "rot_2", "rot_3",
              "skew_0", "skew_1", "skew_2"]
    if two_opacities:
        names.append("opacity_1")
    if split:
        names += ["split_0", "split_1", "split_2"]
    return names


def write_ply(path: str, scene: Scene) -> None:
    n = scene.n
    k = (scene.sh_degree + 1) ** 2
    two = np.asarray(scene.opacity_logits).ndim == 2
    split = scene.split_dir is not None
    names = _fields(scene.sh_degree, two, split)
    a = np.zeros((n, len(names)), np.float32)
    col = {nm: i for i, nm in enumerate(names)}
    a[:, 0:3] = scene.means
    sh = np.asarray(scene.sh, np.float32).reshape(n, k, 3)
    a[:, col["f_dc_0"]:col["f_dc_0"] + 3] = sh[:, 0, :]
    if k > 1:  # channel-major rest: [N, 3, K-1]
        a[:, col["f_dc_2"] + 1:col["f_dc_2"] + 1 + 3 * (k - 1)] = np.transpose(sh[:, 1:, :], (0, 2, 1)).reshape(n, -1)
    op = np.asarray(scene.opacity_logits, np.float32)
    a[:, col["opacity"]] = op[:, 0] if two else op
    if two:
        a[:, col["opacity_1"]] = op[:, 1]
    a[:, col["scale_0"]:col["scale_0"] + 3] = scene.log_scales
    a[:, col["rot_0"]:col["rot_0"] + 4] = scene.quats
    a[:, col["skew_0"]:col["skew_0"] + 3] = scene.skew
    if split:
        a[:, col["split_0"]:col["split_0"] + 3] = scene.split_dir
    header = ["ply", "format binary_little_endian 1.0", f"element vertex {n}"]
    header += [f"property float {nm}" for nm in names]
    header.append("end_header")
    with open(path, "wb") as f:
        f.write(("\n".join(header) + "\n").encode("ascii"))
        f.write(np.ascontiguousarray(a, "<f4").tobytes())


def read_ply(path: str) -> Scene:
    with open(path, "rb") as f:
        names, n = [], None
        line = f.readline().decode("ascii").strip()
        if line != "ply":
            raise ValueError("not a PLY file")
        while True:
            line = f.readline().decode("ascii").strip()
            if line.startswith("format") and "binary_little_endian" not in line:
                raise ValueError("only binary little-endian PLY is supported")
            if line.startswith("element vertex"):
                n = int(line.split()[2])
            elif line.startswith("property"):
                parts = line.split()
                if parts[1] not in ("float", "float32"):
                    raise ValueError(f"unsupported property type {parts[1]}")
                names.append(parts[2])
            elif line == "end_header":
                break
            elif not line:
                raise ValueError("truncated PLY header")
        if n is None:
            raise ValueError("no vertex element")
        a = np.frombuffer(f.read(4 * n * len(names)), dtype="<f4").reshape(n, len(names)).astype(np.float32)
    col = {nm: i for i, nm in enumerate(names)}

    def take(*keys):
        return np.stack([a[:, col[k]] for k in keys], 1)

    n_rest = sum(1 for nm in names if nm.startswith("f_rest_"))
    k = 1 + n_rest // 3
    deg = int(round(np.sqrt(k))) - 1
    if (deg + 1) ** 2 != k:
        raise ValueError(f"{n_rest} rest coefficients is not a full SH degree")
    sh = np.zeros((n, k, 3), np.float32)
    sh[:, 0, :] = take("f_dc_0", "f_dc_1", "f_dc_2")
    if k > 1:
        rest = take(*[f"f_rest_{i}" for i in range(n_rest)]).reshape(n, 3, k - 1)
        sh[:, 1:, :] = np.transpose(rest, (0, 2, 1))
    op = a[:, col["opacity"]]
    if "opacity_1" in col:
        op = np.stack([op, a[:, col["opacity_1"]]], 1)
    skew = take("skew_0", "skew_1", "skew_2") if "skew_0" in col else np.zeros((n, 3), np.float32)
    split = take("split_0", "split_1", "split_2") if "split_0" in col else None
    return Scene(take("x", "y", "z"), take("scale_0", "scale_1", "scale_2"), take("rot_0", "rot_1", "rot_2", "rot_3"),
                 np.ascontiguousarray(op), skew, sh, deg, split, {"source": str(path)})
