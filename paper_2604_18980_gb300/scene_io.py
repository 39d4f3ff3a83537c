"""Scene files: trained 3D-GS scenes in PLY form, and the renderer's own
structure-of-arrays scenes saved with their provenance.

PLY (the layout 3D Gaussian Splatting training writes): one `vertex` element
per Gaussian with float properties x y z (mean), optional nx ny nz (unused),
f_dc_0..2 (the degree-0 SH coefficient of R, G, B), f_rest_0..(3M-1) (the
higher bands, channel-major: f_rest_j is coefficient k = j mod M + 1 of
channel c = j div M, M = (degree+1)^2 - 1), opacity (the logit), scale_0..2
(log-scales) and rot_0..3 (the quaternion w, x, y, z, not necessarily
normalised).  The renderer takes the same quantities in SoA planes:
mean[3][N], log_scale[3][N], quat[4][N], opacity_logit[N], sh[16][3][N]
(coefficients beyond the file's degree are zero).

.pt scenes: the SoA arrays plus a metadata dict (seed, workload name, any
configuration) in one torch.save file, for reproducible synthetic runs and
for fine-tuned scenes.
"""
from __future__ import annotations

import math
import re

import numpy as np

_PLY_TYPES = {"float": "<f4", "float32": "<f4", "double": "<f8", "float64": "<f8", "uchar": "u1", "uint8": "u1",
              "char": "i1", "int8": "i1", "ushort": "<u2", "uint16": "<u2", "short": "<i2", "int16": "<i2",
              "uint": "<u4", "uint32": "<u4", "int": "<i4", "int32": "<i4"}


def _read_header(f):
    if f.readline().strip() != b"ply":
        raise ValueError("not a PLY file")
    fmt, count, props, element = None, None, [], None
    while True:
        line = f.readline()
        if not line:
            raise ValueError("PLY header without end_header")
        tok = line.decode("ascii", "replace").split()
        if not tok or tok[0] in ("comment", "obj_info"):
            continue
        if tok[0] == "end_header":
            break
        if tok[0] == "format":
            fmt = tok[1]
        elif tok[0] == "element":
            element = tok[1]
            if element == "vertex":
                count = int(tok[2])
            elif count is None:
                raise ValueError("PLY element %r before the vertices is not supported" % element)
        elif tok[0] == "property" and element == "vertex":
            if tok[1] == "list":
                raise ValueError("list properties are not supported in the vertex element")
            if tok[1] not in _PLY_TYPES:
                raise ValueError("unknown PLY property type %r" % tok[1])
            props.append((tok[2], _PLY_TYPES[tok[1]]))
    if fmt != "binary_little_endian":
        raise ValueError("only binary_little_endian PLY is supported (got %r)" % fmt)
    if count is None:
        raise ValueError("PLY file without a vertex element")
    return count, props


def read_ply(path: str) -> dict:
    """A 3D-GS PLY file as the renderer's SoA float32 arrays (sh padded to 16 coefficients)."""
    with open(path, "rb") as f:
        n, props = _read_header(f)
        dt = np.dtype(props)
        v = np.fromfile(f, dtype=dt, count=n)
    if len(v) != n:
        raise ValueError("PLY file holds %d of its %d vertices" % (len(v), n))
    names = set(dt.names)

    def col(name):
        if name not in names:
            raise ValueError("PLY vertex lacks property %r" % name)
        return np.asarray(v[name], dtype=np.float32)

    rest = sorted((int(m.group(1)) for m in (re.fullmatch(r"f_rest_(\d+)", nm) for nm in names) if m))
    if rest != list(range(len(rest))) or len(rest) % 3:
        raise ValueError("f_rest properties must be f_rest_0 .. f_rest_(3M-1)")
    M = len(rest) // 3
    degree = int(round(math.sqrt(M + 1))) - 1
    if (degree + 1) ** 2 - 1 != M or degree > 3:
        raise ValueError("f_rest holds %d coefficients per channel: not an SH degree <= 3" % M)
    sh = np.zeros((16, 3, n), dtype=np.float32)
    for c in range(3):
        sh[0, c] = col("f_dc_%d" % c)
        for k in range(M):
            sh[k + 1, c] = col("f_rest_%d" % (c * M + k))
    return dict(mean=np.stack([col("x"), col("y"), col("z")]),
                log_scale=np.stack([col("scale_%d" % k) for k in range(3)]),
                quat=np.stack([col("rot_%d" % k) for k in range(4)]),
                opacity_logit=col("opacity"), sh=sh, sh_degree=degree)


def write_ply(path: str, scene: dict, sh_degree: int = 3) -> None:
    """Write SoA arrays as a 3D-GS PLY file (float32, the higher SH bands up to sh_degree)."""
    if not 0 <= sh_degree <= 3:
        raise ValueError("sh_degree must be 0..3")
    mean = np.asarray(scene["mean"], dtype=np.float32)
    n = mean.shape[1]
    M = (sh_degree + 1) ** 2 - 1
    names = ["x", "y", "z", "nx", "ny", "nz", "f_dc_0", "f_dc_1", "f_dc_2"] + ["f_rest_%d" % j for j in range(3 * M)]
    names += ["opacity", "scale_0", "scale_1", "scale_2", "rot_0", "rot_1", "rot_2", "rot_3"]
    rec = np.zeros(n, dtype=np.dtype([(nm, "<f4") for nm in names]))
    for k, nm in enumerate("xyz"):
        rec[nm] = mean[k]
    sh = np.asarray(scene["sh"], dtype=np.float32)
    for c in range(3):
        rec["f_dc_%d" % c] = sh[0, c]
        for k in range(M):
            rec["f_rest_%d" % (c * M + k)] = sh[k + 1, c]
    rec["opacity"] = np.asarray(scene["opacity_logit"], dtype=np.float32)
    ls = np.asarray(scene["log_scale"], dtype=np.float32)
    q = np.asarray(scene["quat"], dtype=np.float32)
    for k in range(3):
        rec["scale_%d" % k] = ls[k]
    for k in range(4):
        rec["rot_%d" % k] = q[k]
    header = "ply\nformat binary_little_endian 1.0\nelement vertex %d\n" % n
    header += "".join("property float %s\n" % nm for nm in names) + "end_header\n"
    with open(path, "wb") as f:
        f.write(header.encode("ascii"))
        rec.tofile(f)


SCENE_KEYS = ("mean", "log_scale", "quat", "opacity_logit", "sh")


def save_scene(path: str, scene: dict, **meta) -> None:
    """The SoA arrays (numpy or torch, saved as CPU float32 tensors) and a
    metadata dict (e.g. seed=, workload=, and any configuration) in one file."""
    import torch
    data = {k: torch.as_tensor(np.asarray(scene[k].detach().cpu() if hasattr(scene[k], "detach") else scene[k]),
                               dtype=torch.float32).contiguous() for k in SCENE_KEYS}
    torch.save(dict(scene=data, meta=dict(meta), format="ags-scene-1"), path)


def load_scene(path: str) -> tuple:
    """(scene as numpy float32 arrays, metadata) from save_scene's file."""
    import torch
    d = torch.load(path, map_location="cpu", weights_only=True)
    if d.get("format") != "ags-scene-1":
        raise ValueError("not a scene file written by save_scene")
    return {k: d["scene"][k].numpy() for k in SCENE_KEYS}, dict(d["meta"])
