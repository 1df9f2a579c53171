"""Gaussian-splat PLY files on the host (Algorithm 1 reads its input splats
(mu, alpha, s, q, f) from a PLY file and writes the simplified set back).

The layout is the one 3D Gaussian Splatting writes, one ``vertex`` element
with scalar properties:

    x y z                    centre mu
    nx ny nz                 unused normals (written as zeros)
    f_dc_0..2, f_rest_*      SH coefficients f (DC first, then the rest in
                             file order)
    opacity                  opacity logit (alpha = sigmoid(opacity))
    scale_0..2               log scales s
    rot_0..3                 quaternion q in (w, x, y, z) order

The SH coefficients are kept in file order, [f_dc_0, f_dc_1, f_dc_2,
f_rest_0, ...].  Every operation of the method on f (the appearance distance
and the mass-weighted mean of a merge) acts on each coefficient alone, so
the order never changes a result and a file is written back as it was read.

Reading accepts ``ascii``, ``binary_little_endian`` and ``binary_big_endian``
files, any scalar property type, extra vertex properties (ignored) and other
elements with scalar properties before the vertex element (any element after
it).  Writing produces ``binary_little_endian`` float32.
"""
from __future__ import annotations

import os

import numpy as np

from .synth import Scene

_TYPES = {
    "char": "i1", "int8": "i1", "uchar": "u1", "uint8": "u1",
    "short": "i2", "int16": "i2", "ushort": "u2", "uint16": "u2",
    "int": "i4", "int32": "i4", "uint": "u4", "uint32": "u4",
    "float": "f4", "float32": "f4", "double": "f8", "float64": "f8",
}
_FORMATS = {"ascii": None, "binary_little_endian": "<", "binary_big_endian": ">"}


class PlyError(ValueError):
    """The file is not a Gaussian-splat PLY this module can read."""


def _parse_header(f):
    if f.readline().strip() != b"ply":
        raise PlyError("not a PLY file (missing 'ply' magic)")
    fmt, elements = None, []
    while True:
        line = f.readline()
        if not line:
            raise PlyError("header ends before 'end_header'")
        words = line.decode("ascii", "replace").split()
        if not words or words[0] in ("comment", "obj_info"):
            continue
        if words[0] == "end_header":
            break
        if words[0] == "format":
            if len(words) < 2 or words[1] not in _FORMATS:
                raise PlyError(f"unsupported format line: {line!r}")
            fmt = words[1]
        elif words[0] == "element":
            if len(words) != 3:
                raise PlyError(f"bad element line: {line!r}")
            elements.append((words[1], int(words[2]), []))
        elif words[0] == "property":
            if not elements:
                raise PlyError("property before any element")
            if len(words) >= 2 and words[1] == "list":
                elements[-1][2].append((words[-1], None))
            else:
                if len(words) != 3 or words[1] not in _TYPES:
                    raise PlyError(f"bad property line: {line!r}")
                elements[-1][2].append((words[2], _TYPES[words[1]]))
        else:
            raise PlyError(f"unknown header line: {line!r}")
    if fmt is None:
        raise PlyError("no format line")
    return fmt, elements


def _sorted_names(names, prefix):
    idx = sorted(int(n[len(prefix):]) for n in names if n.startswith(prefix)
                 and n[len(prefix):].isdigit())
    if idx != list(range(len(idx))):
        raise PlyError(f"properties {prefix}* are not numbered 0..{len(idx) - 1}")
    return [f"{prefix}{i}" for i in idx]


def read_ply(path: str | os.PathLike) -> Scene:
    """Read the splats of a Gaussian-splat PLY file into FP32 arrays."""
    with open(path, "rb") as f:
        fmt, elements = _parse_header(f)
        order = _FORMATS[fmt]
        vertex = None
        for name, count, props in elements:
            if name == "vertex":
                if any(t is None for _, t in props):
                    raise PlyError("list properties in the vertex element are not supported")
                if len({p for p, _ in props}) != len(props):
                    raise PlyError("a vertex property is declared twice")
                if fmt == "ascii":
                    cols = [p for p, _ in props]
                    data = np.loadtxt(f, dtype=np.float64, max_rows=count, ndmin=2)
                    if count and data.shape != (count, len(cols)):
                        raise PlyError("ascii vertex rows do not match the header")
                    vertex = {c: data[:, k] if count else np.zeros(0) for k, c in enumerate(cols)}
                else:
                    dt = np.dtype([(p, order + t) for p, t in props])
                    raw = f.read(dt.itemsize * count)
                    if len(raw) != dt.itemsize * count:
                        raise PlyError("file ends inside the vertex element")
                    arr = np.frombuffer(raw, dtype=dt, count=count)
                    vertex = {p: arr[p] for p, _ in props}
                break
            # an element before the vertex element: skip it
            if any(t is None for _, t in props):
                raise PlyError(f"cannot skip element '{name}' with list properties")
            if fmt == "ascii":
                for _ in range(count):
                    f.readline()
            else:
                f.seek(sum(np.dtype(t).itemsize for _, t in props) * count, os.SEEK_CUR)
    if vertex is None:
        raise PlyError("no vertex element")
    names = list(vertex)
    need = ["x", "y", "z", "opacity", "scale_0", "scale_1", "scale_2",
            "rot_0", "rot_1", "rot_2", "rot_3", "f_dc_0", "f_dc_1", "f_dc_2"]
    missing = [p for p in need if p not in vertex]
    if missing:
        raise PlyError(f"missing vertex properties: {', '.join(missing)}")
    sh_names = _sorted_names(names, "f_dc_") + _sorted_names(names, "f_rest_")

    def cols(ps):
        return np.ascontiguousarray(np.stack([vertex[p] for p in ps], axis=1), dtype=np.float32)

    return Scene(cols(["x", "y", "z"]), cols(["scale_0", "scale_1", "scale_2"]),
                 cols(["rot_0", "rot_1", "rot_2", "rot_3"]),
                 np.ascontiguousarray(vertex["opacity"], dtype=np.float32), cols(sh_names))


def write_ply(path: str | os.PathLike, scene: Scene) -> None:
    """Write splats as a binary little-endian float32 Gaussian-splat PLY."""
    n, F = scene.n, scene.sh.shape[1]
    if F < 3:
        raise PlyError("a splat PLY needs at least the three DC coefficients")
    names = (["x", "y", "z", "nx", "ny", "nz"] + [f"f_dc_{i}" for i in range(3)] +
             [f"f_rest_{i}" for i in range(F - 3)] + ["opacity"] +
             [f"scale_{i}" for i in range(3)] + [f"rot_{i}" for i in range(4)])
    out = np.empty((n, len(names)), dtype="<f4")
    out[:, 0:3] = scene.xyz
    out[:, 3:6] = 0.0
    out[:, 6:6 + F] = scene.sh
    out[:, 6 + F] = scene.logit.reshape(-1)
    out[:, 7 + F:10 + F] = scene.log_scale
    out[:, 10 + F:14 + F] = scene.rot
    header = ["ply", "format binary_little_endian 1.0", f"element vertex {n}"]
    header += [f"property float {p}" for p in names] + ["end_header"]
    with open(path, "wb") as f:
        f.write(("\n".join(header) + "\n").encode("ascii"))
        f.write(out.tobytes())
