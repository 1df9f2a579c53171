"""Host PLY I/O: exact round trips, the three encodings, foreign headers, and
(on the GPU) the file-to-file simplification equal to the in-memory call."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_2603_16103_gb300 import ply, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _scene(n, F, seed):
    s = synth.surfaces_unit_cube(n, seed=seed)
    s.sh = np.ascontiguousarray(s.sh[:, :F])
    return s


@pytest.mark.parametrize("F", [3, 12, 27, 48])
def test_roundtrip_is_bit_exact(tmp_path, F):
    s = _scene(500, F, F)
    s.logit[0] = np.float32(-0.0)
    s.xyz[1] = np.float32(1e-38)
    p = tmp_path / "a.ply"
    ply.write_ply(p, s)
    t = ply.read_ply(p)
    assert t.n == s.n and t.sh.shape == (s.n, F)
    for a, b in zip(s.arrays(), t.arrays()):
        assert a.dtype == b.dtype == np.float32
        assert np.array_equal(a.view(np.uint32), b.view(np.uint32))
    # the standard header: 14 + F properties (62 for degree-3 SH)
    head = p.read_bytes().split(b"end_header\n")[0].decode().splitlines()
    props = [ln.split()[-1] for ln in head if ln.startswith("property")]
    assert props[:9] == ["x", "y", "z", "nx", "ny", "nz", "f_dc_0", "f_dc_1", "f_dc_2"]
    assert props[-8:] == ["opacity", "scale_0", "scale_1", "scale_2", "rot_0", "rot_1", "rot_2",
                          "rot_3"]
    assert len(props) == 14 + F
    assert os.path.getsize(p) == len("\n".join(head)) + 1 + len("end_header\n") + 4 * s.n * (14 + F)


def test_empty_scene_roundtrip(tmp_path):
    s = _scene(10, 48, 1).subset(np.arange(0))
    ply.write_ply(tmp_path / "e.ply", s)
    t = ply.read_ply(tmp_path / "e.ply")
    assert t.n == 0 and t.sh.shape == (0, 48)


def _foreign_rows(rng, n):
    # columns in a foreign order with an extra property and f_rest before f_dc
    return {
        "rot_1": rng.normal(size=n), "x": rng.normal(size=n), "y": rng.normal(size=n),
        "z": rng.normal(size=n), "red": rng.integers(0, 255, n), "f_rest_1": rng.normal(size=n),
        "f_rest_0": rng.normal(size=n), "f_rest_2": rng.normal(size=n),
        "f_dc_0": rng.normal(size=n), "f_dc_1": rng.normal(size=n), "f_dc_2": rng.normal(size=n),
        "opacity": rng.normal(size=n), "scale_0": rng.normal(size=n), "scale_1": rng.normal(size=n),
        "scale_2": rng.normal(size=n), "rot_0": rng.normal(size=n), "rot_2": rng.normal(size=n),
        "rot_3": rng.normal(size=n),
    }


def _check_foreign(t, cols):
    def f32(k):
        return np.asarray(cols[k], np.float32)
    assert np.array_equal(t.xyz, np.stack([f32("x"), f32("y"), f32("z")], 1))
    assert np.array_equal(t.rot, np.stack([f32(f"rot_{i}") for i in range(4)], 1))
    assert np.array_equal(t.log_scale, np.stack([f32(f"scale_{i}") for i in range(3)], 1))
    assert np.array_equal(t.logit, f32("opacity"))
    sh = np.stack([f32(k) for k in ("f_dc_0", "f_dc_1", "f_dc_2", "f_rest_0", "f_rest_1",
                                    "f_rest_2")], 1)
    assert np.array_equal(t.sh, sh)


def test_big_endian_mixed_types_and_skipped_element(tmp_path):
    rng = np.random.default_rng(3)
    n = 37
    cols = _foreign_rows(rng, n)
    types = {k: (">u1" if k == "red" else (">f8" if k in ("x", "opacity") else ">f4")) for k in cols}
    ply_t = {">u1": "uchar", ">f8": "double", ">f4": "float"}
    cam = np.array([(1.5, 7)], dtype=[("fx", ">f4"), ("id", ">i4")])
    arr = np.zeros(n, dtype=[(k, types[k]) for k in cols])
    for k in cols:
        arr[k] = cols[k]
    head = ["ply", "format binary_big_endian 1.0", "comment made by a test",
            "element camera 1", "property float fx", "property int id", f"element vertex {n}"]
    head += [f"property {ply_t[types[k]]} {k}" for k in cols]
    head += ["element face 0", "property list uchar int vertex_indices", "end_header"]
    p = tmp_path / "be.ply"
    p.write_bytes(("\n".join(head) + "\n").encode() + cam.tobytes() + arr.tobytes())
    _check_foreign(ply.read_ply(p), {k: arr[k] for k in cols})


def test_ascii(tmp_path):
    rng = np.random.default_rng(4)
    n = 9
    cols = _foreign_rows(rng, n)
    keys = list(cols)
    head = ["ply", "format ascii 1.0", f"element vertex {n}"]
    head += [f"property {'uchar' if k == 'red' else 'float'} {k}" for k in keys] + ["end_header"]
    rows = [" ".join(repr(float(np.float32(cols[k][i]))) if k != "red" else str(cols[k][i])
                     for k in keys) for i in range(n)]
    p = tmp_path / "a.ply"
    p.write_text("\n".join(head + rows) + "\n")
    _check_foreign(ply.read_ply(p), cols)


@pytest.mark.parametrize("bad,msg", [
    (lambda h: h.replace("property float opacity\n", ""), "missing"),
    (lambda h: h.replace("f_rest_1\n", "f_rest_9\n"), "numbered"),
    (lambda h: h.replace("f_rest_1\n", "f_rest_2\n"), "twice"),
    (lambda h: h.replace("binary_little_endian", "binary_middle_endian"), "format"),
    (lambda h: "plx" + h[3:], "magic"),
])
def test_bad_headers_raise(tmp_path, bad, msg):
    s = _scene(4, 12, 5)
    p = tmp_path / "g.ply"
    ply.write_ply(p, s)
    head, body = p.read_bytes().split(b"end_header\n", 1)
    p.write_bytes(bad(head.decode() + "end_header\n").encode() + body)
    with pytest.raises(ply.PlyError, match=msg):
        ply.read_ply(p)


def test_truncated_body_raises(tmp_path):
    p = tmp_path / "t.ply"
    ply.write_ply(p, _scene(20, 48, 6))
    p.write_bytes(p.read_bytes()[:-5])
    with pytest.raises(ply.PlyError, match="ends inside"):
        ply.read_ply(p)


@pytest.mark.gpu
def test_file_to_file_equals_in_memory(tmp_path, ngs):
    scene = synth.surfaces_unit_cube(30000, seed=12)
    src, dst = tmp_path / "in.ply", tmp_path / "out.ply"
    ply.write_ply(src, scene)
    p = subprocess.run([sys.executable, "-m", "paper_2603_16103_gb300.simplify_ply", str(src),
                        str(dst), "--ratio", "0.1"], capture_output=True, text=True, cwd=ROOT,
                       timeout=600)
    assert p.returncode == 0, p.stderr[-2000:]
    res = json.loads(p.stdout.strip().splitlines()[-1])
    out = ply.read_ply(dst)
    with ngs.Context() as c:
        ds = ngs.DeviceSplats.from_numpy(scene)
        c.simplify(ds, res["target"])
        ref = ds.numpy()
    assert res["target"] == 3000
    assert res["n_output"] == out.n == ref[0].shape[0] >= 3000
    for a, b in zip(out.arrays(), ref):
        assert np.array_equal(a, b)
