"""Scene files on the CPU: 3D-GS PLY round trips, a hand-written PLY in the
training layout, and .pt scenes with their metadata."""
import numpy as np
import pytest

from paper_2604_18980_gb300 import scene_io as S
from paper_2604_18980_gb300 import synth


def _scene(n=257, seed=3):
    scene, _, _ = synth.workload("c1_cube16k_256", n=n, width=32, height=32)
    return scene


@pytest.mark.parametrize("deg", [0, 1, 3])
def test_ply_round_trip(tmp_path, deg):
    scene = _scene()
    p = str(tmp_path / "s.ply")
    S.write_ply(p, scene, sh_degree=deg)
    got = S.read_ply(p)
    assert got["sh_degree"] == deg
    for k in ("mean", "log_scale", "quat", "opacity_logit"):
        np.testing.assert_array_equal(got[k], np.asarray(scene[k], np.float32))
    nc = (deg + 1) ** 2
    np.testing.assert_array_equal(got["sh"][:nc], np.asarray(scene["sh"], np.float32)[:nc])
    assert not got["sh"][nc:].any()


def test_ply_in_the_training_layout(tmp_path):
    """Properties in another order, an extra normal, double opacity, SH degree 1:
    f_rest_j is coefficient j mod 3 + 1 of channel j div 3."""
    n = 2
    props = [("rot_0", "<f4"), ("rot_1", "<f4"), ("rot_2", "<f4"), ("rot_3", "<f4"), ("x", "<f4"), ("y", "<f4"),
             ("z", "<f4"), ("nx", "<f4"), ("opacity", "<f8"), ("scale_0", "<f4"), ("scale_1", "<f4"),
             ("scale_2", "<f4"), ("f_dc_0", "<f4"), ("f_dc_1", "<f4"), ("f_dc_2", "<f4")]
    props += [("f_rest_%d" % j, "<f4") for j in range(9)]
    rec = np.zeros(n, dtype=np.dtype(props))
    for i in range(n):
        rec["x"][i], rec["y"][i], rec["z"][i] = 1 + i, 2 + i, 3 + i
        rec["rot_0"][i], rec["rot_3"][i] = 0.5, 0.25
        rec["opacity"][i] = -0.75 + i
        rec["scale_0"][i], rec["scale_1"][i], rec["scale_2"][i] = -1, -2, -3
        rec["f_dc_0"][i], rec["f_dc_1"][i], rec["f_dc_2"][i] = 0.1, 0.2, 0.3
        for j in range(9):
            rec["f_rest_%d" % j][i] = 10 * j + i
    tstr = {"<f4": "float", "<f8": "double"}
    hdr = "ply\nformat binary_little_endian 1.0\ncomment made by hand\nelement vertex %d\n" % n
    hdr += "".join("property %s %s\n" % (tstr[t], nm) for nm, t in props) + "end_header\n"
    p = tmp_path / "h.ply"
    with open(p, "wb") as f:
        f.write(hdr.encode())
        rec.tofile(f)
    s = S.read_ply(str(p))
    assert s["sh_degree"] == 1
    np.testing.assert_array_equal(s["mean"][:, 1], [2, 3, 4])
    np.testing.assert_array_equal(s["quat"][:, 0], [0.5, 0, 0, 0.25])
    np.testing.assert_array_equal(s["opacity_logit"], [-0.75, 0.25])
    np.testing.assert_array_equal(s["log_scale"][:, 0], [-1, -2, -3])
    np.testing.assert_array_equal(s["sh"][0, :, 0], np.float32([0.1, 0.2, 0.3]))
    for c in range(3):
        for k in range(3):
            np.testing.assert_array_equal(s["sh"][k + 1, c], [10 * (3 * c + k), 10 * (3 * c + k) + 1])


def test_ply_rejects_what_it_cannot_read(tmp_path):
    p = tmp_path / "a.ply"
    p.write_bytes(b"ply\nformat ascii 1.0\nelement vertex 0\nend_header\n")
    with pytest.raises(ValueError, match="binary_little_endian"):
        S.read_ply(str(p))
    p.write_bytes(b"not a ply\n")
    with pytest.raises(ValueError, match="not a PLY"):
        S.read_ply(str(p))
    p.write_bytes(b"ply\nformat binary_little_endian 1.0\nelement vertex 1\nproperty float x\nend_header\n")
    with pytest.raises(ValueError):
        S.read_ply(str(p))


def test_pt_scene_round_trip(tmp_path):
    scene = _scene()
    p = str(tmp_path / "s.pt")
    S.save_scene(p, scene, seed=1001, workload="c1_cube16k_256", note="round trip")
    got, meta = S.load_scene(p)
    assert meta == dict(seed=1001, workload="c1_cube16k_256", note="round trip")
    for k in S.SCENE_KEYS:
        np.testing.assert_array_equal(got[k], np.asarray(scene[k], np.float32))
