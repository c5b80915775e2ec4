"""PLY round trips (binary and ASCII) and a header with extra vertex
properties, as written by common scanners."""
import numpy as np

from paper_1902_01061_gb300 import plyio


def test_binary_and_ascii_round_trip(tmp_path):
    P = np.random.default_rng(3).normal(size=(257, 3)).astype(np.float32)
    for binary in (True, False):
        path = str(tmp_path / f"c{int(binary)}.ply")
        plyio.write_ply(path, P, binary=binary)
        np.testing.assert_array_equal(plyio.read_ply(path), P)


def test_reads_double_coordinates_and_extra_properties(tmp_path):
    rec = np.zeros(3, dtype=[("x", "<f8"), ("y", "<f8"), ("z", "<f8"), ("red", "u1"), ("i", "<i4")])
    rec["x"], rec["y"], rec["z"] = [1.5, 2.0, -3.0], [0.0, 1.0, 2.0], [7.0, 8.0, 9.0]
    head = ("ply\nformat binary_little_endian 1.0\ncomment scanner\nelement vertex 3\n"
            "property double x\nproperty double y\nproperty double z\nproperty uchar red\nproperty int i\n"
            "element face 0\nproperty list uchar int vertex_indices\nend_header\n")
    path = tmp_path / "s.ply"
    path.write_bytes(head.encode() + rec.tobytes())
    got = plyio.read_ply(str(path))
    np.testing.assert_array_equal(got, np.stack([rec["x"], rec["y"], rec["z"]], 1).astype(np.float32))
