"""Point clouds to and from PLY files (binary little-endian or ASCII), for
viewing reference, template and moved clouds offline.  Only vertex x, y, z
(float32) are written; reading accepts float or double x, y, z and skips
other vertex properties."""
from __future__ import annotations

import numpy as np

_PLY_TYPES = {"char": "i1", "uchar": "u1", "short": "<i2", "ushort": "<u2", "int": "<i4", "uint": "<u4",
              "float": "<f4", "double": "<f8", "int8": "i1", "uint8": "u1", "int16": "<i2", "uint16": "<u2",
              "int32": "<i4", "uint32": "<u4", "float32": "<f4", "float64": "<f8"}


def write_ply(path: str, xyz, binary: bool = True) -> None:
    """Write an [n][3] cloud as PLY vertices (float32)."""
    P = np.ascontiguousarray(np.asarray(xyz, dtype=np.float32).reshape(-1, 3))
    fmt = "binary_little_endian" if binary else "ascii"
    head = (f"ply\nformat {fmt} 1.0\nelement vertex {len(P)}\n"
            "property float x\nproperty float y\nproperty float z\nend_header\n")
    with open(path, "wb") as f:
        f.write(head.encode("ascii"))
        if binary:
            f.write(P.astype("<f4").tobytes())
        else:
            for x, y, z in P:
                f.write(f"{float(x)!r} {float(y)!r} {float(z)!r}\n".encode("ascii"))


def read_ply(path: str) -> np.ndarray:
    """Read the vertex x, y, z of a PLY file as float32 [n][3]."""
    with open(path, "rb") as f:
        if f.readline().strip() != b"ply":
            raise ValueError("not a PLY file")
        fmt, nvert, props, elem = None, None, [], None
        while True:
            line = f.readline()
            if not line:
                raise ValueError("PLY header has no end_header")
            tok = line.decode("ascii").split()
            if not tok:
                continue
            if tok[0] == "format":
                fmt = tok[1]
            elif tok[0] == "element":
                elem = tok[1]
                if elem == "vertex":
                    nvert = int(tok[2])
            elif tok[0] == "property" and elem == "vertex":
                if tok[1] == "list":
                    raise ValueError("list properties on vertices are not supported")
                props.append((tok[2], _PLY_TYPES[tok[1]]))
            elif tok[0] == "end_header":
                break
        names = [n for n, _ in props]
        if nvert is None or not all(c in names for c in "xyz"):
            raise ValueError("PLY file has no vertex x, y, z")
        if fmt == "binary_little_endian":
            data = np.frombuffer(f.read(nvert * np.dtype(props).itemsize), dtype=np.dtype(props), count=nvert)
            return np.stack([data["x"], data["y"], data["z"]], axis=1).astype(np.float32)
        if fmt == "ascii":
            rows = [f.readline().split() for _ in range(nvert)]
            ix = [names.index(c) for c in "xyz"]
            return np.array([[float(r[i]) for i in ix] for r in rows], dtype=np.float32).reshape(-1, 3)
        raise ValueError(f"unsupported PLY format {fmt}")
