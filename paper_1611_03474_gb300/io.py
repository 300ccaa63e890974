"""Molecule and mesh files: PQR input (the paper's input format, section 2.1)
and OFF output (its output format).  Host-side text I/O only."""
import numpy as np


def read_pqr(path):
    """(xyz [n,3], radii [n], charges [n]) from the ATOM/HETATM records of a
    PQR file.  The last five whitespace-separated fields of a record are
    x, y, z, charge, radius (the free-format reading, which also accepts
    records whose name fields run together)."""
    xyz, q, r = [], [], []
    with open(path) as f:
        for line in f:
            if not (line.startswith("ATOM") or line.startswith("HETATM")):
                continue
            parts = line.split()
            if len(parts) < 6:
                raise ValueError("short PQR record: %r" % line)
            x, y, z, c, rad = (float(v) for v in parts[-5:])
            xyz.append((x, y, z))
            q.append(c)
            r.append(rad)
    return np.array(xyz, dtype=np.float64).reshape(-1, 3), np.array(r), np.array(q)


def write_off(path, vertices, triangles):
    """OFF file: header, counts, vertex lines, triangle lines (0-based)."""
    v = np.asarray(vertices, dtype=np.float64).reshape(-1, 3)
    t = np.asarray(triangles, dtype=np.int64).reshape(-1, 3)
    with open(path, "w") as f:
        f.write("OFF\n%d %d 0\n" % (len(v), len(t)))
        np.savetxt(f, v, fmt="%.17g")
        np.savetxt(f, np.hstack([np.full((len(t), 1), 3), t]), fmt="%d")


def read_off(path):
    """(vertices [n,3], triangles [m,3]) of a triangle OFF file."""
    with open(path) as f:
        tokens = f.read().split()
    if not tokens or tokens[0] != "OFF":
        raise ValueError("not an OFF file")
    nv, nf = int(tokens[1]), int(tokens[2])
    p = 4
    v = np.array(tokens[p:p + 3 * nv], dtype=np.float64).reshape(nv, 3)
    p += 3 * nv
    faces = np.array(tokens[p:p + 4 * nf], dtype=np.int64).reshape(nf, 4)
    if nf and not np.all(faces[:, 0] == 3):
        raise ValueError("only triangles are supported")
    return v, faces[:, 1:].copy()
