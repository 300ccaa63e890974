"""PQR reading and OFF round trips (host-side)."""
import numpy as np

from paper_1611_03474_gb300.io import read_off, read_pqr, write_off


def test_read_pqr_fields(tmp_path):
    p = tmp_path / "m.pqr"
    p.write_text("REMARK test\n"
                 "ATOM      1  N   ALA A   1      -1.234   2.500  10.000 -0.3000 1.8240\n"
                 "HETATM    2  O   HOH W   2       0.000  -3.125   4.5    0.4170 1.5200\n"
                 "ATOM      3  CA  GLYA1000      12.000  13.000  14.000  0.1000 1.9080\n"
                 "TER\nEND\n")
    xyz, r, q = read_pqr(str(p))
    assert xyz.shape == (3, 3)
    assert np.allclose(xyz[0], [-1.234, 2.5, 10.0]) and np.allclose(xyz[2], [12.0, 13.0, 14.0])
    assert np.allclose(r, [1.824, 1.52, 1.908]) and np.allclose(q, [-0.3, 0.417, 0.1])


def test_off_round_trip(tmp_path):
    rng = np.random.default_rng(0)
    v = rng.normal(size=(50, 3))
    t = rng.integers(0, 50, size=(80, 3))
    p = tmp_path / "m.off"
    write_off(str(p), v, t)
    v2, t2 = read_off(str(p))
    assert np.array_equal(v, v2) and np.array_equal(t, t2)
