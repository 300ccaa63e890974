"""CPU oracle for the TMSmesh 2.0 meshing path (test infrastructure).

Plain FP64 C (gs_oracle.c) behind ctypes.  Only the test-suite, the smoke
check and the benchmark's CPU-baseline leg may import this package; the
CUDA library never does, and this package never imports the library.

Parity status: pinned by tests/test_oracle_*.py against closed forms, library
routines and brute force; the triangulation of general inputs is pinned by
invariants only (closed manifold, |g - c| = 0 at surface points, consistent
orientation, single-valued pieces).
"""
import ctypes
import os
import platform
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gs_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libgsoracle.so")

DISCARD, ACCEPT, SPLIT, FORCED = 0, 1, 2, 3
CUTOFF_REL = 1e-8


def build(force=False):
    """Compile gs_oracle.c with gcc (-O2, no FP contraction, no fast-math),
    with OpenMP when the compiler has it (the loops over cubes and points
    then run in parallel; the output is the same for any thread count)."""
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + ".tmp%d" % os.getpid()
    base = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    if platform.machine() in ("x86_64", "AMD64"):
        base.append("-lquadmath")   # __float128 for the resolve mode (AArch64 has a binary128 long double)
    try:
        subprocess.check_call(base[:1] + ["-fopenmp"] + base[1:], stderr=subprocess.DEVNULL)
    except subprocess.CalledProcessError:
        subprocess.check_call(base)
    os.replace(tmp, _LIB)
    return _LIB


def set_threads(n):
    """Threads for the oracle's parallel loops (0: OpenMP's default).
    Returns the number that will be used (1 without OpenMP)."""
    return int(lib().or_set_threads(int(n)))


class Stats(ctypes.Structure):
    _fields_ = [("examined", ctypes.c_int64 * 21), ("discarded", ctypes.c_int64 * 21),
                ("accepted", ctypes.c_int64 * 21), ("forced", ctypes.c_int64 * 21),
                ("split", ctypes.c_int64 * 21), ("pair_terms", ctypes.c_int64),
                ("conformity_splits", ctypes.c_int64), ("vertex_terms", ctypes.c_int64),
                ("n_vertices_lattice", ctypes.c_int64), ("n_cubes_final", ctypes.c_int64),
                ("n_cubes_surface", ctypes.c_int64), ("open_faces", ctypes.c_int64),
                ("degenerate_ears", ctypes.c_int64), ("loop_errors", ctypes.c_int64),
                ("min_margin", ctypes.c_double), ("constrained_vertices", ctypes.c_int64),
                ("agreement_splits", ctypes.c_int64), ("near", ctypes.c_int64 * 4),
                ("resolved_cubes", ctypes.c_int64), ("resolved_vertices", ctypes.c_int64),
                ("resolved_changed", ctypes.c_int64), ("vertex_sign_changed", ctypes.c_int64)]


class MeshOut(ctypes.Structure):
    _fields_ = [("n_vertices", ctypes.c_int64), ("n_triangles", ctypes.c_int64),
                ("n_cubes", ctypes.c_int64), ("n_accepted_pre", ctypes.c_int64),
                ("vertices", ctypes.POINTER(ctypes.c_double)),
                ("vkeys", ctypes.POINTER(ctypes.c_uint64)),
                ("triangles", ctypes.POINTER(ctypes.c_int32)),
                ("tri_piece", ctypes.POINTER(ctypes.c_int64)),
                ("cube_keys", ctypes.POINTER(ctypes.c_uint64)),
                ("pre_keys", ctypes.POINTER(ctypes.c_uint64)),
                ("n_lattice", ctypes.c_int64),
                ("lattice_keys", ctypes.POINTER(ctypes.c_uint64)),
                ("lattice_phi", ctypes.POINTER(ctypes.c_double)),
                ("lattice_psi", ctypes.POINTER(ctypes.c_double)),
                ("st", Stats)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        d, i64, i32, p = ctypes.c_double, ctypes.c_int64, ctypes.c_int, ctypes.c_void_p
        L.or_sizeof_mesh_out.restype = i32
        assert L.or_sizeof_mesh_out() == ctypes.sizeof(MeshOut), "oracle struct layout mismatch"
        L.or_axis_projection.argtypes = [d, d, d, d, i32, p]
        L.or_axis_coeffs.argtypes = [d, d, d, d, p]
        L.or_svd_rows.argtypes = [p, i32, i32, p, p, p]
        L.or_cubic_bounds.argtypes = [p, p, p]
        L.or_bounds.argtypes = [p, p]
        L.or_decide.argtypes = [p, d, d, i32, i32, p]
        L.or_decide.restype = i32
        L.or_decide_ex.argtypes = [p, d, d, i32, i32, i32, i32, p]
        L.or_decide_ex.restype = i32
        L.or_high_norm.argtypes = [p, i32]
        L.or_high_norm.restype = d
        L.or_root_grid.argtypes = [i64, p, p, d, d, d, d, i32, p, p, p]
        L.or_root_grid.restype = i32
        L.or_field.argtypes = [i64, p, p, d, d, d, i64, p, p, p]
        L.or_field.restype = i32
        L.or_cube_tensor.argtypes = [i64, p, p, d, d, d, p, d, p]
        L.or_cube_tensor.restype = i64
        L.or_cube_batch.argtypes = [i64, p, p, d, d, d, d, d, i32, i64, p, p, p, p]
        L.or_cube_batch.restype = i32
        L.or_mesh.argtypes = [i64, p, p, d, d, d, d, d, i32, ctypes.POINTER(MeshOut)]
        L.or_mesh.restype = i32
        L.or_partition.argtypes = [i64, p, p, d, d, d, d, d, i32, ctypes.POINTER(MeshOut)]
        L.or_partition.restype = i32
        L.or_mesh_free.argtypes = [ctypes.POINTER(MeshOut)]
        L.or_mesh_grid.argtypes = [i64, i64, i64, p, d, ctypes.POINTER(MeshOut)]
        L.or_mesh_ex.argtypes = [i64, p, p, d, d, d, d, d, i32, i32, i32, i32, i32, ctypes.POINTER(MeshOut)]
        L.or_mesh_ex.restype = i32
        L.or_mesh_ex2.argtypes = [i64, p, p, d, d, d, d, d, i32, i32, i32, i32, i32, i32, ctypes.POINTER(MeshOut)]
        L.or_mesh_ex2.restype = i32
        L.or_have_quad.restype = i32
        if L.or_have_quad():
            L.or_axis_coeffs_quad.argtypes = [d, d, d, d, p, p]
            L.or_axis_coeffs_quad.restype = i32
            L.or_field_quad.argtypes = [i64, p, p, d, d, d, i64, p, p, p]
            L.or_field_quad.restype = i32
            L.or_bounds_quad.argtypes = [p, p, p]
            L.or_bounds_quad.restype = i32
        L.or_child_reexpand.argtypes = [p, i32, p]
        L.or_child_reexpand.restype = None
        L.or_mesh_grad.argtypes = [i64, p, p, d, d, d, d, d, i32, i64, p, p, p, p]
        L.or_mesh_grad.restype = i32
        L.or_volume_area.argtypes = [i64, p, i64, p, p]
        L.or_volume_area.restype = None
        L.or_mesh_grid.restype = i32
        L.or_set_threads.argtypes = [i32]
        L.or_set_threads.restype = i32
        _lib = L
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def axis_projection(xi, a, b, D, q=24):
    out = np.zeros(4)
    lib().or_axis_projection(xi, a, b, D, q, _ptr(out))
    return out


def axis_coeffs(xi, a, b, D):
    """Legendre coefficients of exp(-D (x-xi)^2) on [a,b] with the C0 correction."""
    out = np.zeros(4)
    lib().or_axis_coeffs(xi, a, b, D, _ptr(out))
    return out


def svd_rows(X):
    X = _f64(X)
    m, n = X.shape
    s, u, v = np.zeros(m), np.zeros((m, m)), np.zeros((m, n))
    lib().or_svd_rows(_ptr(X), m, n, _ptr(s), _ptr(u), _ptr(v))
    return s, u, v


def cubic_bounds(cf):
    cf = _f64(cf)
    lo, hi = ctypes.c_double(), ctypes.c_double()
    lib().or_cubic_bounds(_ptr(cf), ctypes.byref(lo), ctypes.byref(hi))
    return lo.value, hi.value


def bounds(A):
    """(L, U, sum|R|, sum|high|, rank j, sum of inner ranks) for a 4x4x4 tensor."""
    A = _f64(A, (64,))
    out = np.zeros(6)
    lib().or_bounds(_ptr(A), _ptr(out))
    return out


def decide(A, c, precision, level, max_depth, order=0, norm=0):
    """Decision for one cube; order 1 is the literal order of steps 2-3,
    norm 1/2 measure the high-order coefficients by max |.| / Euclidean norm."""
    A = _f64(A, (64,))
    out = np.zeros(6)
    d = lib().or_decide_ex(_ptr(A), c, precision, level, max_depth, order, norm, _ptr(out))
    return d, out


def high_norm(A, norm):
    A = _f64(A, (64,))
    return lib().or_high_norm(_ptr(A), int(norm))


def root_grid(xyz, r, D, c, min_edge, max_depth, cutoff_rel=CUTOFF_REL):
    xyz, r = _f64(xyz), _f64(r)
    origin, nroot, pad = np.zeros(3), np.zeros(3, dtype=np.int64), ctypes.c_double()
    e = lib().or_root_grid(len(r), _ptr(xyz), _ptr(r), D, c, cutoff_rel, min_edge, max_depth,
                           _ptr(origin), _ptr(nroot), ctypes.byref(pad))
    if e:
        raise ValueError("oracle status %d" % e)
    return origin, nroot, pad.value


def field(xyz, r, D, c, pts, cutoff_rel=CUTOFF_REL, grad=False):
    xyz, r, pts = _f64(xyz), _f64(r), _f64(pts).reshape(-1, 3)
    phi = np.zeros(len(pts))
    g = np.zeros((len(pts), 3)) if grad else None
    e = lib().or_field(len(r), _ptr(xyz), _ptr(r), D, c, cutoff_rel, len(pts), _ptr(pts), _ptr(phi), _ptr(g))
    if e:
        raise ValueError("oracle status %d" % e)
    return (phi, g) if grad else phi


def cube_tensor(xyz, r, D, c, lo, h, cutoff_rel=CUTOFF_REL):
    xyz, r, lo = _f64(xyz), _f64(r), _f64(lo)
    A = np.zeros(64)
    cnt = lib().or_cube_tensor(len(r), _ptr(xyz), _ptr(r), D, c, cutoff_rel, _ptr(lo), h, _ptr(A))
    return A.reshape(4, 4, 4), cnt


def cube_batch(xyz, r, D, c, precision, min_edge, max_depth, keys, cutoff_rel=CUTOFF_REL):
    xyz, r = _f64(xyz), _f64(r)
    keys = np.ascontiguousarray(keys, dtype=np.uint64)
    n = len(keys)
    A, bnd, dec = np.zeros((n, 64)), np.zeros((n, 6)), np.zeros(n, dtype=np.int32)
    e = lib().or_cube_batch(len(r), _ptr(xyz), _ptr(r), D, c, cutoff_rel, precision, min_edge,
                            max_depth, n, _ptr(keys), _ptr(A), _ptr(bnd), _ptr(dec))
    if e:
        raise ValueError("oracle status %d" % e)
    return A, bnd, dec


def _stats_dict(st, max_depth):
    lv = lambda arr: [int(arr[i]) for i in range(max_depth + 1)]
    return dict(examined=lv(st.examined), discarded=lv(st.discarded), accepted=lv(st.accepted),
                forced=lv(st.forced), split=lv(st.split), pair_terms=int(st.pair_terms),
                conformity_splits=int(st.conformity_splits),
                n_vertices_lattice=int(st.n_vertices_lattice), n_cubes_final=int(st.n_cubes_final),
                n_cubes_surface=int(st.n_cubes_surface), open_faces=int(st.open_faces),
                degenerate_ears=int(st.degenerate_ears), loop_errors=int(st.loop_errors),
                min_margin=float(st.min_margin), constrained_vertices=int(st.constrained_vertices),
                agreement_splits=int(st.agreement_splits), near=[int(st.near[k]) for k in range(4)],
                resolved_cubes=int(st.resolved_cubes), resolved_vertices=int(st.resolved_vertices),
                resolved_changed=int(st.resolved_changed), vertex_sign_changed=int(st.vertex_sign_changed))


def _arr(ptr, n, dtype, shape=None):
    if n == 0 or not ptr:
        out = np.zeros((0,) if shape is None else (0,) + shape[1:], dtype=dtype)
        return out
    a = np.ctypeslib.as_array(ptr, shape=(n if shape is None else int(np.prod(shape)),)).astype(dtype).copy()
    return a if shape is None else a.reshape(shape)


def child_reexpand(A, c8):
    """Coefficients on child c8 of the polynomial with coefficients A[4,4,4]."""
    A = _f64(A, (64,))
    B = np.zeros(64)
    lib().or_child_reexpand(_ptr(A), int(c8), _ptr(B))
    return B.reshape(4, 4, 4)


def have_quad():
    """Whether the oracle was built with a binary128 type (the resolve mode)."""
    return bool(lib().or_have_quad())


def axis_coeffs_quad(xi, a, b, D):
    """axis_coeffs in quad precision, as (hi, lo) double pairs (value = hi + lo)."""
    hi, lo = np.zeros(4), np.zeros(4)
    lib().or_axis_coeffs_quad(xi, a, b, D, _ptr(hi), _ptr(lo))
    return hi, lo


def field_quad(xyz, r, D, c, pts, cutoff_rel=CUTOFF_REL):
    """field in quad precision, as (hi, lo) double pairs."""
    xyz, r, pts = _f64(xyz), _f64(r), _f64(pts).reshape(-1, 3)
    hi, lo = np.zeros(len(pts)), np.zeros(len(pts))
    e = lib().or_field_quad(len(r), _ptr(xyz), _ptr(r), D, c, cutoff_rel, len(pts), _ptr(pts), _ptr(hi), _ptr(lo))
    if e:
        raise ValueError("oracle status %d" % e)
    return hi, lo


def bounds_quad(A_hi, A_lo=None):
    """(L, U, sum|R|, rank) of section 2.2.2 in quad precision for a tensor
    given as hi + lo doubles."""
    A_hi = _f64(A_hi, (64,))
    A_lo = np.zeros(64) if A_lo is None else _f64(A_lo, (64,))
    out = np.zeros(4)
    lib().or_bounds_quad(_ptr(A_hi), _ptr(A_lo), _ptr(out))
    return out


def mesh(xyz, r, D, c, precision, min_edge, max_depth, cutoff_rel=CUTOFF_REL, child_mode=0, order=0, norm=0,
         conform=0, resolve=False):
    """Whole path; returns dict(vertices, vkeys, triangles, cube_keys, pre_keys, stats, ...).
    child_mode 1: child tensors by re-expansion of the parent's polynomial;
    order 1: literal order of steps 2-3; norm 1/2: max |.| / Euclidean norm
    of the high-order coefficients in the precision test; conform 1: cubes
    sharing a face or an edge are split to one size (instead of constrained
    vertex values with at most one level between them).  stats["near"]
    counts the decisions whose margin is below 1e-10 relative (bound test,
    precision test, rank rule, vertex sign); resolve=True takes each of them
    again in quad precision."""
    xyz, r = _f64(xyz), _f64(r)
    out = MeshOut()
    L = lib()
    e = L.or_mesh_ex2(len(r), _ptr(xyz), _ptr(r), D, c, cutoff_rel, precision, min_edge, max_depth, child_mode,
                      order, norm, conform, 1 if resolve else 0, ctypes.byref(out))
    if e:
        raise ValueError("oracle status %d" % e)
    try:
        res = dict(
            vertices=_arr(out.vertices, out.n_vertices, np.float64, (out.n_vertices, 3)),
            vkeys=_arr(out.vkeys, out.n_vertices, np.uint64),
            triangles=_arr(out.triangles, out.n_triangles, np.int32, (out.n_triangles, 3)),
            cube_keys=_arr(out.cube_keys, out.n_cubes, np.uint64),
            pre_keys=_arr(out.pre_keys, out.n_accepted_pre, np.uint64),
            lattice_keys=_arr(out.lattice_keys, out.n_lattice, np.uint64),
            lattice_phi=_arr(out.lattice_phi, out.n_lattice, np.float64),
            lattice_psi=_arr(out.lattice_psi, out.n_lattice, np.float64),
            stats=_stats_dict(out.st, max_depth))
    finally:
        L.or_mesh_free(ctypes.byref(out))
    return res


def mesh_grad(xyz, r, D, c, precision, min_edge, max_depth, dLdp, cutoff_rel=CUTOFF_REL):
    """(dL/dxyz [n,3], dL/dr [n], dL/dD) from dL/dp [nv,3] in the order of
    mesh()'s vertices (sorted keys); cube set and topology held fixed."""
    xyz, r = _f64(xyz), _f64(r)
    g = _f64(dLdp).reshape(-1, 3)
    gx, gr, gD = np.zeros((len(r), 3)), np.zeros(len(r)), np.zeros(1)
    e = lib().or_mesh_grad(len(r), _ptr(xyz), _ptr(r), D, c, cutoff_rel, precision, min_edge, max_depth, len(g),
                           _ptr(g), _ptr(gx), _ptr(gr), _ptr(gD))
    if e:
        raise ValueError("oracle status %d" % e)
    return gx, gr, float(gD[0])


def volume_area(vertices, triangles):
    """(volume, area) of a closed outward mesh (plain sums)."""
    v = _f64(vertices).reshape(-1, 3)
    t = np.ascontiguousarray(triangles, dtype=np.int32)
    out = np.zeros(2)
    lib().or_volume_area(len(v), _ptr(v), len(t), _ptr(t), _ptr(out))
    return out[0], out[1]


def partition(xyz, r, D, c, precision, min_edge, max_depth, cutoff_rel=CUTOFF_REL):
    """Level loop only; returns (sorted accepted cube keys, stats)."""
    xyz, r = _f64(xyz), _f64(r)
    out = MeshOut()
    L = lib()
    e = L.or_partition(len(r), _ptr(xyz), _ptr(r), D, c, cutoff_rel, precision, min_edge, max_depth,
                       ctypes.byref(out))
    if e:
        raise ValueError("oracle status %d" % e)
    try:
        keys = _arr(out.pre_keys, out.n_accepted_pre, np.uint64)
        st = _stats_dict(out.st, max_depth)
    finally:
        L.or_mesh_free(ctypes.byref(out))
    return keys, st


def mesh_grid(values, c):
    """Triangulate a uniform grid of corner values (array [nz+1, ny+1, nx+1])."""
    values = np.ascontiguousarray(values, dtype=np.float64)
    nz, ny, nx = (d - 1 for d in values.shape)
    out = MeshOut()
    L = lib()
    e = L.or_mesh_grid(nx, ny, nz, _ptr(values), c, ctypes.byref(out))
    if e:
        raise ValueError("oracle status %d" % e)
    try:
        res = dict(vertices=_arr(out.vertices, out.n_vertices, np.float64, (out.n_vertices, 3)),
                   vkeys=_arr(out.vkeys, out.n_vertices, np.uint64),
                   triangles=_arr(out.triangles, out.n_triangles, np.int32, (out.n_triangles, 3)),
                   tri_piece=_arr(out.tri_piece, out.n_triangles, np.int64),
                   stats=_stats_dict(out.st, 0))
    finally:
        L.or_mesh_free(ctypes.byref(out))
    return res


def cell_list(xyz, cell, origin, dims):
    """Uniform cell list by definition: cell = floor((x - origin)/cell) clamped
    to [0, dims-1], linear index x + dims0*(y + dims1*z); atoms ordered by
    cell, ties by ascending atom index (a stable sort)."""
    xyz = np.asarray(xyz, dtype=np.float64)
    origin = np.asarray(origin, dtype=np.float64)
    dims = np.asarray(dims, dtype=np.int64)
    c = np.floor((xyz - origin) * (1.0 / cell)).astype(np.int64)
    c = np.clip(c, 0, dims - 1)
    lin = c[:, 0] + dims[0] * (c[:, 1] + dims[1] * c[:, 2])
    perm = np.argsort(lin, kind="stable").astype(np.int32)
    counts = np.bincount(lin, minlength=int(np.prod(dims)))
    start = np.concatenate([[0], np.cumsum(counts)]).astype(np.int32)
    return start, perm
