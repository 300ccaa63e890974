"""ctypes binding of libgsmesh.so (include/gsmesh.h).  Marshalling only."""
import ctypes
import os

import numpy as np

from .build import LIB

GS_PREC_FP64 = 0
GS_PREC_MIXED = 1


class GsError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("gsmesh error %d: %s" % (code, msg))
        self.code = code


class Stats(ctypes.Structure):
    _fields_ = [("examined", ctypes.c_int64 * 21), ("discarded", ctypes.c_int64 * 21),
                ("accepted", ctypes.c_int64 * 21), ("forced", ctypes.c_int64 * 21),
                ("split", ctypes.c_int64 * 21), ("pair_terms", ctypes.c_int64),
                ("vertex_terms", ctypes.c_int64), ("recheck_cubes", ctypes.c_int64),
                ("recheck_vertices", ctypes.c_int64), ("conformity_splits", ctypes.c_int64),
                ("n_cubes_final", ctypes.c_int64), ("n_cubes_surface", ctypes.c_int64),
                ("n_lattice_vertices", ctypes.c_int64), ("n_points", ctypes.c_int64),
                ("n_vertices", ctypes.c_int64), ("n_triangles", ctypes.c_int64),
                ("loop_errors", ctypes.c_int64), ("degenerate_ears", ctypes.c_int64),
                ("ms_total", ctypes.c_double), ("ms_upload", ctypes.c_double), ("ms_bin", ctypes.c_double),
                ("ms_levels", ctypes.c_double), ("ms_conformity", ctypes.c_double),
                ("ms_field", ctypes.c_double), ("ms_triangulate", ctypes.c_double),
                ("ms_weld", ctypes.c_double), ("ms_download", ctypes.c_double),
                ("ms_level", ctypes.c_double * 21), ("ms_accum", ctypes.c_double),
                ("n_accum_launches", ctypes.c_int64), ("atom_octets", ctypes.c_int64),
                ("n_kernel_launches", ctypes.c_int64), ("recheck_bounds", ctypes.c_int64),
                ("recheck_precision", ctypes.c_int64), ("recheck_zero", ctypes.c_int64),
                ("mixed_err_ratio", ctypes.c_double), ("mixed_band_ratio", ctypes.c_double),
                ("recheck_rank", ctypes.c_int64), ("vertex_mark_cubes", ctypes.c_int64 * 3),
                ("estimate_fast_cubes", ctypes.c_int64), ("constrained_vertices", ctypes.c_int64),
                ("agreement_splits", ctypes.c_int64), ("mixed_cubes", ctypes.c_int64), ("retries", ctypes.c_int64),
                ("near_threshold", ctypes.c_int64 * 4), ("refine_vertices", ctypes.c_int64),
                ("vertex_mark_all", ctypes.c_int64), ("vertex_mark_fp64_cubes", ctypes.c_int64 * 3)]

    def as_dict(self, max_depth=20):
        d = {}
        for name, _ in self._fields_:
            v = getattr(self, name)
            if isinstance(v, ctypes.Array):
                # per-level arrays (21 entries) are cut to the levels used
                v = [v[i] for i in range(max_depth + 1 if len(v) == 21 else len(v))]
            d[name] = v
        return d


class Options(ctypes.Structure):
    _fields_ = [("min_edge", ctypes.c_double), ("precision_mode", ctypes.c_int), ("cutoff_rel", ctypes.c_double),
                ("cuda_stream", ctypes.c_void_p), ("device_output", ctypes.c_int), ("debug_flags", ctypes.c_int),
                ("stats", ctypes.POINTER(Stats)), ("child_mode", ctypes.c_int),
                ("decision_order", ctypes.c_int), ("precision_norm", ctypes.c_int), ("conform_mode", ctypes.c_int),
                ("batch_mode", ctypes.c_int)]


class MeshBuffers(ctypes.Structure):
    _fields_ = [("vertices", ctypes.c_void_p), ("triangles", ctypes.c_void_p), ("vertex_keys", ctypes.c_void_p),
                ("cube_keys", ctypes.c_void_p), ("cap_vertices", ctypes.c_int64), ("cap_triangles", ctypes.c_int64),
                ("cap_cubes", ctypes.c_int64), ("n_vertices", ctypes.c_int64), ("n_triangles", ctypes.c_int64),
                ("n_cubes", ctypes.c_int64)]


class MeshC(ctypes.Structure):
    _fields_ = [("vertices", ctypes.POINTER(ctypes.c_double)), ("n_vertices", ctypes.c_int64),
                ("triangles", ctypes.POINTER(ctypes.c_int32)), ("n_triangles", ctypes.c_int64),
                ("vertex_keys", ctypes.POINTER(ctypes.c_uint64)), ("cube_keys", ctypes.POINTER(ctypes.c_uint64)),
                ("n_cubes", ctypes.c_int64), ("on_device", ctypes.c_int), ("mismatches", ctypes.c_int64)]


_lib = None


def library_path():
    return LIB


def load():
    """Load libgsmesh.so; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB):
        raise GsError(-5, "CUDA library not built: %s (run paper_1611_03474_gb300.build.build())" % LIB)
    L = ctypes.CDLL(LIB)
    p, d, i64, i32 = ctypes.c_void_p, ctypes.c_double, ctypes.c_int64, ctypes.c_int
    L.mesh_gaussian_surface.argtypes = [p, p, i64, d, d, d, i32, ctypes.POINTER(Options), ctypes.POINTER(MeshC)]
    L.mesh_gaussian_surface.restype = i32
    L.mesh_gaussian_surface_into.argtypes = [p, p, i64, d, d, d, i32, ctypes.POINTER(Options),
                                             ctypes.POINTER(MeshBuffers)]
    L.mesh_gaussian_surface_into.restype = i32
    L.mesh_free.argtypes = [ctypes.POINTER(MeshC)]
    L.mesh_free.restype = None
    L.gs_status_string.argtypes = [i32]
    L.gs_status_string.restype = ctypes.c_char_p
    L.gs_last_error.restype = ctypes.c_char_p
    L.gs_default_options.restype = Options
    L.gs_bin_atoms.argtypes = [p, i64, d, p, p, p, p, p]
    L.gs_bin_atoms.restype = i32
    L.gs_eval_field.argtypes = [p, p, i64, d, d, d, p, i64, p, p, i32, p]
    L.gs_eval_field.restype = i32
    L.gs_eval_field_bounded.argtypes = [p, p, i64, d, d, d, p, i64, p, p, p]
    L.gs_eval_field_bounded.restype = i32
    L.gs_cube_decisions.argtypes = [p, p, i64, d, d, d, d, i32, d, p, i64, p, p, p, i32, p]
    L.gs_cube_decisions.restype = i32
    L.gs_triangulate_grid.argtypes = [i64, i64, i64, p, d, ctypes.POINTER(Options), ctypes.POINTER(MeshC)]
    L.gs_triangulate_grid.restype = i32
    L.gs_bin_atoms_static.argtypes = [p, i64, d, p, p, p, p, p]
    L.gs_bin_atoms_static.restype = i32
    L.gs_struct_size.argtypes = [i32]
    L.gs_struct_size.restype = i64
    L.gs_mesh_backward.argtypes = [p, p, i64, d, d, d, i32, ctypes.POINTER(Options), p, i64, p, p, p]
    L.gs_mesh_backward.restype = i32
    L.gs_volume_area.argtypes = [p, i64, p, i64, p, p, p, ctypes.POINTER(Options)]
    L.gs_volume_area.restype = i32
    L.mesh_gaussian_surface_batch.argtypes = [p, p, p, i64, p, d, d, i32, ctypes.POINTER(Options), i32, p, p]
    L.mesh_gaussian_surface_batch.restype = i32
    L.gs_mesh_intersections.argtypes = [p, i64, p, i64, d, p, ctypes.POINTER(Options)]
    L.gs_mesh_intersections.restype = i32
    L.gs_autotune_report.argtypes = [ctypes.c_char_p, i64]
    L.gs_autotune_report.restype = i64
    L.gs_autotune_reset.argtypes = []
    L.gs_autotune_reset.restype = None
    L.gs_memory_kind.argtypes = [p]
    L.gs_memory_kind.restype = i32
    for which, cls in ((0, Stats), (1, Options), (2, MeshC)):
        if L.gs_struct_size(which) != ctypes.sizeof(cls):
            raise GsError(-1, "ABI struct %s: library %d bytes, binding %d" % (cls.__name__, L.gs_struct_size(which),
                                                                            ctypes.sizeof(cls)))
    _lib = L
    return L


def _check(rc):
    if rc != 0:
        L = load()
        raise GsError(rc, "%s: %s" % (L.gs_status_string(rc).decode(), L.gs_last_error().decode()))


def _ptr(a):
    """Data pointer of a numpy array or torch tensor (contiguous required)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        assert a.is_contiguous(), "tensor must be contiguous"
        return ctypes.c_void_p(a.data_ptr())
    assert a.flags["C_CONTIGUOUS"], "array must be C-contiguous"
    return a.ctypes.data_as(ctypes.c_void_p)


def _host64(a, shape=None):
    if hasattr(a, "data_ptr"):
        return a
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a.reshape(shape) if shape is not None else a


def _stream_ptr(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


class Mesh:
    """Result of mesh_gaussian_surface: vertices [nv,3] f64, triangles [nt,3]
    i32 (CCW seen from outside), vertex_keys [nv] u64, cube_keys [nc] u64,
    stats dict.  Host numpy arrays unless device_output was requested."""

    def __init__(self, vertices, triangles, vertex_keys, cube_keys, stats, mismatches=0):
        self.vertices = vertices
        self.triangles = triangles
        self.vertex_keys = vertex_keys
        self.cube_keys = cube_keys
        self.stats = stats
        self.mismatches = mismatches


def _take_host(ptr, n, dtype, shape):
    if n == 0:
        return np.zeros(shape, dtype=dtype)
    arr = np.ctypeslib.as_array(ptr, shape=(int(np.prod(shape)),))
    return np.array(arr, dtype=dtype).reshape(shape)


def _mesh_from_c(m, L, stats, max_depth):
    try:
        res = Mesh(_take_host(m.vertices, m.n_vertices, np.float64, (m.n_vertices, 3)),
                   _take_host(m.triangles, m.n_triangles, np.int32, (m.n_triangles, 3)),
                   _take_host(m.vertex_keys, m.n_vertices, np.uint64, (m.n_vertices,)),
                   _take_host(m.cube_keys, m.n_cubes, np.uint64, (m.n_cubes,)),
                   stats.as_dict(max_depth), m.mismatches)
    finally:
        L.mesh_free(ctypes.byref(m))
    return res


GS_CHILD_REPROJECT, GS_CHILD_REEXPAND = 0, 1
GS_ORDER_BOUNDS_FIRST, GS_ORDER_LITERAL = 0, 1
GS_NORM_SUM, GS_NORM_MAX, GS_NORM_RSS = 0, 1, 2
GS_CONFORM_CONSTRAIN, GS_CONFORM_EQUAL = 0, 1
GS_BATCH_SHARED_LEVELS, GS_BATCH_THREADS = 0, 1


def mesh_gaussian_surface(atoms, radii, D, c, precision, max_depth, min_edge=0.25, precision_mode=GS_PREC_FP64,
                          cutoff_rel=1e-8, stream=None, debug_flags=0, device_output=False,
                          child_mode=GS_CHILD_REPROJECT, decision_order=GS_ORDER_BOUNDS_FIRST,
                          precision_norm=GS_NORM_SUM, conform_mode=GS_CONFORM_CONSTRAIN):
    """Mesh {phi = c}; see include/gsmesh.h.  With device_output the mesh
    stays in device memory and only its sizes and stats are returned (the
    arrays are released)."""
    L = load()
    atoms = _host64(atoms, (-1, 3))
    radii = _host64(radii)
    n = atoms.shape[0]
    st = Stats()
    o = L.gs_default_options()
    o.min_edge = min_edge
    o.precision_mode = precision_mode
    o.cutoff_rel = cutoff_rel
    o.cuda_stream = _stream_ptr(stream)
    o.device_output = 1 if device_output else 0
    o.debug_flags = debug_flags
    o.child_mode = child_mode
    o.decision_order = decision_order
    o.precision_norm = precision_norm
    o.conform_mode = conform_mode
    o.stats = ctypes.pointer(st)
    m = MeshC()
    rc = L.mesh_gaussian_surface(_ptr(atoms), _ptr(radii), n, D, c, precision, max_depth, ctypes.byref(o),
                                 ctypes.byref(m))
    _check(rc)
    if device_output:
        res = Mesh(None, None, None, None, st.as_dict(max_depth), m.mismatches)
        res.n_vertices, res.n_triangles, res.n_cubes = m.n_vertices, m.n_triangles, m.n_cubes
        L.mesh_free(ctypes.byref(m))
        return res
    return _mesh_from_c(m, L, st, max_depth)


class _DeviceArray:
    """A view of library-owned device memory for torch.as_tensor (the CUDA
    array interface); the caller copies it before the memory is released."""

    def __init__(self, ptr, shape, typestr):
        self.__cuda_array_interface__ = {"data": (int(ptr) if ptr else 0, False), "shape": tuple(shape),
                                         "typestr": typestr, "strides": None, "version": 3}


def mesh_gaussian_surface_device(atoms, radii, D, c, precision, max_depth, min_edge=0.25, precision_mode=GS_PREC_FP64,
                                 cutoff_rel=1e-8, stream=None, debug_flags=0, conform_mode=GS_CONFORM_CONSTRAIN):
    """Mesh {phi = c} with the result in device memory owned by torch:
    atoms [n,3] and radii [n] (float64 torch tensors, CUDA or host) in;
    returns (vertices [nv,3] float64, triangles [nt,3] int32, vertex_keys
    [nv] int64 (the uint64 keys' bits), cube_keys [nc] int64, stats) as
    tensors on the current CUDA device.  The mesh never visits the host: the
    library's device arrays are copied into torch's (device to device) and
    released."""
    import torch
    L = load()
    atoms = _host64(atoms, (-1, 3))
    radii = _host64(radii)
    n = atoms.shape[0]
    st = Stats()
    o = L.gs_default_options()
    o.min_edge = min_edge
    o.precision_mode = precision_mode
    o.cutoff_rel = cutoff_rel
    o.cuda_stream = _stream_ptr(stream)
    o.device_output = 1
    o.debug_flags = debug_flags
    o.conform_mode = conform_mode
    o.stats = ctypes.pointer(st)
    m = MeshC()
    _check(L.mesh_gaussian_surface(_ptr(atoms), _ptr(radii), n, D, c, precision, max_depth, ctypes.byref(o),
                                   ctypes.byref(m)))
    try:
        dev = torch.device("cuda", torch.cuda.current_device())

        def grab(ptr, shape, typestr, dtype):
            if int(np.prod(shape)) == 0:
                return torch.empty(shape, dtype=dtype, device=dev)
            addr = ctypes.cast(ptr, ctypes.c_void_p).value
            return torch.as_tensor(_DeviceArray(addr, shape, typestr), device=dev).clone()

        v = grab(m.vertices, (m.n_vertices, 3), "<f8", torch.float64)
        t = grab(m.triangles, (m.n_triangles, 3), "<i4", torch.int32)
        k = grab(m.vertex_keys, (m.n_vertices,), "<i8", torch.int64)
        ck = grab(m.cube_keys, (m.n_cubes,), "<i8", torch.int64)
        torch.cuda.synchronize(dev)
    finally:
        L.mesh_free(ctypes.byref(m))
    return v, t, k, ck, st.as_dict(max_depth)


def mesh_gaussian_surface_into(atoms, radii, D, c, precision, max_depth, vertices, triangles, vertex_keys=None,
                               cube_keys=None, min_edge=0.25, precision_mode=GS_PREC_FP64, cutoff_rel=1e-8,
                               stream=None, stats=False):
    """Mesh {phi = c} into caller-owned buffers (torch tensors on the host,
    pinned or not, or on the device, or numpy arrays): vertices float64
    [cap, 3], triangles int32 [cap, 3], vertex_keys / cube_keys uint64 (or
    int64) or None.  Returns (n_vertices, n_triangles, n_cubes), plus the
    stats dict when stats=True.  Buffers too small raise GsError with code
    GS_ERR_CAPACITY (-3) and the sizes needed in its .needed attribute."""
    L = load()
    atoms = _host64(atoms, (-1, 3))
    radii = _host64(radii)
    st = Stats()
    o = L.gs_default_options()
    o.min_edge = min_edge
    o.precision_mode = precision_mode
    o.cutoff_rel = cutoff_rel
    o.cuda_stream = _stream_ptr(stream)
    o.stats = ctypes.pointer(st)
    b = MeshBuffers()
    b.vertices, b.triangles = _ptr(vertices), _ptr(triangles)
    b.vertex_keys, b.cube_keys = _ptr(vertex_keys), _ptr(cube_keys)
    b.cap_vertices, b.cap_triangles = int(vertices.shape[0]), int(triangles.shape[0])
    b.cap_cubes = int(cube_keys.shape[0]) if cube_keys is not None else 0
    if vertex_keys is not None and int(vertex_keys.shape[0]) < b.cap_vertices:
        b.cap_vertices = int(vertex_keys.shape[0])
    rc = L.mesh_gaussian_surface_into(_ptr(atoms), _ptr(radii), atoms.shape[0], D, c, precision, max_depth,
                                      ctypes.byref(o), ctypes.byref(b))
    try:
        _check(rc)
    except GsError as e:
        e.needed = (b.n_vertices, b.n_triangles, b.n_cubes)
        raise
    sizes = (b.n_vertices, b.n_triangles, b.n_cubes)
    return (sizes + (st.as_dict(max_depth),)) if stats else sizes


def gs_triangulate_grid(values, c, stream=None):
    """Triangulate a uniform grid of corner values [nz+1, ny+1, nx+1]."""
    L = load()
    values = _host64(values)
    nz, ny, nx = (int(d) - 1 for d in values.shape)
    st = Stats()
    o = L.gs_default_options()
    o.cuda_stream = _stream_ptr(stream)
    o.stats = ctypes.pointer(st)
    m = MeshC()
    _check(L.gs_triangulate_grid(nx, ny, nz, _ptr(values), c, ctypes.byref(o), ctypes.byref(m)))
    return _mesh_from_c(m, L, st, 0)


def gs_eval_field(atoms, radii, D, c, points, cutoff_rel=1e-8, grad=False, precision_mode=GS_PREC_FP64, stream=None,
                  out=None):
    """phi (and grad phi) at points [n,3]; returns numpy arrays unless `out`
    (a tuple of preallocated arrays/tensors) is given."""
    L = load()
    atoms = _host64(atoms, (-1, 3))
    radii = _host64(radii)
    points = _host64(points, (-1, 3))
    n = points.shape[0]
    if out is None:
        phi = np.zeros(n)
        g = np.zeros((n, 3)) if grad else None
    else:
        phi, g = out
    _check(L.gs_eval_field(_ptr(atoms), _ptr(radii), atoms.shape[0], D, c, cutoff_rel, _ptr(points), n, _ptr(phi),
                           _ptr(g), precision_mode, _stream_ptr(stream)))
    return (phi, g) if grad else phi


def gs_eval_field_bounded(atoms, radii, D, c, points, cutoff_rel=1e-8, stream=None):
    """(phi [n] FP64, err [n] FP32) at points [n,3]: the double-word FP32
    evaluation with its bound on |phi - phi_exact|."""
    L = load()
    atoms = _host64(atoms, (-1, 3))
    radii = _host64(radii)
    points = _host64(points, (-1, 3))
    n = points.shape[0]
    phi = np.zeros(n)
    err = np.zeros(n, dtype=np.float32)
    _check(L.gs_eval_field_bounded(_ptr(atoms), _ptr(radii), atoms.shape[0], D, c, cutoff_rel, _ptr(points), n,
                                   _ptr(phi), _ptr(err), _stream_ptr(stream)))
    return phi, err


def gs_cube_decisions(atoms, radii, D, c, precision, min_edge, max_depth, cube_keys, cutoff_rel=1e-8,
                      precision_mode=GS_PREC_FP64, stream=None):
    """(A [n,64], bounds [n,6], dec [n]) for listed cube keys."""
    L = load()
    atoms = _host64(atoms, (-1, 3))
    radii = _host64(radii)
    keys = np.ascontiguousarray(cube_keys, dtype=np.uint64)
    n = len(keys)
    A, b, d = np.zeros((n, 64)), np.zeros((n, 6)), np.zeros(n, dtype=np.int32)
    _check(L.gs_cube_decisions(_ptr(atoms), _ptr(radii), atoms.shape[0], D, c, precision, min_edge, max_depth,
                               cutoff_rel, _ptr(keys), n, _ptr(A), _ptr(b), _ptr(d), precision_mode,
                               _stream_ptr(stream)))
    return A, b, d


def gs_bin_atoms(atoms, cell_size, origin, dims, stream=None):
    """(cell_start [ncell+1] i32, atom_perm [n] i32) of the stable counting sort."""
    L = load()
    atoms = _host64(atoms, (-1, 3))
    origin = np.ascontiguousarray(origin, dtype=np.float64)
    dims = np.ascontiguousarray(dims, dtype=np.int64)
    ncell = int(np.prod(dims))
    cs = np.zeros(ncell + 1, dtype=np.int32)
    pm = np.zeros(atoms.shape[0], dtype=np.int32)
    _check(L.gs_bin_atoms(_ptr(atoms), atoms.shape[0], cell_size, _ptr(origin), _ptr(dims), _ptr(cs), _ptr(pm),
                          _stream_ptr(stream)))
    return cs, pm


def _require_device_tensor(name, t, dtype, min_numel, device):
    """t must be a contiguous torch tensor of dtype on `device` with at least
    min_numel elements (checked before the call: nothing reaches the GPU)."""
    import torch
    if not isinstance(t, torch.Tensor):
        raise GsError(-1, "%s must be a torch tensor in device memory" % name)
    if t.dtype != dtype:
        raise GsError(-1, "%s must be %s, not %s" % (name, dtype, t.dtype))
    if t.device.type != "cuda" or t.device.index != device:
        raise GsError(-1, "%s must be on cuda:%d (the current device), not %s" % (name, device, t.device))
    if not t.is_contiguous():
        raise GsError(-1, "%s must be contiguous" % name)
    if t.numel() < min_numel:
        raise GsError(-1, "%s has %d elements, needs at least %d" % (name, t.numel(), min_numel))


def gs_bin_atoms_static(atoms, cell_size, origin, dims, cell_start, atom_perm, stream=None):
    """Allocation-free cell list into caller-provided device buffers (torch
    CUDA tensors on the current device: atoms float64 [n,3], cell_start int32
    with at least prod(dims)+1 elements, atom_perm int32 with at least n);
    see include/gsmesh.h for the limits and the sharing rules.  Wrong types,
    shapes, sizes or devices raise GsError before any GPU work."""
    import torch
    L = load()
    origin = np.ascontiguousarray(origin, dtype=np.float64)
    dims = np.ascontiguousarray(dims, dtype=np.int64)
    if origin.shape != (3,) or dims.shape != (3,):
        raise GsError(-1, "origin and dims must have 3 entries")
    dev = torch.cuda.current_device()
    if not isinstance(atoms, torch.Tensor) or atoms.dim() != 2 or atoms.shape[1] != 3:
        raise GsError(-1, "atoms must be a torch tensor of shape [n, 3]")
    _require_device_tensor("atoms", atoms, torch.float64, 3 * atoms.shape[0], dev)
    ncell = int(np.prod(dims)) if np.all(dims > 0) else 0
    _require_device_tensor("cell_start", cell_start, torch.int32, ncell + 1, dev)
    _require_device_tensor("atom_perm", atom_perm, torch.int32, atoms.shape[0], dev)
    _check(L.gs_bin_atoms_static(_ptr(atoms), int(atoms.shape[0]), cell_size, _ptr(origin), _ptr(dims),
                                 _ptr(cell_start), _ptr(atom_perm), _stream_ptr(stream)))


def gs_mesh_backward(atoms, radii, D, c, precision, max_depth, grad_vertices, min_edge=0.25,
                     precision_mode=GS_PREC_FP64, cutoff_rel=1e-8, stream=None):
    """dL/d(atoms [n,3], radii [n], D) from dL/d(vertices) [nv,3] of the mesh
    mesh_gaussian_surface returns for the same arguments (numpy arrays)."""
    L = load()
    atoms = _host64(atoms, (-1, 3))
    radii = _host64(radii)
    gv = _host64(grad_vertices, (-1, 3))
    n = atoms.shape[0]
    if hasattr(atoms, "is_cuda") and atoms.is_cuda:
        # device tensors in, device tensors out (no host round trip)
        import torch
        ga = torch.zeros((n, 3), dtype=torch.float64, device=atoms.device)
        gr = torch.zeros(n, dtype=torch.float64, device=atoms.device)
        gD = torch.zeros(1, dtype=torch.float64, device=atoms.device)
    else:
        ga, gr, gD = np.zeros((n, 3)), np.zeros(n), np.zeros(1)
    o = L.gs_default_options()
    o.min_edge = min_edge
    o.precision_mode = precision_mode
    o.cutoff_rel = cutoff_rel
    o.cuda_stream = _stream_ptr(stream)
    _check(L.gs_mesh_backward(_ptr(atoms), _ptr(radii), n, D, c, precision, max_depth, ctypes.byref(o), _ptr(gv),
                              gv.shape[0], _ptr(ga), _ptr(gr), _ptr(gD)))
    if not isinstance(ga, np.ndarray):
        return ga, gr, gD[0]
    return ga, gr, float(gD[0])


def gs_volume_area(vertices, triangles, grad=False, stream=None):
    """(volume, area) of a closed outward mesh, and with grad=True their
    gradients per vertex ([nv,3] each)."""
    L = load()
    v = _host64(vertices, (-1, 3))
    t = triangles if hasattr(triangles, "data_ptr") else np.ascontiguousarray(triangles, dtype=np.int32)
    nv, nt = v.shape[0], t.shape[0]
    if hasattr(v, "is_cuda") and v.is_cuda:
        # device tensors in, device tensors out
        import torch
        va = torch.zeros(2, dtype=torch.float64, device=v.device)
        gV = torch.zeros((nv, 3), dtype=torch.float64, device=v.device) if grad else None
        gA = torch.zeros((nv, 3), dtype=torch.float64, device=v.device) if grad else None
    else:
        va = np.zeros(2)
        gV = np.zeros((nv, 3)) if grad else None
        gA = np.zeros((nv, 3)) if grad else None
    o = L.gs_default_options()
    o.cuda_stream = _stream_ptr(stream)
    _check(L.gs_volume_area(_ptr(v), nv, _ptr(t), nt, _ptr(va), _ptr(gV), _ptr(gA), ctypes.byref(o)))
    return (va[0], va[1], gV, gA) if grad else (va[0], va[1])


def mesh_gaussian_surface_batch(molecules, c, precision, max_depth, min_edge=0.25, precision_mode=GS_PREC_FP64,
                                cutoff_rel=1e-8, n_workers=8, device_output=False,
                                batch_mode=GS_BATCH_SHARED_LEVELS, debug_flags=0):
    """Mesh several molecules: molecules is a list of (atoms [n,3], radii
    [n], D).  batch_mode GS_BATCH_SHARED_LEVELS runs one level loop per
    group of equal D over all the group's molecules, GS_BATCH_THREADS whole
    meshes on n_workers host threads.  Returns a list of Mesh (host arrays
    unless device_output, as in mesh_gaussian_surface)."""
    L = load()
    xs = [np.ascontiguousarray(m[0], dtype=np.float64).reshape(-1, 3) for m in molecules]
    rs = [np.ascontiguousarray(m[1], dtype=np.float64).reshape(-1) for m in molecules]
    Ds = np.ascontiguousarray([float(m[2]) for m in molecules], dtype=np.float64)
    offsets = np.zeros(len(molecules) + 1, dtype=np.int64)
    offsets[1:] = np.cumsum([len(r) for r in rs])
    atoms = np.ascontiguousarray(np.concatenate(xs))
    radii = np.ascontiguousarray(np.concatenate(rs))
    nm = len(molecules)
    outs = (MeshC * nm)()
    stats = (Stats * nm)()
    o = L.gs_default_options()
    o.min_edge = min_edge
    o.precision_mode = precision_mode
    o.cutoff_rel = cutoff_rel
    o.device_output = 1 if device_output else 0
    o.batch_mode = batch_mode
    o.debug_flags = debug_flags
    _check(L.mesh_gaussian_surface_batch(_ptr(atoms), _ptr(radii), _ptr(offsets), nm, _ptr(Ds), c, precision,
                                         max_depth, ctypes.byref(o), n_workers, ctypes.cast(outs, ctypes.c_void_p),
                                         ctypes.cast(stats, ctypes.c_void_p)))
    res = []
    for m in range(nm):
        if device_output:
            r = Mesh(None, None, None, None, stats[m].as_dict(max_depth), outs[m].mismatches)
            r.n_vertices, r.n_triangles, r.n_cubes = outs[m].n_vertices, outs[m].n_triangles, outs[m].n_cubes
            L.mesh_free(ctypes.byref(outs[m]))
            res.append(r)
        else:
            res.append(_mesh_from_c(outs[m], L, stats[m], max_depth))
    return res


def autotune_report():
    """The autotuner's choices: a list of dicts (kernel, size_class (log2 of
    the item count), choice, trial_ms per shape)."""
    L = load()
    need = L.gs_autotune_report(None, 0)
    buf = ctypes.create_string_buffer(int(need))
    L.gs_autotune_report(buf, need)
    out = []
    for line in buf.value.decode().splitlines():
        f = line.split()
        out.append({"kernel": f[0], "size_class": int(f[1][2:]), "choice": int(f[2]),
                    "trial_ms": [float(x) for x in f[3:]]})
    return out


def memory_kind(buf):
    """How the library sees a buffer (numpy array or torch tensor): 0 device,
    1 page-locked host memory mapped into the device, 2 other host memory."""
    return int(load().gs_memory_kind(_ptr(buf)))


def autotune_reset():
    """Forget every autotuner choice."""
    load().gs_autotune_reset()


def gs_mesh_intersections(vertices, triangles, tol=1e-9, stream=None):
    """Number of vertex-disjoint triangle pairs that overlap by more than tol."""
    L = load()
    v = _host64(vertices, (-1, 3))
    t = triangles if hasattr(triangles, "data_ptr") else np.ascontiguousarray(triangles, dtype=np.int32)
    n = ctypes.c_int64(0)
    o = L.gs_default_options()
    o.cuda_stream = _stream_ptr(stream)
    _check(L.gs_mesh_intersections(_ptr(v), v.shape[0], _ptr(t), t.shape[0], tol, ctypes.byref(n), ctypes.byref(o)))
    return int(n.value)
