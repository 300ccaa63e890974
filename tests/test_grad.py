"""Differentiation of the mesh (vertex positions, enclosed volume and surface
area with respect to atom centres, radii and D), cube set and topology held
fixed.  CPU tests pin the oracle's gradient and the loss helpers; GPU tests
compare the adjoint kernels with the oracle and with central differences."""
import numpy as np
import pytest

import oracle
import synth
from meshcheck import key_normal_weights, surface_loss, surface_loss_grad

ARGS = dict(c=1.0, precision=1e-3, min_edge=0.25, max_depth=3)


def _omesh(xyz, r, D):
    return oracle.mesh(xyz, r, D, ARGS["c"], ARGS["precision"], ARGS["min_edge"], ARGS["max_depth"])


def _same(a, b):
    return (np.array_equal(a["vkeys"], b["vkeys"]) and np.array_equal(a["triangles"], b["triangles"])
            and np.array_equal(a["cube_keys"], b["cube_keys"]))


def _oloss(m):
    return surface_loss(m["vertices"], m["triangles"], key_normal_weights(m["vkeys"]))


def test_loss_gradient_helper_matches_differences():
    """surface_loss_grad against central differences of surface_loss in the
    vertex positions of a real mesh (pins the helper both sides use)."""
    m = _omesh(np.array([[0.31, 0.12, -0.23]]), np.array([1.5]), 0.5)
    v, t = m["vertices"], m["triangles"]
    W = key_normal_weights(m["vkeys"])
    g = surface_loss_grad(v, t, W)
    rng = np.random.default_rng(3)
    for i in rng.integers(0, len(v), 12):
        for q in range(3):
            vp, vm = v.copy(), v.copy()
            vp[i, q] += 1e-6
            vm[i, q] -= 1e-6
            fd = (surface_loss(vp, t, W) - surface_loss(vm, t, W)) / 2e-6
            assert abs(fd - g[i, q]) <= 1e-6 * max(1.0, abs(g[i, q]))


def test_volume_area_of_one_atom():
    """One atom: the surface is the sphere of radius sqrt(r^2 - ln(c)/D); the
    mesh's volume and area approach 4/3 pi R^3 and 4 pi R^2 (inscribed
    polyhedron: slightly below, within the 0.25 A cube size)."""
    r0, D, c = 1.5, 0.5, 1.0
    m = _omesh(np.array([[0.3, 0.1, -0.2]]), np.array([r0]), D)
    R = np.sqrt(r0 * r0 - np.log(c) / D)
    vol, area = oracle.volume_area(m["vertices"], m["triangles"])
    assert 0.97 * 4 / 3 * np.pi * R ** 3 < vol < 4 / 3 * np.pi * R ** 3
    assert 0.97 * 4 * np.pi * R ** 2 < area < 4 * np.pi * R ** 2


def test_oracle_gradient_matches_differences():
    """The oracle's chain-rule gradient against central differences of the
    oracle's own loss (step 1e-6; components whose +-h meshes change cubes or
    topology are skipped)."""
    xyz = np.array([[0.31, 0.12, -0.23], [1.9, 0.4, 0.3]])
    r = np.array([1.5, 1.2])
    D = 0.5
    m = _omesh(xyz, r, D)
    gx, gr, gD = oracle.mesh_grad(xyz, r, D, ARGS["c"], ARGS["precision"], ARGS["min_edge"], ARGS["max_depth"],
                                  surface_loss_grad(m["vertices"], m["triangles"], key_normal_weights(m["vkeys"])))
    h = 1e-6
    checked = 0
    cases = [("x", i, q) for i in range(2) for q in range(3)] + [("r", i, 0) for i in range(2)] + [("D", 0, 0)]
    for kind, i, q in cases:
        xp, xm, rp, rm, Dp, Dm = xyz.copy(), xyz.copy(), r.copy(), r.copy(), D, D
        if kind == "x":
            xp[i, q] += h; xm[i, q] -= h; ref = gx[i, q]
        elif kind == "r":
            rp[i] += h; rm[i] -= h; ref = gr[i]
        else:
            Dp, Dm, ref = D + h, D - h, gD
        mp, mm = _omesh(xp, rp, Dp), _omesh(xm, rm, Dm)
        if not (_same(mp, m) and _same(mm, m)):
            continue
        fd = (_oloss(mp) - _oloss(mm)) / (2 * h)
        assert abs(fd - ref) <= 2e-6 * max(1.0, abs(ref)), (kind, i, q, fd, ref)
        checked += 1
    assert checked >= 7


# ---------------------------------------------------------------- GPU
@pytest.fixture(scope="module")
def gs():
    import paper_1611_03474_gb300 as g
    return g


def _gpu_loss_grad(gs, xyz, r, D, mode):
    m = gs.mesh_gaussian_surface(xyz, r, D, ARGS["c"], ARGS["precision"], ARGS["max_depth"],
                                 min_edge=ARGS["min_edge"], precision_mode=mode)
    W = key_normal_weights(m.vertex_keys)
    return m, surface_loss(m.vertices, m.triangles, W), surface_loss_grad(m.vertices, m.triangles, W)


@pytest.mark.gpu
@pytest.mark.parametrize("mode", ["fp64", "mixed"])
def test_gpu_gradient_matches_oracle(gs, mode):
    """gs_mesh_backward (adjoint kernels) against the oracle's gradient of the
    same loss on the 100-atom chain; the loss gradient per vertex is mapped by
    vertex key, so vertex order does not matter."""
    cfg = synth.config("chain100")
    xyz, r, D = cfg["xyz"], cfg["r"], cfg["D"]
    prec = gs.GS_PREC_FP64 if mode == "fp64" else gs.GS_PREC_MIXED
    m, _, g = _gpu_loss_grad(gs, xyz, r, D, prec)
    ga, gr, gD = gs.gs_mesh_backward(xyz, r, D, ARGS["c"], ARGS["precision"], ARGS["max_depth"], g,
                                     min_edge=ARGS["min_edge"], precision_mode=prec)
    om = _omesh(xyz, r, D)
    assert np.array_equal(np.sort(m.vertex_keys), om["vkeys"])
    og = surface_loss_grad(om["vertices"], om["triangles"], key_normal_weights(om["vkeys"]))
    ox, orr, oD = oracle.mesh_grad(xyz, r, D, ARGS["c"], ARGS["precision"], ARGS["min_edge"], ARGS["max_depth"], og)
    scale = max(np.abs(ox).max(), np.abs(orr).max(), abs(oD))
    tol = 1e-9 if mode == "fp64" else 1e-5
    assert np.abs(ga - ox).max() <= tol * scale
    assert np.abs(gr - orr).max() <= tol * scale
    assert abs(gD - oD) <= tol * max(1.0, abs(oD))


@pytest.mark.gpu
def test_gpu_gradient_matches_differences(gs):
    """Central differences (h = 1e-4 A, FP64 meshes) of the loss on a 300-atom
    globular molecule for a sample of centres and radii and for D, relative
    tolerance 1e-4.  Near-degenerate vertices (an edge root or fold root with
    a small denominator) give the central difference an O(h^2) error of that
    order, so the compared value is its Richardson extrapolation from h and
    h/2; components whose meshes change cubes or topology are skipped."""
    xyz, r = synth.globular(300, seed=4)
    D = 0.5
    prec = gs.GS_PREC_FP64
    m, L0, g = _gpu_loss_grad(gs, xyz, r, D, prec)
    ga, gr, gD = gs.gs_mesh_backward(xyz, r, D, ARGS["c"], ARGS["precision"], ARGS["max_depth"], g,
                                     min_edge=ARGS["min_edge"], precision_mode=prec)

    def L_of(x, rr, DD):
        mm, L, _ = _gpu_loss_grad(gs, x, rr, DD, prec)
        same = (np.array_equal(mm.vertex_keys, m.vertex_keys) and np.array_equal(mm.triangles, m.triangles)
                and np.array_equal(mm.cube_keys, m.cube_keys))
        return L, same

    rng = np.random.default_rng(11)
    h = 1e-4
    checked = 0
    scale = max(np.abs(ga).max(), np.abs(gr).max())
    for i in rng.choice(len(r), 12, replace=False):
        for kind in ("x", "r"):
            q = int(rng.integers(0, 3))
            ref = ga[i, q] if kind == "x" else gr[i]
            fds, ok = [], True
            for hh in (h, h / 2):
                xp, xm, rp, rm = xyz.copy(), xyz.copy(), r.copy(), r.copy()
                if kind == "x":
                    xp[i, q] += hh; xm[i, q] -= hh
                else:
                    rp[i] += hh; rm[i] -= hh
                Lp, sp = L_of(xp, rp, D)
                Lm, sm = L_of(xm, rm, D)
                ok = ok and sp and sm
                fds.append((Lp - Lm) / (2 * hh))
            if not ok:
                continue
            fd = (4.0 * fds[1] - fds[0]) / 3.0
            assert abs(fd - ref) <= 1e-4 * max(abs(ref), 1e-3 * scale), (kind, i, fds, ref)
            checked += 1
    Lp, sp = L_of(xyz, r, D + 1e-6)
    Lm, sm = L_of(xyz, r, D - 1e-6)
    if sp and sm:
        fd = (Lp - Lm) / 2e-6
        assert abs(fd - gD) <= 1e-4 * abs(gD)
        checked += 1
    assert checked >= 12


@pytest.mark.gpu
def test_gpu_volume_area_matches_oracle(gs):
    cfg = synth.config("chain100")
    m = gs.mesh_gaussian_surface(cfg["xyz"], cfg["r"], cfg["D"], ARGS["c"], ARGS["precision"], ARGS["max_depth"],
                                 min_edge=ARGS["min_edge"])
    vol, area, gV, gA = gs.gs_volume_area(m.vertices, m.triangles, grad=True)
    ov, oa = oracle.volume_area(m.vertices, m.triangles)
    assert abs(vol - ov) <= 1e-12 * abs(ov) and abs(area - oa) <= 1e-12 * oa
    W0 = np.zeros_like(m.vertices)
    g = surface_loss_grad(m.vertices, m.triangles, W0)
    assert np.abs(gV + gA - g).max() <= 1e-12 * np.abs(g).max()


@pytest.mark.gpu
def test_autograd_function(gs):
    """The torch.autograd wrappers give the same gradient as the direct calls."""
    torch = pytest.importorskip("torch")
    from paper_1611_03474_gb300.autograd import gaussian_surface, volume_area
    cfg = synth.config("chain100")
    x = torch.tensor(cfg["xyz"], dtype=torch.float64, requires_grad=True)
    r = torch.tensor(cfg["r"], dtype=torch.float64, requires_grad=True)
    D = torch.tensor(cfg["D"], dtype=torch.float64, requires_grad=True)
    v, t = gaussian_surface(x, r, D, **ARGS)
    m = gs.mesh_gaussian_surface(cfg["xyz"], cfg["r"], cfg["D"], ARGS["c"], ARGS["precision"], ARGS["max_depth"],
                                 min_edge=ARGS["min_edge"])
    W = torch.from_numpy(key_normal_weights(m.vertex_keys))
    vol, area = volume_area(v, t)
    L = (W * v).sum() + vol + area
    L.backward()
    g = surface_loss_grad(m.vertices, m.triangles, W.numpy())
    ga, gr, gD = gs.gs_mesh_backward(cfg["xyz"], cfg["r"], cfg["D"], ARGS["c"], ARGS["precision"], ARGS["max_depth"],
                                     g, min_edge=ARGS["min_edge"])
    scale = np.abs(ga).max()
    assert np.abs(x.grad.numpy() - ga).max() <= 1e-10 * scale
    assert np.abs(r.grad.numpy() - gr).max() <= 1e-10 * scale
    assert abs(D.grad.item() - gD) <= 1e-10 * max(1.0, abs(gD))


def _sat_pairs(v, t, tol=1e-9):
    """Brute-force count of vertex-disjoint intersecting triangle pairs
    (separating-axis test on the 11 axes, coplanar pairs in their plane)."""
    P = v[t]
    n = len(t)
    count = 0
    for i in range(n):
        for j in range(i + 1, n):
            if set(t[i]) & set(t[j]):
                continue
            A, B = P[i], P[j]
            if np.any(A.max(0) < B.min(0) - tol) or np.any(B.max(0) < A.min(0) - tol):
                continue
            eA, eB = np.roll(A, -1, 0) - A, np.roll(B, -1, 0) - B
            nA = np.cross(eA[0], eA[1])
            axes = [nA, np.cross(eB[0], eB[1])] + [np.cross(a, b) for a in eA for b in eB]
            lA = np.linalg.norm(nA)
            if lA > 0 and np.all(np.abs((B - A[0]) @ nA) / lA <= tol):
                axes = [np.cross(e, nA) for e in list(eA) + list(eB)]
            sep = False
            for ax in axes:
                l = np.linalg.norm(ax)
                if l <= 1e-15:
                    continue
                ax = ax / l
                a, b = A @ ax, B @ ax
                if a.max() <= b.min() + tol or b.max() <= a.min() + tol:
                    sep = True
                    break
            if not sep:
                count += 1
    return count


@pytest.mark.gpu
def test_gpu_intersections(gs):
    """The chain mesh has no intersecting triangle pairs; two single-atom
    meshes pushed into each other have as many as a brute-force check finds."""
    cfg = synth.config("chain100")
    m = gs.mesh_gaussian_surface(cfg["xyz"], cfg["r"], cfg["D"], ARGS["c"], ARGS["precision"], ARGS["max_depth"],
                                 min_edge=1.0)
    assert gs.gs_mesh_intersections(m.vertices, m.triangles) == 0
    a = gs.mesh_gaussian_surface(np.zeros((1, 3)), np.array([1.3]), 0.5, 1.0, 1e-3, 2, min_edge=0.5)
    b = gs.mesh_gaussian_surface(np.array([[1.7, 0.3, 0.1]]), np.array([1.2]), 0.5, 1.0, 1e-3, 2, min_edge=0.5)
    v = np.vstack([a.vertices, b.vertices])
    t = np.vstack([a.triangles, b.triangles + len(a.vertices)]).astype(np.int32)
    n_gpu = gs.gs_mesh_intersections(v, t)
    assert n_gpu > 0
    assert n_gpu == _sat_pairs(v, t)


@pytest.mark.gpu
def test_autograd_on_device_matches_host_path(gs):
    """CUDA tensors go through the library by pointer (mesh, volume/area and
    adjoint on the device); the gradient equals the host path's."""
    torch = pytest.importorskip("torch")
    from paper_1611_03474_gb300.autograd import gaussian_surface, volume_area
    cfg = synth.config("chain100")
    grads = []
    for dev in ("cpu", "cuda"):
        x = torch.tensor(cfg["xyz"], dtype=torch.float64, device=dev, requires_grad=True)
        r = torch.tensor(cfg["r"], dtype=torch.float64, device=dev, requires_grad=True)
        D = torch.tensor(cfg["D"], dtype=torch.float64, device=dev, requires_grad=True)
        v, t = gaussian_surface(x, r, D, **ARGS)
        assert v.device.type == dev and t.device.type == dev
        vol, area = volume_area(v, t)
        (vol + area + (v * 0.01).sum()).backward()
        grads.append([g.detach().cpu().numpy() for g in (x.grad, r.grad, D.grad)])
    for a, b in zip(*grads):
        assert np.abs(a - b).max() <= 1e-9 * max(1.0, np.abs(a).max())


@pytest.mark.gpu
@pytest.mark.parametrize("mode", ["fp64", "mixed"])
def test_gradient_matches_differences_globular10k(gs, mode):
    """The differentiation form's workload (10,000-atom globular molecule):
    the adjoint's dL/d(centres), dL/d(radii) and dL/dD for L = volume + area
    + sum w.p (w ~ N(0,1) per vertex, seeded), in both precision forms,
    against central differences of the FP64 form's L (h = 1e-4 A and h/2,
    Richardson-extrapolated) on a sample of components; relative tolerance
    1e-4.  Components whose +-h meshes change cubes or topology are skipped."""
    cfg = synth.config("globular10k")
    xyz, r, D = cfg["xyz"], cfg["r"], cfg["D"]
    rng = np.random.default_rng(0)
    m = gs.mesh_gaussian_surface(xyz, r, D, ARGS["c"], ARGS["precision"], ARGS["max_depth"], min_edge=ARGS["min_edge"])
    key_w = dict(zip(m.vertex_keys.tolist(), rng.standard_normal((len(m.vertex_keys), 3))))

    def loss(mm):
        W = np.array([key_w.get(k, np.zeros(3)) for k in mm.vertex_keys.tolist()])
        vol, area = gs.gs_volume_area(mm.vertices, mm.triangles)
        return vol + area + float((W * mm.vertices).sum()), W

    prec = gs.GS_PREC_FP64 if mode == "fp64" else gs.GS_PREC_MIXED
    mp = gs.mesh_gaussian_surface(xyz, r, D, ARGS["c"], ARGS["precision"], ARGS["max_depth"], min_edge=ARGS["min_edge"],
                                  precision_mode=prec)
    _, W = loss(mp)
    vol, area, gV, gA = gs.gs_volume_area(mp.vertices, mp.triangles, grad=True)
    ga, gr, gD = gs.gs_mesh_backward(xyz, r, D, ARGS["c"], ARGS["precision"], ARGS["max_depth"], gV + gA + W,
                                     min_edge=ARGS["min_edge"], precision_mode=prec)

    def L_of(x, rr, DD):
        mm = gs.mesh_gaussian_surface(x, rr, DD, ARGS["c"], ARGS["precision"], ARGS["max_depth"],
                                      min_edge=ARGS["min_edge"])
        same = (np.array_equal(mm.vertex_keys, m.vertex_keys) and np.array_equal(mm.triangles, m.triangles)
                and np.array_equal(mm.cube_keys, m.cube_keys))
        return loss(mm)[0], same

    h = 1e-4
    scale = max(np.abs(ga).max(), np.abs(gr).max())
    checked = 0
    # atoms near the surface (their derivatives are not zero)
    near = np.argsort(-np.abs(ga).sum(1))[:200]
    for i in rng.choice(near, 8, replace=False):
        for kind in ("x", "r"):
            q = int(rng.integers(0, 3))
            ref = ga[i, q] if kind == "x" else gr[i]
            fds, ok = [], True
            for hh in (h, h / 2):
                xp, xm, rp, rm = xyz.copy(), xyz.copy(), r.copy(), r.copy()
                if kind == "x":
                    xp[i, q] += hh; xm[i, q] -= hh
                else:
                    rp[i] += hh; rm[i] -= hh
                Lp, sp = L_of(xp, rp, D)
                Lm, sm = L_of(xm, rm, D)
                ok = ok and sp and sm
                fds.append((Lp - Lm) / (2 * hh))
            if not ok:
                continue
            fd = (4.0 * fds[1] - fds[0]) / 3.0
            assert abs(fd - ref) <= 1e-4 * max(abs(ref), 1e-3 * scale), (kind, i, fds, ref)
            checked += 1
    Lp, sp = L_of(xyz, r, D + 1e-6)
    Lm, sm = L_of(xyz, r, D - 1e-6)
    if sp and sm:
        fd = (Lp - Lm) / 2e-6
        assert abs(fd - gD) <= 1e-4 * abs(gD)
        checked += 1
    assert checked >= 10
