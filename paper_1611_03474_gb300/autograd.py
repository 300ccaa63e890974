"""torch.autograd wrappers of the mesher: vertex positions as a function of
atom centres, radii and D (backward through gs_mesh_backward, the adjoint
kernels), and the enclosed volume and surface area as functions of the
vertex positions (gs_volume_area).  The cube set and the topology are held
fixed in the derivative.  Marshalling only: every value and derivative comes
from the CUDA library, and CUDA tensors are passed by pointer (no host round
trip).
"""
import numpy as np
import torch

from . import _native as nat


def _np(t):
    return t.detach().to("cpu", torch.float64).contiguous().numpy()


def _dev(t):
    """float64, contiguous, on the tensor's own CUDA device (no host copy);
    the library is called on torch's current stream, so it sees this work"""
    return t.detach().to(torch.float64).contiguous()


class GaussianSurface(torch.autograd.Function):
    """(vertices [nv,3] f64, triangles [nt,3] i64) of {phi = c}; differentiable
    in atoms [n,3], radii [n] and D (a 0-d tensor).  CUDA inputs stay on the
    device throughout: the library reads them by pointer, the mesh comes back
    as device tensors and the adjoint writes its gradients into device
    tensors.  Host inputs take the host path."""

    @staticmethod
    def forward(ctx, atoms, radii, D, c, precision, max_depth, min_edge, precision_mode):
        ctx.save_for_backward(atoms, radii, D)
        ctx.args = (c, precision, max_depth, min_edge, precision_mode)
        if atoms.is_cuda:
            v, t, _, _, _ = nat.mesh_gaussian_surface_device(_dev(atoms), _dev(radii), float(D), c, precision,
                                                             max_depth, min_edge=min_edge,
                                                             precision_mode=precision_mode,
                                                             stream=torch.cuda.current_stream(atoms.device))
            t = t.to(torch.int64)
        else:
            m = nat.mesh_gaussian_surface(_np(atoms), _np(radii), float(D), c, precision, max_depth,
                                          min_edge=min_edge, precision_mode=precision_mode)
            v = torch.from_numpy(m.vertices)
            t = torch.from_numpy(m.triangles.astype(np.int64))
        ctx.mark_non_differentiable(t)
        return v, t

    @staticmethod
    def backward(ctx, gv, gt):
        atoms, radii, D = ctx.saved_tensors
        c, precision, max_depth, min_edge, mode = ctx.args
        if atoms.is_cuda:
            ga, gr, gD = nat.gs_mesh_backward(_dev(atoms), _dev(radii), float(D), c, precision, max_depth, _dev(gv),
                                              min_edge=min_edge, precision_mode=mode,
                                              stream=torch.cuda.current_stream(atoms.device))
            return (ga.to(atoms.dtype), gr.to(radii.dtype), gD.to(D.dtype).reshape(D.shape).to(D.device),
                    None, None, None, None, None)
        ga, gr, gD = nat.gs_mesh_backward(_np(atoms), _np(radii), float(D), c, precision, max_depth, _np(gv),
                                          min_edge=min_edge, precision_mode=mode)
        return (torch.from_numpy(ga).to(atoms), torch.from_numpy(gr).to(radii),
                torch.tensor(gD, dtype=D.dtype, device=D.device), None, None, None, None, None)


class VolumeArea(torch.autograd.Function):
    """(volume, area) of a closed outward mesh; differentiable in the vertices
    (device tensors stay on the device)."""

    @staticmethod
    def forward(ctx, vertices, triangles):
        if vertices.is_cuda:
            t = triangles.detach().to(torch.int32).contiguous()
            vol, area, gV, gA = nat.gs_volume_area(_dev(vertices), t, grad=True,
                                                   stream=torch.cuda.current_stream(vertices.device))
            ctx.save_for_backward(gV.to(vertices.dtype), gA.to(vertices.dtype))
            return vol.to(vertices.dtype), area.to(vertices.dtype)
        t = triangles.detach().to("cpu", torch.int32).contiguous().numpy()
        vol, area, gV, gA = nat.gs_volume_area(_np(vertices), t, grad=True)
        ctx.save_for_backward(torch.from_numpy(gV).to(vertices), torch.from_numpy(gA).to(vertices))
        return (torch.tensor(vol, dtype=vertices.dtype, device=vertices.device),
                torch.tensor(area, dtype=vertices.dtype, device=vertices.device))

    @staticmethod
    def backward(ctx, gvol, garea):
        gV, gA = ctx.saved_tensors
        return gvol * gV + garea * gA, None


def gaussian_surface(atoms, radii, D, c=1.0, precision=1e-3, max_depth=3, min_edge=0.25,
                     precision_mode=nat.GS_PREC_FP64):
    """Differentiable mesh: returns (vertices, triangles)."""
    if not torch.is_tensor(D):
        D = torch.tensor(float(D), dtype=torch.float64)
    return GaussianSurface.apply(atoms, radii, D, c, precision, max_depth, min_edge, precision_mode)


def volume_area(vertices, triangles):
    return VolumeArea.apply(vertices, triangles)
