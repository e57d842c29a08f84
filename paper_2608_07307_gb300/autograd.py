"""torch.autograd bindings of the SRP evaluation.

Forward runs srp_eval_batch; backward runs srp_grad, the hand-written adjoint
with the hit set frozen (each ray keeps the triangles it hit, the window keeps
its extreme vertices), which returns the gradients with respect to the Sun
direction, the Sun distance, the optical coefficients (rho_s, rho_d) of every
material and the joint angle parameters.  All arithmetic runs in libsrp's
kernels; this module only moves tensors across the C ABI, except the attitude
composition of ``srp_accel_inertial`` (a 3 x 3 rotation built from the
quaternion with torch operations, differentiated by torch).
"""
from __future__ import annotations

import numpy as np
import torch

from . import srp as _srp


def _t(x, like):
    return torch.from_numpy(x).to(like.device) if isinstance(x, np.ndarray) else x


class SRPForceFunction(torch.autograd.Function):
    """(sun_dirs [n,3], sun_dist [n], mat [M,2], angles [P]) -> (F [n,3], T [n,3])."""

    @staticmethod
    def forward(ctx, sun_dirs, sun_dist, mat, angles, handle, mesh_id, opts):
        handle.set_materials(mesh_id, mat)
        handle.set_panel_angles(mesh_id, angles)
        F, T = handle.eval_batch(mesh_id, sun_dirs.detach().contiguous(), sun_dist.detach().contiguous(), **opts)
        ctx.save_for_backward(sun_dirs, sun_dist, mat, angles)
        ctx.handle, ctx.mesh_id, ctx.opts = handle, mesh_id, opts
        return _t(F, sun_dirs), _t(T, sun_dirs)

    @staticmethod
    def backward(ctx, gF, gT):
        sun_dirs, sun_dist, mat, angles = ctx.saved_tensors
        h = ctx.handle
        h.set_materials(ctx.mesh_id, mat)
        h.set_panel_angles(ctx.mesh_id, angles)
        gF = torch.zeros_like(sun_dirs) if gF is None else gF
        gT = torch.zeros_like(sun_dirs) if gT is None else gT
        g = h.grad(ctx.mesh_id, sun_dirs.detach().contiguous(), gF.detach().to(sun_dirs.dtype).contiguous(),
                   gT.detach().to(sun_dirs.dtype).contiguous(), sun_dist.detach().contiguous(), **ctx.opts)
        out = [_t(g["sun"], sun_dirs), _t(g["dist"], sun_dirs), _t(g["mat"], sun_dirs).to(mat.device),
               _t(g["angle"], sun_dirs).to(angles.device)]
        return out[0], out[1], out[2].to(mat.dtype), out[3].to(angles.dtype), None, None, None


def srp_force(handle, mesh_id, sun_dirs, sun_dist, mat, angles, N=256, bounces=1, P0=4.56e-6, eps_rel=1e-9,
              panel_mode=_srp.PANELS_TRACK_OFFSET):
    """Differentiable SRP force and torque (body frame) of a loaded mesh.
    sun_dirs [n,3] float64 (body frame, any length), sun_dist [n] AU,
    mat [n_mats,2] optical coefficients, angles [n_parts] joint offsets
    (PANELS_TRACK_OFFSET) or commanded angles (PANELS_SET)."""
    opts = dict(N=N, bounces=bounces, P0=P0, eps_rel=eps_rel, panel_mode=panel_mode)
    return SRPForceFunction.apply(sun_dirs, sun_dist, mat, angles, handle, mesh_id, opts)


def quat_to_matrix(q):
    """Rotation matrices [n,3,3] (body -> inertial) of scalar-first quaternions
    [n,4], normalised first (the gradient is that of the normalised map)."""
    q = q / q.norm(dim=-1, keepdim=True)
    w, x, y, z = q.unbind(-1)
    return torch.stack([
        torch.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)], -1),
        torch.stack([2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)], -1),
        torch.stack([2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], -1)], -2)


def srp_accel_inertial(handle, mesh_id, q, sun_inertial, sun_dist, mat, angles, mass, **opts):
    """SRP acceleration in the inertial frame for attitudes q [n,4] (body ->
    inertial): the Sun direction is rotated into the body frame, the force is
    evaluated there and rotated back, divided by the mass.  Differentiable in
    q, the Sun direction and distance, the coefficients and the angles."""
    R = quat_to_matrix(q)
    s_body = torch.einsum("nji,nj->ni", R, sun_inertial)
    F, T = srp_force(handle, mesh_id, s_body, sun_dist, mat, angles, **opts)
    return torch.einsum("nij,nj->ni", R, F) / mass, T
