"""torch.autograd bindings of the SRP evaluation.

Forward runs srp_eval_batch; backward runs srp_grad, the hand-written adjoint
with the hit set frozen (each ray keeps the triangles it hit, the window keeps
its extreme vertices), which returns the gradients with respect to the Sun
direction, the Sun distance, the optical coefficients (rho_s, rho_d) of every
material, the joint angle parameters and, for the inertial-frame
acceleration, the attitude quaternion.  All arithmetic runs in libsrp's
kernels; this module only moves tensors across the C ABI.
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


class SRPAccelFunction(torch.autograd.Function):
    """(q [n,4], sun_inertial [n,3], sun_dist [n], mat [M,2], angles [P]) ->
    (acceleration [n,3] m/s^2 inertial frame, torque [n,3] N m body frame)."""

    @staticmethod
    def forward(ctx, q, sun_inertial, sun_dist, mat, angles, handle, mesh_id, opts):
        handle.set_materials(mesh_id, mat)
        handle.set_panel_angles(mesh_id, angles)
        a, T = handle.eval_batch(mesh_id, sun_inertial.detach().contiguous(), sun_dist.detach().contiguous(),
                                 quat=q.detach().contiguous(), **opts)
        ctx.save_for_backward(q, sun_inertial, sun_dist, mat, angles)
        ctx.handle, ctx.mesh_id, ctx.opts = handle, mesh_id, opts
        return _t(a, sun_inertial), _t(T, sun_inertial)

    @staticmethod
    def backward(ctx, ga, gT):
        q, s_in, dist, mat, angles = ctx.saved_tensors
        h = ctx.handle
        h.set_materials(ctx.mesh_id, mat)
        h.set_panel_angles(ctx.mesh_id, angles)
        ga = torch.zeros_like(s_in) if ga is None else ga
        gT = torch.zeros_like(s_in) if gT is None else gT
        g = h.grad(ctx.mesh_id, s_in.detach().contiguous(), ga.detach().to(s_in.dtype).contiguous(),
                   gT.detach().to(s_in.dtype).contiguous(), dist.detach().contiguous(), quat=q.detach().contiguous(),
                   **ctx.opts)
        return (_t(g["quat"], s_in).to(q.dtype), _t(g["sun"], s_in), _t(g["dist"], s_in),
                _t(g["mat"], s_in).to(mat.device, mat.dtype), _t(g["angle"], s_in).to(angles.device, angles.dtype),
                None, None, None)


def srp_accel_inertial(handle, mesh_id, q, sun_inertial, sun_dist, mat, angles, N=256, bounces=1, P0=4.56e-6,
                       eps_rel=1e-9, panel_mode=_srp.PANELS_TRACK_OFFSET):
    """SRP acceleration in the inertial frame, R(q) F_body / mass (mass of the
    loaded mesh), and the body-frame torque, for attitudes q [n,4] (body ->
    inertial, scalar first) and inertial Sun directions [n,3].
    Differentiable in q, the Sun direction and distance, the coefficients and
    the angles; the rotation and its derivative run in the library."""
    opts = dict(N=N, bounces=bounces, P0=P0, eps_rel=eps_rel, panel_mode=panel_mode)
    return SRPAccelFunction.apply(q, sun_inertial, sun_dist, mat, angles, handle, mesh_id, opts)
