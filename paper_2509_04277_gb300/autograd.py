"""``torch.autograd.Function`` over the rod rollout and its hand-written CUDA adjoint.

``RodRollout.apply(batch, n_steps, ckpt_every, K, uhat, vel0, pos0, quat0=None,
omega0=None)`` sets the per-joint stiffness ``K`` and intrinsic Darboux vectors ``uhat``
([n_elem, 4] device tensors, the per-joint layout of ``rod_set_material``), the initial
velocities and positions ([n_elem, 4]) and, when given, the initial frames (quaternions
x, y, z, w) and body angular velocities ([n_elem, 4]), runs ``rod_rollout`` and returns
the node trajectory [n_steps, n_elem, 4].  The backward pass calls ``rod_adjoint``.
Frames and angular velocities that are not given start from the batch's state at the
time of the call and receive no gradient.
"""
from __future__ import annotations

import torch

from . import corde


class RodRollout(torch.autograd.Function):
    @staticmethod
    def forward(ctx, batch, n_steps, ckpt_every, K, uhat, vel0, pos0, quat0=None, omega0=None):
        mat = torch.cat([K.detach(), uhat.detach()], dim=1).contiguous()
        corde.rod_set_material(batch.handle, mat)
        corde.rod_set_state(batch.handle, pos4=pos0.detach().contiguous(), vel4=vel0.detach().contiguous(),
                            quat4=None if quat0 is None else quat0.detach().contiguous(),
                            omega4=None if omega0 is None else omega0.detach().contiguous())
        traj = batch.rollout(int(n_steps), int(ckpt_every))
        ctx.batch = batch
        ctx.frames = (quat0 is not None, omega0 is not None)
        return traj

    @staticmethod
    def backward(ctx, g_traj):
        g = ctx.batch.adjoint(g_traj.contiguous())
        gq = g["quat0"] if ctx.frames[0] else None
        go = g["omega0"] if ctx.frames[1] else None
        return None, None, None, g["K"], g["uhat"], g["vel0"], g["pos0"], gq, go
