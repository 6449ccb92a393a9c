"""torch.autograd.Function over the acoustic forward model.

``acoustic_modeling(m, src_wav, ...)`` returns the receiver traces of
``acoustic_forward``; its backward pass returns the vector-Jacobian products
with respect to the squared slowness ``m`` (``acoustic_gradient``, the
adjoint-state FWI gradient with forward-wavefield checkpointing) and with
respect to the source wavelets (``acoustic_adjoint``).  Everything runs in the
library's CUDA kernels; this module only wires the calls into autograd.
"""
from __future__ import annotations

import torch

from . import acoustic_adjoint, acoustic_forward, acoustic_gradient


class AcousticModeling(torch.autograd.Function):
    @staticmethod
    def forward(ctx, m, src_wav, grid, so, dt, src_xyz, rec_xyz, damp, checkpoint_every):
        m = m.contiguous()
        src_wav = src_wav.contiguous()
        nt = int(src_wav.shape[1])
        rec, _ = acoustic_forward(grid, so, dt, nt, m, src_xyz, src_wav, rec_xyz, damp=damp,
                                  return_final=False)
        ctx.save_for_backward(m, src_wav)
        ctx.cfg = (grid, so, dt, nt, src_xyz, rec_xyz, damp, checkpoint_every)
        return rec

    @staticmethod
    def backward(ctx, grad_rec):
        m, src_wav = ctx.saved_tensors
        grid, so, dt, nt, src_xyz, rec_xyz, damp, ck = ctx.cfg
        grad_rec = grad_rec.contiguous()
        gm = gq = None
        if ctx.needs_input_grad[0]:
            gm = acoustic_gradient(grid, so, dt, nt, m, src_xyz, src_wav, rec_xyz, grad_rec,
                                   damp=damp, checkpoint_every=ck)
        if ctx.needs_input_grad[1]:
            gq = acoustic_adjoint(grid, so, dt, nt, m, src_xyz, rec_xyz, grad_rec, damp=damp)
        return gm, gq, None, None, None, None, None, None, None


def acoustic_modeling(m, src_wav, grid, so, dt, src_xyz, rec_xyz, damp=None, checkpoint_every=0):
    """Differentiable receiver traces d(m, q) [nshots][nt][nrec]."""
    return AcousticModeling.apply(m, src_wav, grid, so, dt, src_xyz, rec_xyz, damp,
                                  checkpoint_every)
