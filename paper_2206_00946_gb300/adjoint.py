"""torch.autograd wrapper of the library's discrete adjoint.

    rho, T = ThermalLBMRun.apply(params, rho0, n_steps, K, T0, T_face0, ..., T_face5)

runs n_steps of the step from f = f^eq(rho0, 0), g_i = w_i T0 with the given
per-node face temperatures (FP64 leaf tensors, cast to FP32 for the library),
keeping a checkpoint every K steps, and returns the final rho = sum f and
T = sum g.  backward() calls lbm_adjoint_step, which recomputes each K-step
segment from its checkpoint and returns FP64 gradients with respect to T0
and every face-temperature tensor that was given (None for the others).
All work runs in the CUDA library; this module only moves pointers.
"""
from __future__ import annotations

import numpy as np
import torch

from . import lbm


def face_shape(params: dict, face: int):
    n = (params["nx"], params["ny"], params["nz"])
    t = [b for b in range(3) if b != face // 2]
    return n[t[0]] * n[t[1]]


class ThermalLBMRun(torch.autograd.Function):
    @staticmethod
    def forward(ctx, params, rho0, n_steps, K, T0, *faces):
        dev = T0.device
        rho0_d = rho0.detach().to(device=dev, dtype=torch.float32).contiguous()
        T0_d = T0.detach().to(dtype=torch.float32).contiguous()
        lat = lbm.Lattice(dict(params, storage=lbm.STORE_F32), rho0_d, T0_d,
                          stream=torch.cuda.current_stream(dev).cuda_stream)
        for fc, t in enumerate(faces):
            if t is not None:
                lat.lbm_set_face_T(fc, t.detach().to(dtype=torch.float32).contiguous())
        lat.lbm_record(n_steps, K)
        N = lat.N
        rho = torch.empty(N, dtype=torch.float32, device=dev)
        T = torch.empty(N, dtype=torch.float32, device=dev)
        st = lat.lbm_macros(rho=rho, T=T)
        if st != lbm.OK:
            raise lbm.LBMError(st, "lbm_macros")
        ctx.lat, ctx.n, ctx.params = lat, n_steps, params
        ctx.faces_given = [t is not None for t in faces]
        return rho, T

    @staticmethod
    def backward(ctx, grad_rho, grad_T):
        lat, p = ctx.lat, ctx.params
        dev = grad_rho.device if grad_rho is not None else grad_T.device
        gr = None if grad_rho is None else grad_rho.to(torch.float32).contiguous()
        gt = None if grad_T is None else grad_T.to(torch.float32).contiguous()
        lens = [0 if p["face_kind"][fc] == 0 else face_shape(p, fc) for fc in range(6)]
        dTf = torch.zeros(max(1, sum(lens)), dtype=torch.float64, device=dev)
        dT0 = torch.empty(lat.N, dtype=torch.float64, device=dev)
        lat.lbm_adjoint_step(ctx.n, gr, gt, dTf, dT0)
        out, off = [], 0
        for fc in range(6):
            out.append(dTf[off:off + lens[fc]].clone() if ctx.faces_given[fc] else None)
            off += lens[fc]
        lat.close()
        return (None, None, None, None, dT0, *out)


def run(params, rho0, T0, n_steps, K=100, faces=None):
    """rho, T after n_steps, differentiable with respect to T0 and the face tensors."""
    faces = list(faces) if faces is not None else [None] * 6
    return ThermalLBMRun.apply(params, rho0, n_steps, K, T0, *faces)


def liquid_mass(rho, rho_l, rho_v):
    """sum rho * (1 + tanh((rho - rho_mid) / (0.1 (rho_l - rho_v)))) / 2: the smooth liquid mass."""
    mid = 0.5 * (rho_l + rho_v)
    return (rho * 0.5 * (1 + torch.tanh((rho - mid) / (0.1 * (rho_l - rho_v))))).sum()
