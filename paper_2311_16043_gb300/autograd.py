"""``torch.autograd.Function`` over the C ABI: visibility of rays cast from
every Gaussian in a direction set, differentiable with respect to mean,
scale, quaternion and opacity through the hand-written adjoint
(``rt_trace_visibility_backward``).

The forward builds the LBVH, traces, and keeps a per-ray hit log when it fits
the memory budget; otherwise (or for rays that overflow the log) the backward
re-traverses.  Log-scale parameterisations compose in torch
(``scale = log_scale.exp()``), which supplies the s * d/ds factor.
"""
from __future__ import annotations

import torch

from . import rt


class Visibility(torch.autograd.Function):
    @staticmethod
    def forward(ctx, mean, scale, quat, opacity, dirs, prm=None, hit_cap=64, log_budget_bytes=1 << 30):
        mean_c, scale_c, quat_c, opac_c = (t.detach().contiguous() for t in (mean, scale, quat, opacity))
        dirs_c = dirs.detach().contiguous()
        bvh = rt.rt_build_bvh(mean_c, scale_c, quat_c, opac_c, prm)
        rs = rt.rayspec(rt.RT_RAYS_DIRS, dirs=dirs_c)
        R = rt.rt_rayspec_count(bvh, rs)
        cap = hit_cap if R * hit_cap * 4 <= log_budget_bytes else 0
        hit_ids = torch.empty((R, cap), dtype=torch.int32, device=mean.device) if cap else None
        hit_count = torch.empty(R, dtype=torch.int32, device=mean.device) if cap else None
        opts = rt.trace_opts(hit_ids=hit_ids, hit_count=hit_count)
        T = rt.rt_trace_visibility(bvh, rs, opts=opts)
        ctx.bvh, ctx.rs = bvh, rs
        ctx.save_for_backward(mean_c, scale_c, quat_c, opac_c, T,
                              *(x for x in (hit_ids, hit_count) if x is not None))
        ctx.has_log = cap > 0
        return T.view(bvh.n, dirs.shape[0])

    @staticmethod
    def backward(ctx, gT):
        saved = ctx.saved_tensors
        mean, scale, quat, opac, T = saved[:5]
        hit_ids, hit_count = (saved[5], saved[6]) if ctx.has_log else (None, None)
        g = rt.rt_trace_visibility_backward(ctx.bvh, ctx.rs, mean, scale, quat, opac, T,
                                            gT.contiguous().view(-1), hit_ids, hit_count)
        return g["mean"], g["scale"], g["quat"], g["opacity"], None, None, None, None


def visibility(mean, scale, quat, opacity, dirs, prm=None, hit_cap=64, log_budget_bytes=1 << 30):
    """T[n, K]: transmittance of the ray from each Gaussian along each direction."""
    return Visibility.apply(mean, scale, quat, opacity, dirs, prm, hit_cap, log_budget_bytes)
