"""torch.autograd.Function wrappers of the adjoint kernels (differentiable ray end points).

`RayEndpoints.apply(tc, *records)` maps the gridded potential records of every level (FP64
CUDA tensors [count, n_slices, 4]) to the rays' end points on their iso-eta stop surfaces,
xi [3, N]; its backward runs mt_trace_rays_adjoint (reverse mode) on the GPU.
`CoarsePhiEndpoints.apply(tc, phi0)` starts from the coarse potential phi0 [N, N, N]: the
records are rebuilt on the GPU by the field model (mt_field_from_coarse_phi, with the workload's
phi0-independent detail terms computed once) and the backward adds mt_pullback_coarse_phi, its
transpose.  Both integrate in FP64 arithmetic (the adjoint's forward map).
"""
from __future__ import annotations

import numpy as np
import torch

from . import binding as B


class TraceContext:
    """The part of a differentiable trace that is not differentiated: geometry, rays, parameters."""

    def __init__(self, workload, checkpoint_every=64):
        self.w = workload
        self.params = B.TraceParams.from_workload(workload)
        self.dirs = torch.from_numpy(np.ascontiguousarray(workload.dirs)).cuda()
        self.checkpoint_every = checkpoint_every

    def morton_index(self):
        """key[i * N^2 + j * N + k] = Morton key of coarse cell (i, j, k) (CUDA int64)."""
        if getattr(self, "_key", None) is None:
            from . import inputs as I
            n = self.w.n_coarse
            ii, jj, kk = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
            self._key = torch.from_numpy(I.morton3(ii.ravel(), jj.ravel(), kk.ravel()).astype(np.int64)).cuda()
        return self._key

    def field_records(self, phi0):
        """The records of every level from phi0 [N, N, N] (CUDA), by the field model on the GPU; the
        terms that do not depend on phi0 (the workload's detail tiles) are computed once."""
        from . import inputs as I
        w = self.w
        if getattr(self, "_base", None) is None:
            zero = I.records_from_phi0(w, np.zeros((w.n_coarse,) * 3))
            self._base = [torch.from_numpy(l.records).cuda() for l in zero]
            self._geom = B.Octree(w.box, w.n_coarse, w.periodic, w.slice_eta, w.levels, w.bg, "fp64")
        key = self.morton_index()
        phi_m = torch.empty(key.numel(), dtype=torch.float64, device=key.device)
        phi_m[key] = phi0.detach().to(torch.float64).reshape(-1)
        return B.field_from_coarse_phi(self._geom, phi_m, w.slice_weight, base=self._base)

    def tree(self, records):
        w = self.w
        levels = [_Lv(l.keys, r) for l, r in zip(w.levels, records)]
        return B.Octree(w.box, w.n_coarse, w.periodic, w.slice_eta, levels, w.bg, "fp64",
                        residency=B.MT_DEVICE_BORROW)

    def endpoints(self, records):
        tree = self.tree(records)
        out = B.alloc_outputs(self.dirs.shape[1], self.dirs.device, names=["xi", "status"])
        B.trace_rays_adjoint(tree, self.params, self.dirs, jacobian=False, lensing=True, out=out)
        torch.cuda.synchronize()
        tree.free()
        return out["xi"]

    def record_grads(self, records, grad_xi):
        tree = self.tree(records)
        res = B.trace_rays_adjoint(tree, self.params, self.dirs, jacobian=False, lensing=False,
                                   dL_dxi=grad_xi.contiguous().to(torch.float64),
                                   checkpoint_every=self.checkpoint_every,
                                   out=B.alloc_outputs(self.dirs.shape[1], self.dirs.device, names=["status"]))
        torch.cuda.synchronize()
        return tree, res["dL_drec"]


class _Lv:
    def __init__(self, keys, records):
        self.keys = keys
        self.records = records


class RayEndpoints(torch.autograd.Function):
    @staticmethod
    def forward(ctx, tc, *records):
        recs = [r.detach().to(torch.float64).contiguous() for r in records]
        ctx.tc = tc
        ctx.save_for_backward(*recs)
        return tc.endpoints(recs)

    @staticmethod
    def backward(ctx, grad_xi):
        tree, grads = ctx.tc.record_grads(ctx.saved_tensors, grad_xi)
        tree.free()
        return (None, *grads)


class CoarsePhiEndpoints(torch.autograd.Function):
    @staticmethod
    def forward(ctx, tc, phi0):
        recs = tc.field_records(phi0)
        ctx.tc = tc
        ctx.recs = recs
        return tc.endpoints(recs)

    @staticmethod
    def backward(ctx, grad_xi):
        tc = ctx.tc
        tree, grads = tc.record_grads(ctx.recs, grad_xi)
        g = B.pullback_coarse_phi(tree, grads, tc.w.slice_weight, tc.w.n_coarse)
        torch.cuda.synchronize()
        tree.free()
        n = tc.w.n_coarse
        return None, g[tc.morton_index()].reshape(n, n, n)
