"""Differentiable Kalman fit: torch.autograd.Function over mkf_fit_tracks (the
forward, with per-layer checkpoints) and mkf_fit_tracks_adjoint (the
hand-written reverse sweep).  Gradients flow to the hit positions, the
per-layer alignment and the per-layer thickness; the start state is treated
as a constant."""
import torch

from . import api


class KalmanFitFunction(torch.autograd.Function):
    @staticmethod
    def forward(fctx, hit_xyz, align, x0, mctx, lcov, layer, hits, init_par, init_cov):
        T, K = int(hits.shape[0]), int(hits.shape[1])
        ckpt = torch.empty((K, 27, T), dtype=torch.float32, device=hit_xyz.device)
        out = api.mkf_fit_tracks(mctx, hit_xyz.detach().contiguous(), lcov, layer, hits, init_par, init_cov,
                                 align=None if align is None else align.detach().contiguous(),
                                 x0=None if x0 is None else x0.detach().contiguous(), ckpt=ckpt)
        fctx.mctx = mctx
        fctx.has_align = align is not None
        fctx.has_x0 = x0 is not None
        fctx.save_for_backward(hit_xyz.detach(), align.detach() if align is not None else None,
                               x0.detach() if x0 is not None else None, lcov, layer, hits, init_par, init_cov, ckpt)
        fctx.set_materialize_grads(False)
        fctx.mark_non_differentiable(out["ok"])
        return out["chi2"], out["par"], out["cov"], out["ok"]

    @staticmethod
    def backward(fctx, g_chi2, g_par, g_cov, g_ok):
        hit_xyz, align, x0, lcov, layer, hits, init_par, init_cov, ckpt = fctx.saved_tensors

        def c(t):
            return None if t is None else t.contiguous()

        g = api.mkf_fit_tracks_adjoint(fctx.mctx, hit_xyz.contiguous(), lcov, layer, hits, init_par, init_cov, ckpt,
                                       g_chi2=c(g_chi2), g_par=c(g_par), g_cov=c(g_cov),
                                       align=None if align is None else align.contiguous(),
                                       x0=None if x0 is None else x0.contiguous())
        return (g["g_hit"], g["g_align"] if fctx.has_align else None, g["g_x0"] if fctx.has_x0 else None,
                None, None, None, None, None, None)


def kalman_fit(mctx, hit_xyz, lcov, layer, hits, init_par, init_cov, align=None, x0=None):
    """Differentiable outward fit.  hit_xyz [3][H] (requires_grad allowed),
    align [L][3] and x0 [L] optional (requires_grad allowed).  Returns
    (chi2 [T], par [6][T], cov [21][T], ok [T])."""
    return KalmanFitFunction.apply(hit_xyz, align, x0, mctx, lcov, layer, hits, init_par, init_cov)
