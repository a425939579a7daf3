"""torch.autograd.Function over the march (argument marshalling only: the forward is
mot_march, the backward the adjoint march mot_adjoint_begin/run/end).

    J = march(eps_r, taps, wave, n_steps, probes=None, checkpoint_every=None, ...)

eps_r is a float64 tensor [W][V][U] (requires_grad for gradients); the excitation is
the tested plane wave of Eq. E, E_n = chi e_n, generated on the GPU from `wave`
(dict k_hat, p_hat, f_c, sigma_t, t0), so it depends on eps_r through chi and the
adjoint gradient includes that dependence.  The result is J [N][M][3] (float64, on the
GPU), or J at the voxels `probes` only, [N][len(probes)][3].

    E = probe_field(J, pctx)

is the scattered field at probe voxels outside (or inside) the grid, the objective of
field-energy problems: for O = sum over gated steps of |E|^2, O.backward() runs the
transposed probe operator and then the adjoint march.

Checkpointing (checkpoint_every = K): the forward keeps only, at every K-step
boundary b, the block of the last min(b, ell) currents (they determine every later
step, see mot_restart); the backward walks the segments from the last to the first,
recomputes each one's currents from its block with mot_restart + mot_march, and
advances the adjoint over it.  Device memory then holds one segment and the blocks
instead of all N currents; the forward is marched twice.  Without checkpointing all
N currents are kept for the backward.
"""
import numpy as np
import torch

from .mot import Context


def _plane_wave(ctx, wave, n_first, n_count):
    E = torch.empty((n_count, ctx.M, 3), dtype=torch.float64, device="cuda")
    ctx.plane_wave(wave["k_hat"], wave["p_hat"], wave["f_c"], wave["sigma_t"], wave["t0"],
                   n_first, n_count, out=E)
    return E


def _march_into(ctx, wave, n_first, n_count, out):
    """March steps n_first .. n_first + n_count - 1 into the device tensor `out`."""
    ctx.set_excitation(_plane_wave(ctx, wave, n_first, n_count))
    ctx.march(n_count, out=out)


class MarchFunction(torch.autograd.Function):
    @staticmethod
    def forward(fctx, eps_r, taps, wave, n_steps, probes, checkpoint_every, options):
        eps = eps_r.detach().cpu().numpy().astype(np.float64)
        ctx = Context(eps, taps, **options)
        M = ctx.M
        K = checkpoint_every or n_steps
        seg = min(K, n_steps)
        probe_idx = None if probes is None else torch.as_tensor(probes, device="cuda").long()
        out_cols = M if probe_idx is None else probe_idx.numel()
        J_out = torch.empty((n_steps, out_cols, 3), dtype=torch.float64, device="cuda")
        keep_all = checkpoint_every is None
        J_all = torch.empty((n_steps, M, 3), dtype=torch.float64, device="cuda") if keep_all else None
        blocks = {}
        buf = torch.empty((seg, M, 3), dtype=torch.float64, device="cuda")
        tail = None                                # last currents before the segment
        done = 0
        while done < n_steps:
            k = min(seg, n_steps - done)
            Js = J_all[done:done + k] if keep_all else buf[:k]
            _march_into(ctx, wave, done + 1, k, Js)
            J_out[done:done + k] = Js if probe_idx is None else Js[:, probe_idx]
            done += k
            if not keep_all and done < n_steps:
                # block of the last min(done, ell) currents at the boundary `done`
                h = min(done, ctx.ell)
                prev = tail if tail is not None else Js[:0]
                joined = torch.cat([prev, Js[:k]])[-h:]
                blocks[done] = joined.clone()
                tail = joined
        fctx.mot = ctx
        fctx.wave, fctx.n_steps, fctx.K = wave, n_steps, seg
        fctx.probe_idx, fctx.J_all, fctx.blocks = probe_idx, J_all, blocks
        fctx.eps, fctx.eps_shape, fctx.eps_device = eps, eps_r.shape, eps_r.device
        fctx.taps, fctx.options = taps, options
        return J_out

    @staticmethod
    def backward(fctx, grad_out):
        ctx, wave, N, K = fctx.mot, fctx.wave, fctx.n_steps, fctx.K
        M = ctx.M
        grad_out = grad_out.to(device="cuda", dtype=torch.float64).contiguous()

        def dO_dJ(lo, hi):                         # g_n for steps lo .. hi (1-based)
            if fctx.probe_idx is None:
                return grad_out[lo - 1:hi].contiguous()
            g = torch.zeros((hi - lo + 1, M, 3), dtype=torch.float64, device="cuda")
            # a voxel listed twice among the probes receives both contributions
            g.index_add_(1, fctx.probe_idx, grad_out[lo - 1:hi])
            return g

        adj = Context(fctx.eps, fctx.taps, **fctx.options)
        try:
            adj.adjoint_begin(N)
            if fctx.J_all is not None:
                adj.adjoint_run(N, fctx.J_all, 1, dO_dJ(1, N))
            else:
                L = max(len(fctx.taps), 2)
                hi = N
                while hi >= 1:
                    lo = ((hi - 1) // K) * K + 1     # segment lo .. hi after the boundary lo - 1
                    b = lo - 1
                    block = fctx.blocks.get(b)
                    if b == 0:
                        ctx.restart(0, None)
                        pre = torch.empty((0, M, 3), dtype=torch.float64, device="cuda")
                    else:
                        ctx.restart(b, block)
                        pre = block[-(L - 1):] if L > 1 else block[:0]
                    Js = torch.empty((hi - lo + 1, M, 3), dtype=torch.float64, device="cuda")
                    _march_into(ctx, wave, lo, hi - lo + 1, Js)
                    win = torch.cat([pre, Js]).contiguous()
                    adj.adjoint_run(hi - lo + 1, win, lo - pre.shape[0], dO_dJ(lo, hi))
                    hi = lo - 1
            grad = adj.adjoint_end()
        finally:
            adj.close()
            ctx.close()
            fctx.mot = None
        g = torch.as_tensor(grad, dtype=torch.float64).reshape(fctx.eps_shape)
        return g.to(fctx.eps_device), None, None, None, None, None, None


class ProbeFieldFunction(torch.autograd.Function):
    """E = probe field of J (mot_probe_field); backward: the transposed probe operator
    (mot_probe_transpose).  `pctx` is a Context of the same grid whose probes are set."""

    @staticmethod
    def forward(fctx, J, pctx):
        J = J.detach().to(device="cuda", dtype=torch.float64).contiguous()
        E = torch.empty((J.shape[0], pctx.n_probes, 3), dtype=torch.float64, device="cuda")
        pctx.probe_field(J, out=E)
        fctx.pctx = pctx
        fctx.shape = J.shape
        return E

    @staticmethod
    def backward(fctx, grad_E):
        g = torch.empty(fctx.shape, dtype=torch.float64, device="cuda")
        fctx.pctx.probe_transpose(grad_E.to(dtype=torch.float64).contiguous(), out=g)
        return g, None


def probe_field(J, pctx):
    """Scattered field E [N][P][3] at the probes of `pctx` for currents J [N][M][3],
    differentiable in J: E^s_p(t_n) = sum_l sum_m G_l(r_p - r_m) J_{n-l,m}."""
    return ProbeFieldFunction.apply(J, pctx)


def march(eps_r, taps, wave, n_steps, probes=None, checkpoint_every=None,
          precision="fp64", scheme="direct", block=0):
    """J (or J at `probes`) of the tested plane wave `wave` on eps_r, differentiable in
    eps_r; see the module docstring."""
    options = {"precision": precision, "scheme": scheme, "block": block}
    return MarchFunction.apply(eps_r, np.asarray(taps, dtype=np.float64), wave, n_steps,
                               probes, checkpoint_every, options)
