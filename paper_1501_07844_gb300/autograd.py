"""Differentiable Potts solve: gradients of a loss on the labelling after K
unrolled iterations (Algorithm 1, NORMALISED gradient source) with respect
to the data term D and the capacity field S.

Forward: K iterations through the C ABI, saving the state (u, q) every
`checkpoint_every` iterations.  Backward: for each segment, last first, the
state is restored from its checkpoint, the segment is recomputed one
iteration at a time (the kernels are deterministic, so the recomputed states
equal the forward ones bit for bit), and its iterations' reverse-mode steps
run in one pfm_adjoint_steps call.  Memory: K / checkpoint_every checkpoints plus one
segment of states.
"""
import torch

from .binding import FUSED, ISO, Problem


class PottsSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, D, S_field, iters, c, tau, norm, checkpoint_every, s_label):
        D = D.detach().to(torch.float32).contiguous()
        S = None if S_field is None else S_field.detach().to(torch.float32).contiguous()
        prob = Problem(D, S_field=S, s_node=s_label, c=c, tau=tau, norm=norm, schedule=FUSED)
        ckpts = []
        k = 0
        while k < iters:
            ckpts.append((k,) + prob.state_async())
            step = min(checkpoint_every, iters - k)
            prob.iterate(step)
            k += step
        u = prob.labels()
        ctx.prob, ctx.ckpts, ctx.iters, ctx.has_S = prob, ckpts, iters, S is not None
        ctx.ce = checkpoint_every
        return u

    @staticmethod
    def backward(ctx, grad_u):
        prob = ctx.prob
        # the segment states below are read on the problem's stream, which the
        # forward pass captured; allocating them under that stream makes the
        # caching allocator reuse their memory only after those reads
        cur = torch.cuda.current_stream()
        stream = torch.cuda.ExternalStream(prob.stream) if prob.stream else cur
        if stream.cuda_stream != cur.cuda_stream:
            stream.wait_stream(cur)      # grad_u was produced on the caller's stream
        with torch.cuda.stream(stream):
            grads = PottsSolve._backward(ctx, grad_u)
        if stream.cuda_stream != cur.cuda_stream:
            cur.wait_stream(stream)      # the gradients are consumed there
        return grads

    @staticmethod
    def _backward(ctx, grad_u):
        prob = ctx.prob
        ubar = grad_u.detach().to(torch.float32).contiguous().clone()
        q_shape = (prob.n_nodes, prob.ndim) + prob.spatial
        qbar = torch.zeros(q_shape, dtype=torch.float32, device=ubar.device)
        Dbar = torch.zeros_like(ubar)
        Sbar = torch.zeros(prob.spatial, dtype=torch.float32, device=ubar.device) if ctx.has_S else None
        n = 1
        for s in prob.spatial:
            n *= s
        work = torch.empty((prob.ndim + 1) * prob.n_leaf * n, dtype=torch.float32, device=ubar.device)
        dummy = torch.zeros(1, dtype=torch.float32, device=ubar.device)
        for k0, u0, q0 in reversed(ctx.ckpts):
            seg = min(ctx.ce, ctx.iters - k0)
            prob.set_labels(u0)
            prob.set_flows(q0)
            us, qs = [u0], [q0]
            for _ in range(seg):
                prob.iterate(1)
                u1, q1 = prob.state_async()
                us.append(u1)
                qs.append(q1)
            # the segment's reverse steps in one call (equal to pfm_adjoint_step
            # applied from its last iteration to its first)
            prob.adjoint_steps(us, qs[:seg], ubar, qbar, Dbar, Sbar if Sbar is not None else dummy, work)
        return Dbar, Sbar, None, None, None, None, None, None


def potts_solve(D, S_field=None, iters=100, c=0.5, tau=0.11, norm=ISO, checkpoint_every=10, s_label=None):
    """Labelling u after `iters` iterations from u = 1/#L, q = 0; differentiable
    with respect to D ([n_leaf, *spatial], CUDA FP32) and S_field ([*spatial])."""
    return PottsSolve.apply(D, S_field, int(iters), float(c), float(tau), int(norm), int(checkpoint_every), s_label)
