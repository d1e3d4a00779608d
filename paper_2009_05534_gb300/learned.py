"""Learned normalised-offset min-sum: autograd wrapper around the CUDA forward / backward.

The paper's min-sum check rule has one correction factor beta (Sec. III).  Here every
(iteration t, base row r) gets its own pair, m' = beta[t][r] * max(m - gamma[t][r], 0),
initialised to beta = 0.75, gamma = 0 (plain normalised min-sum) and trained by gradient
descent on the binary cross-entropy between sigma(-L) and the transmitted codeword bits.

Both passes run in libldpc.so (`ldpc_learned_forward` / `ldpc_learned_backward`): the
forward pass stores per-iteration checkpoints in a workspace tensor, the backward pass
replays each iteration from its checkpoint and sweeps the layers in reverse.  The
`_iter` variants expose the posteriors after every iteration and take one adjoint per
iteration, for a loss over all of them (the final-posterior loss gives the parameters of
early iterations almost no gradient through the unrolled chain).  torch only holds the
tensors, evaluates the loss and runs the optimiser.
Trained tables decode with the regular path (`decode(..., algo=LEARNED, learned=table)`).
"""
from __future__ import annotations

import ctypes
import itertools
import os

import numpy as np

from . import Graph, _check, _stream_ptr, lib

_P, _I = ctypes.c_void_p, ctypes.c_int


def _bind():
    L = lib()
    if getattr(L, "_learned_bound", False):
        return L
    L.ldpc_learned_workspace_floats.argtypes = [_P, _I, _I, _I]
    L.ldpc_learned_workspace_floats.restype = ctypes.c_size_t
    L.ldpc_learned_forward.argtypes = [_P, _P, _I, _I, _I, _I, _P, _P, _P, _P]
    L.ldpc_learned_forward.restype = _I
    L.ldpc_learned_backward.argtypes = [_P, _P, _I, _I, _I, _I, _P, _P, _P, _P, _P]
    L.ldpc_learned_backward.restype = _I
    L.ldpc_learned_forward_iter.argtypes = [_P, _P, _I, _I, _I, _I, _P, _P, _P, _P]
    L.ldpc_learned_forward_iter.restype = _I
    L.ldpc_learned_backward_iter.argtypes = [_P, _P, _I, _I, _I, _I, _P, _P, _P, _P, _P, _I]
    L.ldpc_learned_backward_iter.restype = _I
    L._learned_bound = True
    return L


def _vp(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def workspace(graph: Graph, batch: int, T: int, n_rows: int = 0):
    import torch
    n = int(_bind().ldpc_learned_workspace_floats(graph.handle, batch, T, n_rows))
    if n == 0 and batch > 0:
        raise ValueError("invalid learned-decoder shape")
    return torch.empty((max(n, 1),), dtype=torch.float32, device="cuda")


def forward(graph: Graph, llr, params, *, n_rows: int = 0, n_tx: int = 0, ws=None, stream=None):
    """Final posteriors [batch][(K_b + n_rows) * Z] of the learned decoder (T = params rows)."""
    import torch
    L = _bind()
    llr = llr.contiguous().float()
    params = params.contiguous().float()
    B, T = llr.shape[0], params.shape[0]
    if ws is None:
        ws = workspace(graph, B, T, n_rows)
    post = torch.empty((B, graph.vars(n_rows)), dtype=torch.float32, device=llr.device)
    _check(L.ldpc_learned_forward(graph.handle, _vp(llr), B, T, n_rows, n_tx, _vp(params),
                                  _stream_ptr(stream), _vp(post), _vp(ws)),
           "ldpc_learned_forward")
    return post, ws


def backward(graph: Graph, grad_post, params, ws, *, n_tx: int, n_rows: int = 0,
             want_grad_llr: bool = False, stream=None):
    """(dLoss/dparams per codeword [batch][T][n_rows][2], dLoss/dLLR or None)."""
    import torch
    L = _bind()
    grad_post = grad_post.contiguous().float()
    params = params.contiguous().float()
    B, T = grad_post.shape[0], params.shape[0]
    gp = torch.empty((B,) + tuple(params.shape), dtype=torch.float32, device=grad_post.device)
    gl = (torch.empty((B, n_tx), dtype=torch.float32, device=grad_post.device)
          if want_grad_llr else None)
    _check(L.ldpc_learned_backward(graph.handle, _vp(grad_post), B, T, n_rows, n_tx,
                                   _vp(params), _stream_ptr(stream), _vp(ws), _vp(gp),
                                   _vp(gl)), "ldpc_learned_backward")
    return gp, gl


def forward_iter(graph: Graph, llr, params, *, n_rows: int = 0, n_tx: int = 0, ws=None,
                 stream=None):
    """Posteriors after every iteration [T][batch][(K_b + n_rows) * Z] (slice T-1 = final)."""
    import torch
    L = _bind()
    llr = llr.contiguous().float()
    params = params.contiguous().float()
    B, T = llr.shape[0], params.shape[0]
    if ws is None:
        ws = workspace(graph, B, T, n_rows)
    post = torch.empty((T, B, graph.vars(n_rows)), dtype=torch.float32, device=llr.device)
    _check(L.ldpc_learned_forward_iter(graph.handle, _vp(llr), B, T, n_rows, n_tx, _vp(params),
                                       _stream_ptr(stream), _vp(post), _vp(ws)),
           "ldpc_learned_forward_iter")
    return post, ws


def backward_iter(graph: Graph, grad_post_iter, params, ws, *, n_tx: int, n_rows: int = 0,
                  want_grad_llr: bool = False, stream=None, detach: bool = False):
    """Gradients of a loss over every iteration's posteriors (adjoints [T][batch][N]).

    detach: no adjoint flows between iterations, so iteration t's parameters get the
    partial derivative of iteration t's own loss term only."""
    import torch
    L = _bind()
    g = grad_post_iter.contiguous().float()
    params = params.contiguous().float()
    T, B = g.shape[0], g.shape[1]
    gp = torch.empty((B,) + tuple(params.shape), dtype=torch.float32, device=g.device)
    gl = torch.empty((B, n_tx), dtype=torch.float32, device=g.device) if want_grad_llr else None
    _check(L.ldpc_learned_backward_iter(graph.handle, _vp(g), B, T, n_rows, n_tx, _vp(params),
                                        _stream_ptr(stream), _vp(ws), _vp(gp), _vp(gl),
                                        int(detach)),
           "ldpc_learned_backward_iter")
    return gp, gl


def _autograd():
    import torch

    class LearnedDecodeFn(torch.autograd.Function):
        @staticmethod
        def forward(ctx, params, llr, graph, n_rows, n_tx):
            post, ws = forward(graph, llr, params, n_rows=n_rows, n_tx=n_tx)
            ctx.graph, ctx.n_rows, ctx.n_tx = graph, n_rows, llr.shape[1]
            ctx.save_for_backward(params, ws)
            return post

        @staticmethod
        def backward(ctx, grad_post):
            params, ws = ctx.saved_tensors
            gp, gl = backward(ctx.graph, grad_post, params, ws, n_tx=ctx.n_tx,
                              n_rows=ctx.n_rows, want_grad_llr=ctx.needs_input_grad[1])
            return gp.sum(0), gl, None, None, None

    class LearnedDecodeIterFn(torch.autograd.Function):
        @staticmethod
        def forward(ctx, params, llr, graph, n_rows, n_tx, detach):
            post, ws = forward_iter(graph, llr, params, n_rows=n_rows, n_tx=n_tx)
            ctx.graph, ctx.n_rows, ctx.n_tx, ctx.detach = graph, n_rows, llr.shape[1], detach
            ctx.save_for_backward(params, ws)
            return post

        @staticmethod
        def backward(ctx, grad_post):
            params, ws = ctx.saved_tensors
            gp, gl = backward_iter(ctx.graph, grad_post, params, ws, n_tx=ctx.n_tx,
                                   n_rows=ctx.n_rows, want_grad_llr=ctx.needs_input_grad[1],
                                   detach=ctx.detach)
            return gp.sum(0), gl, None, None, None, None

    return LearnedDecodeFn, LearnedDecodeIterFn


_FN = None


def learned_decode(params, llr, graph: Graph, n_rows: int = 0, n_tx: int = 0,
                   every_iteration: bool = False, detach: bool = False):
    """Differentiable learned decode: posteriors = f(params, llr) [batch][N], or with
    every_iteration the posteriors after each iteration [T][batch][N] (detach: gradients
    do not flow between iterations)."""
    global _FN
    if _FN is None:
        _FN = _autograd()
    if every_iteration:
        return _FN[1].apply(params, llr, graph, n_rows, n_tx, bool(detach))
    return _FN[0].apply(params, llr, graph, n_rows, n_tx)


def bce_loss(post, codewords, iter_weights=None):
    """Mean binary cross-entropy between sigma(-L) (P[bit = 1]) and the codeword bits.

    post [batch][N], or [T][batch][N] with iter_weights [T]: the weighted sum over
    iterations of each iteration's mean BCE."""
    import torch.nn.functional as F
    c = codewords[:, : post.shape[-1]].float()
    per = F.softplus(-post) + c * post
    if post.dim() == 2:
        return per.mean()
    return (per.mean(dim=(1, 2)) * iter_weights).sum()


def init_params(T: int, n_rows: int, beta: float = 0.75, gamma: float = 0.0):
    import torch
    p = torch.zeros((T, n_rows, 2), dtype=torch.float32, device="cuda")
    p[..., 0] = beta
    p[..., 1] = gamma
    return p


def save_checkpoint(path, params, opt, step: int, history=()):
    """Write the (beta, gamma) table, the Adam state and the step counter with torch.save."""
    import torch
    torch.save({"params": params.detach().cpu(), "adam": opt.state_dict(), "step": int(step),
                "loss": [float(x) for x in history]}, str(path) + ".tmp")
    os.replace(str(path) + ".tmp", str(path))


def load_checkpoint(path):
    import torch
    return torch.load(str(path), map_location="cpu", weights_only=False)


def train(graph: Graph, n_rows: int, T: int, batches, *, lr: float = 1e-3, params=None,
          log_every: int = 0, n_steps: int | None = None, checkpoint=None,
          checkpoint_every: int = 0, iter_weights=None, detach: bool = False):
    """Adam on the BCE loss.  Returns (params, loss history).

    iter_weights ([T] or None): None trains on the final posteriors; otherwise the loss is
    the weighted sum of the BCE after every iteration, and with detach each iteration's
    parameters follow only their own iteration's term.

    batches: an iterable of (llr float CUDA [B][n_tx], codeword bits CUDA [B][N]) pairs, or a
    callable k -> pair for steps k = 0 .. n_steps-1.  With a checkpoint path, an existing
    checkpoint is resumed (table, Adam state, step counter; an iterable skips the steps
    already taken) and the state is saved every checkpoint_every steps and at the end.
    """
    import torch
    p = init_params(T, n_rows) if params is None else params.clone()
    p.requires_grad_(True)
    opt = torch.optim.Adam([p], lr=lr)
    start, hist = 0, []
    if checkpoint is not None and os.path.exists(str(checkpoint)):
        ck = load_checkpoint(checkpoint)
        if tuple(ck["params"].shape) != tuple(p.shape):
            raise ValueError("checkpoint table shape does not match (T, n_rows, 2)")
        with torch.no_grad():
            p.copy_(ck["params"].to(p.device))
        opt.load_state_dict(ck["adam"])
        start, hist = int(ck["step"]), list(ck["loss"])
    if callable(batches):
        if n_steps is None:
            raise ValueError("a batch function needs n_steps")
        stream = (batches(k) for k in range(start, n_steps))
    else:
        stream = itertools.islice(batches, start, None)
    w = None
    if iter_weights is not None:
        w = torch.as_tensor(np.asarray(iter_weights, np.float32), device=p.device)
        if w.shape != (T,):
            raise ValueError("iter_weights needs one weight per iteration")
    k = start
    for llr, cw in stream:
        opt.zero_grad(set_to_none=True)
        post = learned_decode(p, llr, graph, n_rows, llr.shape[1], every_iteration=w is not None,
                              detach=detach)
        loss = bce_loss(post, cw, w)
        loss.backward()
        opt.step()
        hist.append(float(loss.item()))
        k += 1
        if log_every and (k - 1) % log_every == 0:
            print(f"step {k - 1}: loss {hist[-1]:.5f}", flush=True)
        if checkpoint is not None and checkpoint_every and k % checkpoint_every == 0:
            save_checkpoint(checkpoint, p, opt, k, hist)
    if checkpoint is not None:
        save_checkpoint(checkpoint, p, opt, k, hist)
    return p.detach(), np.array(hist)
