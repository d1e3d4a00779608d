"""Learned normalised-offset min-sum: autograd wrapper around the CUDA forward / backward.

The paper's min-sum check rule has one correction factor beta (Sec. III).  Here every
(iteration t, base row r) gets its own pair, m' = beta[t][r] * max(m - gamma[t][r], 0),
initialised to beta = 0.75, gamma = 0 (plain normalised min-sum) and trained by gradient
descent on the binary cross-entropy between sigma(-L) and the transmitted codeword bits.

Both passes run in libldpc.so (`ldpc_learned_forward` / `ldpc_learned_backward`): the
forward pass stores per-iteration checkpoints in a workspace tensor, the backward pass
replays each iteration from its checkpoint and sweeps the layers in reverse.  torch only
holds the tensors, evaluates the loss on the final posteriors and runs the optimiser.
Trained tables decode with the regular path (`decode(..., algo=LEARNED, learned=table)`).
"""
from __future__ import annotations

import ctypes

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

    return LearnedDecodeFn


_FN = None


def learned_decode(params, llr, graph: Graph, n_rows: int = 0, n_tx: int = 0):
    """Differentiable learned decode: posteriors = f(params, llr)."""
    global _FN
    if _FN is None:
        _FN = _autograd()
    return _FN.apply(params, llr, graph, n_rows, n_tx)


def bce_loss(post, codewords):
    """Mean binary cross-entropy between sigma(-L) (P[bit = 1]) and the codeword bits."""
    import torch.nn.functional as F
    c = codewords[:, : post.shape[1]].float()
    return (F.softplus(-post) + c * post).mean()


def init_params(T: int, n_rows: int, beta: float = 0.75, gamma: float = 0.0):
    import torch
    p = torch.zeros((T, n_rows, 2), dtype=torch.float32, device="cuda")
    p[..., 0] = beta
    p[..., 1] = gamma
    return p


def train(graph: Graph, n_rows: int, T: int, batches, *, lr: float = 1e-3, params=None,
          log_every: int = 0):
    """Adam on the BCE loss over an iterable of (llr float CUDA [B][n_tx], codeword bits CUDA
    [B][N]) batches.  Returns (params, loss history)."""
    import torch
    p = init_params(T, n_rows) if params is None else params.clone()
    p.requires_grad_(True)
    opt = torch.optim.Adam([p], lr=lr)
    hist = []
    for k, (llr, cw) in enumerate(batches):
        opt.zero_grad(set_to_none=True)
        post = learned_decode(p, llr, graph, n_rows, llr.shape[1])
        loss = bce_loss(post, cw)
        loss.backward()
        opt.step()
        hist.append(float(loss.item()))
        if log_every and k % log_every == 0:
            print(f"step {k}: loss {hist[-1]:.5f}", flush=True)
    return p.detach(), np.array(hist)
