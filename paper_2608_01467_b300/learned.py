"""Learned pruning at the checkpoint boundary (argument marshalling only).

Pipeline, every numeric step in libfeynsparse.so:
  1. log: an exact run with a fixed cut c1 = c2 (checkpoint table = the
     items) writes each checkpoint entry's exact subtree sum
     (fs_batch_log_subtrees) and its 16 features (fs_batch_features);
  2. train: Adam on mean((MLP(x) - log10 |subtree sum|)^2) with the library's
     tensor-core forward/backward kernels (fs_mlp_grad, fs_mlp_adam);
  3. prune: fs_batch_set_pruner attaches the trained parameters and a
     threshold tau; fs_batch_run cuts the entries the MLP scores below tau
     and enumerates the rest exactly.
PyTorch only holds device buffers and shuffles minibatch indices.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib
from ._lib import check
from .api import Batch, Circuit

N_PARAMS = _lib.MLP_PARAMS
TARGET_FLOOR = -12.0


def _vp(t):
    return ctypes.c_void_p(t.data_ptr())


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def forward(params: torch.Tensor, x: torch.Tensor) -> torch.Tensor:
    y = torch.empty(x.shape[0], dtype=torch.float32, device=x.device)
    check(_lib.load().fs_mlp_forward(_vp(params), _vp(x), x.shape[0], _vp(y), _stream()))
    return y


def grad(params: torch.Tensor, x: torch.Tensor, target: torch.Tensor):
    """(gradient [N_PARAMS], loss) of mean((MLP(x) - target)^2)."""
    g = torch.empty(N_PARAMS + 1, dtype=torch.float32, device=x.device)
    check(_lib.load().fs_mlp_grad(_vp(params), _vp(x), _vp(target), x.shape[0], _vp(g), _stream()))
    return g[:N_PARAMS], g[N_PARAMS]


def adam_step(params, m, v, g, lr: float, step: int):
    check(_lib.load().fs_mlp_adam(_vp(params), _vp(m), _vp(v), _vp(g), float(lr), int(step), _stream()))


def subtree_targets(log_sums: torch.Tensor) -> torch.Tensor:
    """max(log10 |S|, TARGET_FLOOR) of complex subtree sums (re, im pairs),
    computed by the library (fs_mlp_targets)."""
    sums = log_sums.contiguous()
    t = torch.empty(sums.shape[0], dtype=torch.float32, device=sums.device)
    check(_lib.load().fs_mlp_targets(_vp(sums), sums.shape[0], TARGET_FLOOR, _vp(t), _stream()))
    return t


def table_data(circuit, inputs, outputs, cut: int, device="cuda"):
    """Features [entries, 16] (NaN in column 0 for bottom entries) and exact
    subtree sums [entries, 2] (re, im) of the whole checkpoint table after
    the first `cut` gates in evaluation order, in table order
    (entry = ((output * S + input) << A_p) | h_p), and the run's stats."""
    C = Circuit(circuit)
    C.set_input(inputs)
    b = Batch(split="fixed", c1=cut, c2=cut)
    b.add(C, outputs, 0.0)
    b.plan()
    items = ctypes.c_uint64()
    check(_lib.load().fs_batch_log_items(b._h, 0, ctypes.byref(items)))
    log = torch.zeros((items.value, 2), dtype=torch.float64, device=device)
    check(_lib.load().fs_batch_log_subtrees(b._h, 0, ctypes.c_void_p(log.data_ptr())))
    b.allocate(device)
    b.upload()
    b.run()
    st = b.finish()
    feat = torch.empty((items.value, 16), dtype=torch.float32, device=device)
    check(_lib.load().fs_batch_features(b._h, 0, ctypes.c_void_p(b.ws_ptr), _vp(feat), _stream()))
    torch.cuda.synchronize()
    return feat, log, st[0]


def log_training_data(circuit, inputs, outputs, cut: int, device="cuda"):
    """Features and exact log10 |subtree sum| of every live checkpoint entry
    after the first `cut` gates in evaluation order (output-to-input)."""
    feat, log, st = table_data(circuit, inputs, outputs, cut, device)
    live = ~torch.isnan(feat[:, 0])
    return feat[live].contiguous(), subtree_targets(log[live]).contiguous(), st


def train(x: torch.Tensor, t: torch.Tensor, init: np.ndarray, steps: int = 400, batch: int = 4096,
          lr: float = 2e-3, seed: int = 0):
    """Adam training on the GPU; returns (params, loss history)."""
    dev = x.device
    p = torch.from_numpy(np.asarray(init, np.float32)).to(dev).contiguous()
    m = torch.zeros_like(p)
    v = torch.zeros_like(p)
    gen = torch.Generator(device="cpu").manual_seed(seed)
    n = x.shape[0]
    losses = []
    for step in range(1, steps + 1):
        idx = torch.randint(0, n, (min(batch, n),), generator=gen).to(dev)
        xb = x.index_select(0, idx).contiguous()
        tb = t.index_select(0, idx).contiguous()
        g, loss = grad(p, xb, tb)
        adam_step(p, m, v, g, lr, step)
        if step % 50 == 0 or step == steps:
            losses.append(float(loss))
    return p, losses


def attach(batch: Batch, job: int, params: torch.Tensor, tau: float):
    """The library reads the parameters at every run: the batch keeps a
    reference so that the device buffer outlives it."""
    check(_lib.load().fs_batch_set_pruner(batch._h, job, _vp(params), float(tau)))
    if not hasattr(batch, "_pruner_params"):
        batch._pruner_params = {}
    batch._pruner_params[job] = params
