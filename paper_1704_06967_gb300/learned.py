"""Learned inverse-depth proposal (include/pba_mlp.h): the network's
parameters as torch tensors and the calls that train it, run it and let it
initialise a bundle. Marshalling only: features, forward, backward, Adam and
inference run in libpba.so's kernels.

Training data come from the method itself: each generated bundle is solved
with IC from its usual initialisation, and the converged inverse depths are
the targets for the features taken at the bundle's initial poses.
"""
from __future__ import annotations

import ctypes
import math

import numpy as np

from .pba import PbaError, load

N_IN, N_HID = 96, 128
N_PARAMS = 45569
PACKED_BYTES = 92176
SHAPES = [("W1", (N_HID, N_IN)), ("b1", (N_HID,)), ("W2", (N_HID, N_HID)), ("b2", (N_HID,)),
          ("W3", (N_HID, N_HID)), ("b3", (N_HID,)), ("w4", (N_HID,)), ("b4", (1,))]


def _vp(t):
    return ctypes.c_void_p(t.data_ptr())


class DepthMLP:
    """The 96 -> 128 -> 128 -> 128 -> 1 proposal network on the GPU: FP32
    master parameters with Adam moments, and the packed BF16 inference copy."""

    def __init__(self, seed: int = 0, params: np.ndarray | None = None, stream=None):
        import torch
        self.torch = torch
        self.lib = load()
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        if params is None:
            params = self.initial_params(seed)
        self.params = torch.tensor(np.asarray(params, dtype=np.float32), device="cuda")
        assert self.params.numel() == N_PARAMS
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.step = 0
        self.packed = torch.empty(PACKED_BYTES, dtype=torch.uint8, device="cuda")
        self.flag = torch.zeros(4, dtype=torch.int32, device="cuda")
        self._packed_step = -1

    @staticmethod
    def initial_params(seed: int) -> np.ndarray:
        """He-style N(0, 2 / fan_in) weights, zero biases, b4 = 1 (the mean
        inverse depth of a normalised scene)."""
        rng = np.random.default_rng(seed)
        out = []
        for k, s in SHAPES:
            if k.startswith("W"):
                out.append(rng.normal(0.0, math.sqrt(2.0 / s[1]), size=s).ravel())
            elif k == "w4":
                out.append(rng.normal(0.0, math.sqrt(1.0 / s[0]), size=s).ravel())
            elif k == "b4":
                out.append(np.ones(1))
            else:
                out.append(np.zeros(s))
        return np.concatenate(out)

    def _st(self):
        return ctypes.c_void_p(self.stream.cuda_stream)

    def _check(self, st):
        if st != 0:
            raise PbaError(st, "learned proposal call failed")

    # ------------------------------------------------------------------
    def grad(self, X, T):
        """(loss sum, gradient) of a batch: torch CUDA float32 X [n, 96], T [n]."""
        torch = self.torch
        n = int(X.shape[0])
        scratch = torch.empty(int(self.lib.pba_mlp_scratch_floats(n)), dtype=torch.float32, device="cuda")
        g = torch.empty(N_PARAMS, dtype=torch.float32, device="cuda")
        loss = torch.empty(1, dtype=torch.float32, device="cuda")
        self._check(self.lib.pba_mlp_grad(_vp(self.params), n, _vp(X), _vp(T), _vp(g), _vp(loss), _vp(scratch),
                                          self._st()))
        return loss, g

    def train(self, X, T, epochs: int = 10, batch: int = 1024, lr: float = 1e-3, seed: int = 0):
        """Adam over shuffled minibatches; returns the mean loss per epoch."""
        torch = self.torch
        n = int(X.shape[0])
        scratch = torch.empty(int(self.lib.pba_mlp_scratch_floats(batch)), dtype=torch.float32, device="cuda")
        loss = torch.zeros(1, dtype=torch.float32, device="cuda")
        gen = torch.Generator(device="cpu").manual_seed(seed)
        history = []
        for _ in range(epochs):
            perm = torch.randperm(n, generator=gen).cuda()
            Xs, Ts = X[perm].contiguous(), T[perm].contiguous()
            tot = torch.zeros(1, dtype=torch.float64, device="cuda")
            for b0 in range(0, n - batch + 1, batch):
                self.step += 1
                self._check(self.lib.pba_mlp_train_step(
                    _vp(self.params), _vp(self.m), _vp(self.v), self.step, ctypes.c_float(lr), batch,
                    _vp(Xs[b0:]), _vp(Ts[b0:]), _vp(scratch), _vp(loss), self._st()))
                tot += loss.double()
            history.append(float(tot) / max(1, (n // batch) * batch))
        return history

    def pack(self):
        if self._packed_step != self.step:
            self._check(self.lib.pba_mlp_pack(_vp(self.params), _vp(self.packed), self._st()))
            self._packed_step = self.step
        return self.packed

    def infer(self, X):
        """Tensor-core inference: torch CUDA float32 [n] from X [n, 96]."""
        torch = self.torch
        n = int(X.shape[0])
        out = torch.empty(max(n, 1), dtype=torch.float32, device="cuda")
        self._check(self.lib.pba_mlp_infer(_vp(self.pack()), n, _vp(X), _vp(out), _vp(self.flag), self._st()))
        return out[:n]

    def propose(self, ctx, bundle: int = 0):
        """Sets the inverse depths of `bundle` of a Batch/Bundle to the proposals."""
        ctx.propose_depths(self.pack(), bundle)


def training_pairs(scene, iters: int = 20, stream=None, damping: float = 0.01, reanchor_every: int = 3, **kw):
    """(features at p_0, converged inverse depths, mask of usable points) of
    one generated bundle, or None when the method cannot solve it: the
    bundle is solved with IC (damped, re-anchored) from its own
    initialisation; points that no target frame observes, or whose converged
    inverse depth lies outside [0.05, 20], are not usable."""
    from .pba import Bundle
    b = Bundle.from_scene(scene, stream=stream, damping=damping, **kw)
    X = b.depth_features()
    try:
        b.solve_ic(iters, reanchor_every=reanchor_every, stats=False)
    except PbaError:
        b.close()
        return None  # a bundle the method cannot solve gives no targets
    _, d = b.params()
    b.close()
    # points no target frame observes, and converged values outside the
    # range a proposal can take (pba_propose_depths clamps to [0.05, 20]:
    # points the solve drove away), give no targets
    usable = (scene.vis[:, 1:].sum(1) > 0) & np.isfinite(d) & (d >= 0.05) & (d <= 20.0)
    return X, d, usable
