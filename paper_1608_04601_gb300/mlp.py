"""Python binding of the warm-start network (include/mlp.h): argument marshalling only.

Inputs and outputs are CUDA tensors (float32, row-major); every product, loss and update runs in
the library's kernels.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _native as NV


def _dev(t, cols=None):
    import torch
    if not isinstance(t, torch.Tensor):
        t = torch.as_tensor(np.ascontiguousarray(t, np.float32))
    t = t.to(device="cuda", dtype=torch.float32).contiguous()
    if cols is not None:
        assert t.dim() == 2 and t.shape[1] == cols, (tuple(t.shape), cols)
    return t


class MLP:
    """sizes = [inputs, hidden..., outputs]; tanh hidden layers, linear output; BF16 weights."""

    def __init__(self, sizes, max_batch: int = 256, seed: int = 1, stream=None):
        import torch
        self.L = NV.lib()
        self.sizes = [int(s) for s in sizes]
        arr = (C.c_int32 * len(self.sizes))(*self.sizes)
        st = torch.cuda.current_stream().cuda_stream if stream == "torch" else stream
        h = C.c_void_p()
        s = self.L.mlp_create(C.byref(h), len(self.sizes) - 1, arr, int(max_batch), int(seed),
                              C.c_void_p(st) if st else None)
        if s != NV.PIC_OK:
            raise NV.PicError(s, "mlp_create")
        self.h = h
        self.max_batch = int(max_batch)
        self.n_params = int(self.L.mlp_param_count(h))
        self._loss = torch.zeros(1, dtype=torch.float32, device="cuda")

    def _ck(self, s):
        if s != NV.PIC_OK:
            m = self.L.mlp_last_error(self.h)
            raise NV.PicError(s, m.decode() if m else "")

    def close(self):
        if getattr(self, "h", None):
            self.L.mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()

    def get_params(self) -> np.ndarray:
        out = np.zeros(self.n_params, np.float32)
        self._ck(self.L.mlp_get_params(self.h, out.ctypes.data))
        return out

    def set_params(self, p):
        a = np.ascontiguousarray(p, np.float32)
        assert a.size == self.n_params
        self._ck(self.L.mlp_set_params(self.h, a.ctypes.data))

    def forward(self, x):
        import torch
        x = _dev(x, self.sizes[0])
        y = torch.empty((x.shape[0], self.sizes[-1]), dtype=torch.float32, device="cuda")
        self._ck(self.L.mlp_forward(self.h, x.shape[0], x.data_ptr(), y.data_ptr()))
        self._ck(self.L.mlp_sync(self.h))
        return y

    def loss_grad(self, x, t) -> float:
        x, t = _dev(x, self.sizes[0]), _dev(t, self.sizes[-1])
        self._ck(self.L.mlp_loss_grad(self.h, x.shape[0], x.data_ptr(), t.data_ptr(), self._loss.data_ptr()))
        self._ck(self.L.mlp_sync(self.h))
        return float(self._loss.item())

    def grads(self) -> np.ndarray:
        out = np.zeros(self.n_params, np.float32)
        self._ck(self.L.mlp_get_grads(self.h, out.ctypes.data))
        return out

    def adam(self, lr: float, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8):
        self._ck(self.L.mlp_adam(self.h, lr, beta1, beta2, eps))

    def train_step(self, x, t, lr: float, sync: bool = True):
        """One Adam step on the batch (x, t); returns the loss before the step when sync."""
        self._ck(self.L.mlp_train_step(self.h, x.shape[0], x.data_ptr(), t.data_ptr(), float(lr),
                                       self._loss.data_ptr()))
        if sync:
            self._ck(self.L.mlp_sync(self.h))
            return float(self._loss.item())
        return None
