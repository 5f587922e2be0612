"""Python front end of the MLP surrogate entry points (argument marshalling).

Device memory comes from PyTorch tensors; every computation runs in the
library's kernels (include/ofmlmc.h, MLP section).
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import native as nv


def _ptr(t):
    return C.c_void_p(t.data_ptr())


def _stream():
    import torch
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


class MLP:
    def __init__(self, d_in: int, hidden: int = 256, n_hidden: int = 3, d_out: int = 1, max_rows: int = 4096):
        import torch
        self.d_in, self.hidden, self.n_hidden, self.d_out, self.max_rows = d_in, hidden, n_hidden, d_out, max_rows
        nbytes = C.c_size_t()
        L = nv.lib()
        nv.check(L.ofm_mlp_workspace_bytes(d_in, hidden, n_hidden, d_out, max_rows, C.byref(nbytes)),
                 "ofm_mlp_workspace_bytes")
        self.ws = torch.empty(nbytes.value + 256, dtype=torch.uint8, device="cuda")
        base = (self.ws.data_ptr() + 255) // 256 * 256
        h = C.c_void_p()
        nv.check(L.ofm_mlp_create(C.byref(h), d_in, hidden, n_hidden, d_out, max_rows, C.c_void_p(base),
                                  nbytes.value), "ofm_mlp_create")
        self.h = h
        n = C.c_int64()
        nv.check(L.ofm_mlp_param_count(h, C.byref(n)), "ofm_mlp_param_count")
        self.n_params = n.value

    @property
    def sizes(self):
        return [self.d_in] + [self.hidden] * self.n_hidden + [self.d_out]

    def set_params(self, vec: np.ndarray):
        v = np.ascontiguousarray(vec, dtype=np.float32)
        assert v.size == self.n_params
        nv.check(nv.lib().ofm_mlp_set_params(self.h, v.ctypes.data_as(C.POINTER(C.c_float))), "ofm_mlp_set_params")

    def get_params(self) -> np.ndarray:
        v = np.empty(self.n_params, dtype=np.float32)
        nv.check(nv.lib().ofm_mlp_get_params(self.h, v.ctypes.data_as(C.POINTER(C.c_float))), "ofm_mlp_get_params")
        return v

    def set_scaling(self, x_mean, x_std, y_mean, y_std):
        arrs = [np.ascontiguousarray(a, dtype=np.float32) for a in (x_mean, x_std, y_mean, y_std)]
        p = [a.ctypes.data_as(C.POINTER(C.c_float)) for a in arrs]
        nv.check(nv.lib().ofm_mlp_set_scaling(self.h, *p), "ofm_mlp_set_scaling")

    def forward(self, X):
        import torch
        Y = torch.empty((X.shape[0], self.d_out), dtype=torch.float32, device="cuda")
        nv.check(nv.lib().ofm_mlp_forward(self.h, _ptr(X), X.shape[0], _ptr(Y), _stream()), "ofm_mlp_forward")
        return Y

    def gradients(self, X, T):
        g = np.empty(self.n_params, dtype=np.float32)
        loss = C.c_float()
        nv.check(nv.lib().ofm_mlp_gradients(self.h, _ptr(X), _ptr(T), X.shape[0],
                                            g.ctypes.data_as(C.POINTER(C.c_float)), C.byref(loss), _stream()),
                 "ofm_mlp_gradients")
        return g, loss.value

    def train(self, X, T, steps: int, lr: float = 1e-3) -> np.ndarray:
        hist = np.empty(max(steps, 1), dtype=np.float32)
        nv.check(nv.lib().ofm_mlp_train(self.h, _ptr(X), _ptr(T), X.shape[0], steps, lr,
                                        hist.ctypes.data_as(C.POINTER(C.c_float)), _stream()), "ofm_mlp_train")
        return hist[:steps]

    def close(self):
        if getattr(self, "h", None):
            nv.lib().ofm_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()


def column_moments(X):
    import torch
    rows, cols = X.shape
    mean = torch.empty(cols, dtype=torch.float64, device="cuda")
    std = torch.empty(cols, dtype=torch.float64, device="cuda")
    nv.check(nv.lib().ofm_column_moments(_ptr(X), rows, cols, _ptr(mean), _ptr(std), _stream()), "ofm_column_moments")
    return mean, std


def cloud_features(bubbles_dev, n_bubbles: int, domain_L: float, scale: float, n_keep: int = 0):
    """bubbles_dev: (n_clouds, n_bubbles, 4) float64 CUDA tensor in metres; features of the
    n_keep bubbles nearest the centre (0: all)."""
    import torch
    n = bubbles_dev.shape[0]
    k = n_bubbles if n_keep <= 0 else n_keep
    X = torch.empty((n, 4 * k), dtype=torch.float32, device="cuda")
    nv.check(nv.lib().ofm_cloud_features(_ptr(bubbles_dev), n, n_bubbles, n_keep, domain_L, scale, _ptr(X),
                                         _stream()), "ofm_cloud_features")
    return X


def surrogate_cv(D, s_paired, s_extra):
    D = np.ascontiguousarray(D, dtype=np.float64)
    sp = np.ascontiguousarray(s_paired, dtype=np.float64)
    se = np.ascontiguousarray(s_extra, dtype=np.float64)
    b, m, v = C.c_double(), C.c_double(), C.c_double()
    dp = lambda a: a.ctypes.data_as(C.POINTER(C.c_double))
    nv.check(nv.lib().ofm_surrogate_cv(dp(D), dp(sp), D.size, dp(se), se.size, C.byref(b), C.byref(m), C.byref(v)),
             "ofm_surrogate_cv")
    return dict(beta=b.value, mean=m.value, var=v.value)
