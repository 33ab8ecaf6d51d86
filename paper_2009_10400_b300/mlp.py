"""ctypes binding of the surrogate MLP in ``libtled`` (include/tled_mlp.h).

Marshalling only: the forward, backward and Adam passes run in the library's
tcgen05 kernels.  Tensors are PyTorch CUDA float32 tensors (row-major).
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from .tled import TledError, lib as _tled_lib

_SIGS = {
    "tled_mlp_create": ([C.POINTER(C.c_void_p), C.c_int, C.c_void_p, C.c_int32, C.POINTER(C.c_int32), C.c_int32],
                        C.c_int),
    "tled_mlp_destroy": ([C.c_void_p], C.c_int),
    "tled_mlp_last_error": ([C.c_void_p], C.c_char_p),
    "tled_mlp_num_params": ([C.c_void_p, C.POINTER(C.c_int64)], C.c_int),
    "tled_mlp_workspace_size": ([C.c_void_p, C.POINTER(C.c_int64)], C.c_int),
    "tled_mlp_init": ([C.c_void_p, C.c_void_p, C.c_int64], C.c_int),
    "tled_mlp_set_params": ([C.c_void_p, C.POINTER(C.c_float)], C.c_int),
    "tled_mlp_get_params": ([C.c_void_p, C.POINTER(C.c_float)], C.c_int),
    "tled_mlp_forward": ([C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p], C.c_int),
    "tled_mlp_gradients": ([C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p], C.c_int),
    "tled_mlp_train_step": ([C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_float, C.c_void_p], C.c_int),
    "tled_mlp_sync": ([C.c_void_p], C.c_int),
    "tled_mlp_set_stream": ([C.c_void_p, C.c_void_p], C.c_int),
    "tled_mlp_set_input_scaling": ([C.c_void_p, C.POINTER(C.c_float), C.POINTER(C.c_float)], C.c_int),
    "tled_mlp_train_step_rows": ([C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_float, C.c_void_p],
                                 C.c_int),
    "tled_mlp_ensemble": ([C.c_int, C.c_void_p, C.c_int32, C.POINTER(C.c_void_p), C.c_int32, C.c_int32, C.c_void_p,
                           C.c_void_p, C.c_void_p, C.c_int32, C.c_float, C.c_int32, C.c_void_p, C.c_int32, C.c_float,
                           C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
    "tled_sur_create": ([C.POINTER(C.c_void_p), C.c_int, C.c_void_p, C.c_int32, C.c_int32, C.c_int32, C.c_int32,
                         C.c_int32, C.c_int32, C.c_int32, C.c_int64, C.c_int32, C.c_int32, C.c_uint32, C.c_int32],
                        C.c_int),
    "tled_sur_set_symmetries": ([C.c_void_p, C.c_int32, C.POINTER(C.c_int32), C.POINTER(C.c_float),
                                 C.POINTER(C.c_float), C.POINTER(C.c_int32)], C.c_int),
    "tled_sur_destroy": ([C.c_void_p], C.c_int),
    "tled_sur_last_error": ([C.c_void_p], C.c_char_p),
    "tled_sur_workspace_size": ([C.c_void_p, C.POINTER(C.c_int64)], C.c_int),
    "tled_sur_init": ([C.c_void_p, C.c_void_p, C.c_int64], C.c_int),
    "tled_sur_set_inputs": ([C.c_void_p, C.POINTER(C.c_float), C.POINTER(C.c_float)], C.c_int),
    "tled_sur_set_outputs": ([C.c_void_p, C.c_int32, C.c_float, C.c_float, C.c_int32], C.c_int),
    "tled_sur_train": ([C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_int32, C.c_int32, C.c_float, C.c_float,
                        C.c_int32, C.c_uint64, C.POINTER(C.c_float)], C.c_int),
    "tled_sur_predict": ([C.c_void_p, C.c_void_p, C.c_int32, C.c_int32, C.c_float, C.c_void_p, C.c_void_p,
                          C.c_void_p, C.c_void_p], C.c_int),
    "tled_sur_calibrate": ([C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_int32, C.c_float, C.c_float,
                            C.POINTER(C.c_float), C.POINTER(C.c_float)], C.c_int),
    "tled_sur_spread_threshold": ([C.c_int64, C.POINTER(C.c_float), C.POINTER(C.c_float), C.c_float, C.c_float,
                                   C.POINTER(C.c_float), C.POINTER(C.c_float)], C.c_int),
    "tled_sur_member": ([C.c_void_p, C.c_int32, C.POINTER(C.c_void_p)], C.c_int),
    "tled_sur_sync": ([C.c_void_p], C.c_int),
}
_ready = False


def lib():
    global _ready
    L = _tled_lib()
    if not _ready:
        for name, (args, res) in _SIGS.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _ready = True
    return L


def exported_symbols():
    return list(_SIGS)


class MLP:
    """A network dims[0] -> dims[1] -> ... -> dims[-1] with GELU hidden layers."""

    def __init__(self, dims, max_batch, device=0, stream=None):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("the surrogate MLP needs a CUDA device; there is no CPU fallback")
        self._torch = torch
        self.dims = list(dims)
        self.device = device
        self.stream = stream if stream is not None else torch.cuda.current_stream(device)
        d = (C.c_int32 * len(dims))(*dims)
        h = C.c_void_p()
        rc = lib().tled_mlp_create(C.byref(h), device, C.c_void_p(self.stream.cuda_stream), len(dims) - 1, d,
                                   int(max_batch))
        if rc:
            raise TledError(rc, "invalid MLP dimensions (widths and outputs multiples of 128, batch of 128)")
        self.h = h
        n = C.c_int64()
        self._check(lib().tled_mlp_num_params(h, C.byref(n)))
        self.n_params = n.value
        self._check(lib().tled_mlp_workspace_size(h, C.byref(n)))
        self.ws = torch.empty(n.value + 256, dtype=torch.uint8, device=f"cuda:{device}")
        self._check(lib().tled_mlp_init(h, C.c_void_p((self.ws.data_ptr() + 255) & ~255), n.value))
        self.loss_buf = torch.zeros(1, dtype=torch.float32, device=f"cuda:{device}")

    def _check(self, rc):
        if rc:
            raise TledError(rc, lib().tled_mlp_last_error(self.h).decode())
        return rc

    def close(self):
        if getattr(self, "h", None):
            lib().tled_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, p):
        p = np.ascontiguousarray(p, np.float32)
        assert p.size == self.n_params
        self._check(lib().tled_mlp_set_params(self.h, p.ctypes.data_as(C.POINTER(C.c_float))))

    def get_params(self):
        p = np.empty(self.n_params, np.float32)
        self._check(lib().tled_mlp_get_params(self.h, p.ctypes.data_as(C.POINTER(C.c_float))))
        return p

    def forward(self, x, out=None):
        torch = self._torch
        B = x.shape[0]
        if out is None:
            out = torch.empty(B, self.dims[-1], dtype=torch.float32, device=x.device)
        self._check(lib().tled_mlp_forward(self.h, C.c_void_p(x.data_ptr()), B, C.c_void_p(out.data_ptr())))
        return out

    def gradients(self, x, t):
        torch = self._torch
        g = torch.empty(self.n_params, dtype=torch.float32, device=x.device)
        self._check(lib().tled_mlp_gradients(self.h, C.c_void_p(x.data_ptr()), C.c_void_p(t.data_ptr()), x.shape[0],
                                             C.c_void_p(g.data_ptr()), C.c_void_p(self.loss_buf.data_ptr())))
        return g, self.loss_buf

    def set_input_scaling(self, shift=None, scale=None):
        """Inputs enter the first layer as (x - shift) * scale (None: identity)."""
        if shift is None:
            self._check(lib().tled_mlp_set_input_scaling(self.h, None, None))
            return
        sh = np.ascontiguousarray(shift, np.float32)
        sc = np.ascontiguousarray(scale, np.float32)
        assert sh.size == self.dims[0] and sc.size == self.dims[0]
        fp = C.POINTER(C.c_float)
        self._check(lib().tled_mlp_set_input_scaling(self.h, sh.ctypes.data_as(fp), sc.ctypes.data_as(fp)))

    def train_step_rows(self, x, t, rows, lr):
        """Adam step on rows `rows` (device int32) of the device data set x, t."""
        assert rows.dtype == self._torch.int32 and rows.is_cuda
        self._check(lib().tled_mlp_train_step_rows(self.h, C.c_void_p(x.data_ptr()), C.c_void_p(t.data_ptr()),
                                                   C.c_void_p(rows.data_ptr()), rows.numel(), float(lr),
                                                   C.c_void_p(self.loss_buf.data_ptr())))
        return self.loss_buf

    def train_step(self, x, t, lr):
        self._check(lib().tled_mlp_train_step(self.h, C.c_void_p(x.data_ptr()), C.c_void_p(t.data_ptr()), x.shape[0],
                                              float(lr), C.c_void_p(self.loss_buf.data_ptr())))
        return self.loss_buf

    def sync(self):
        self._check(lib().tled_mlp_sync(self.h))

    def set_stream(self, stream):
        """Enqueue later work on `stream` (a torch.cuda.Stream of the same device)."""
        self.stream = stream
        self._check(lib().tled_mlp_set_stream(self.h, C.c_void_p(stream.cuda_stream)))


def ensemble(ys, out_scale=None, out_shift=None, n_spread=0, tol=0.0, device=0, stream=None, want_std=True,
             row_src=None, row_mult=1.0, n_row_scaled=0, out_offset=None):
    """Ensemble mean, std, spread and fallback flags of member outputs ys
    (list of device float32 tensors [B][n_out]) in the library's kernel.
    row_src: device float32 matrix whose column 0 (row stride = its width),
    times row_mult, scales the first n_row_scaled outputs of each row."""
    import torch

    B, n_out = ys[0].shape
    dev = ys[0].device
    stream = stream if stream is not None else torch.cuda.current_stream(dev)
    mean = torch.empty(B, n_out, dtype=torch.float32, device=dev)
    std = torch.empty(B, n_out, dtype=torch.float32, device=dev) if want_std else None
    spread = torch.empty(B, dtype=torch.float32, device=dev)
    fb = torch.empty(B, dtype=torch.uint8, device=dev)
    ptrs = (C.c_void_p * len(ys))(*[y.data_ptr() for y in ys])
    vp = lambda t: C.c_void_p(t.data_ptr()) if t is not None else None
    stride = row_src.stride(0) if row_src is not None else 1
    rc = lib().tled_mlp_ensemble(device, C.c_void_p(stream.cuda_stream), len(ys), ptrs, B, n_out, vp(out_scale),
                                 vp(out_shift), vp(row_src), int(stride), float(row_mult), int(n_row_scaled),
                                 vp(out_offset), int(n_spread), float(tol), vp(mean), vp(std), vp(spread), vp(fb))
    if rc:
        raise TledError(rc, "tled_mlp_ensemble: invalid arguments or CUDA error")
    return mean, std, spread, fb


def spread_threshold(spread, err, tol, coverage=1.0):
    """The library's calibration rule (tled_sur_spread_threshold) on host
    arrays: returns (tau, accepted fraction); tau = -1 if nothing qualifies."""
    sp = np.ascontiguousarray(spread, np.float32)
    er = np.ascontiguousarray(err, np.float32)
    tau, frac = C.c_float(), C.c_float()
    fp = C.POINTER(C.c_float)
    rc = lib().tled_sur_spread_threshold(sp.size, sp.ctypes.data_as(fp), er.ctypes.data_as(fp), float(tol),
                                         float(coverage), C.byref(tau), C.byref(frac))
    if rc:
        raise TledError(rc, "tled_sur_spread_threshold: invalid arguments")
    return float(tau.value), float(frac.value)


class SurrogateEngine:
    """ctypes handle of a tled_sur (an ensemble of MLPs with its data handling);
    tensors are PyTorch CUDA float32 (inputs, outputs) on the engine's device."""

    def __init__(self, dims, members, n_T, max_batch, max_rows, max_epochs, device=0, stream=None, n_freq=0,
                 enc_cols=(), max_sym=0):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("the surrogate needs a CUDA device; there is no CPU fallback")
        self._torch = torch
        self.dims, self.members, self.max_batch, self.device = list(dims), int(members), int(max_batch), device
        self.stream = stream if stream is not None else torch.cuda.current_stream(device)
        h = C.c_void_p()
        mask = sum(1 << int(j) for j in enc_cols)
        rc = lib().tled_sur_create(C.byref(h), device, C.c_void_p(self.stream.cuda_stream), self.members, dims[0],
                                   dims[1], len(dims) - 1, dims[-1], int(n_T), self.max_batch, int(max_rows),
                                   int(max_epochs), int(n_freq), mask, int(max_sym))
        self.n_feat = dims[0] + 2 * int(n_freq) * len(set(enc_cols))
        if rc:
            raise TledError(rc, "tled_sur_create: invalid sizes (widths and outputs multiples of 128, batch of 128)")
        self.h = h
        n = C.c_int64()
        self._check(lib().tled_sur_workspace_size(h, C.byref(n)))
        self.ws = torch.empty(n.value + 256, dtype=torch.uint8, device=f"cuda:{device}")
        self._check(lib().tled_sur_init(h, C.c_void_p((self.ws.data_ptr() + 255) & ~255), n.value))

    def _check(self, rc):
        if rc:
            raise TledError(rc, lib().tled_sur_last_error(self.h).decode())
        return rc

    def close(self):
        if getattr(self, "h", None):
            lib().tled_sur_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_inputs(self, lo, hi):
        fp = C.POINTER(C.c_float)
        lo = np.ascontiguousarray(lo, np.float32)
        hi = np.ascontiguousarray(hi, np.float32)
        self._check(lib().tled_sur_set_inputs(self.h, lo.ctypes.data_as(fp), hi.ctypes.data_as(fp)))

    def set_symmetries(self, src, a, b, perm):
        """src, a, b [n_sym][n_in] (x'_j = a x[src] + b), perm [n_sym][n_out] (y'_o = y[perm])."""
        src = np.ascontiguousarray(src, np.int32)
        a = np.ascontiguousarray(a, np.float32)
        b = np.ascontiguousarray(b, np.float32)
        perm = np.ascontiguousarray(perm, np.int32)
        ip, fp = C.POINTER(C.c_int32), C.POINTER(C.c_float)
        self._check(lib().tled_sur_set_symmetries(self.h, src.shape[0], src.ctypes.data_as(ip), a.ctypes.data_as(fp),
                                                  b.ctypes.data_as(fp), perm.ctypes.data_as(ip)))

    def set_outputs(self, power_col, power_ref, T_ref, norm):
        self._check(lib().tled_sur_set_outputs(self.h, int(power_col), float(power_ref), float(T_ref), int(norm)))

    def train(self, x, y, epochs, batch, lr, seed, lr_end=None, bootstrap=False):
        hist = np.zeros((self.members, epochs), np.float32)
        self._check(lib().tled_sur_train(self.h, C.c_void_p(x.data_ptr()), C.c_void_p(y.data_ptr()), x.shape[0],
                                         int(epochs), int(batch), float(lr), float(lr if lr_end is None else lr_end),
                                         int(bool(bootstrap)), int(seed), hist.ctypes.data_as(C.POINTER(C.c_float))))
        return hist

    def predict(self, x, n_spread, tol, mean=None, std=None, spread=None, fallback=None):
        vp = lambda t: C.c_void_p(t.data_ptr()) if t is not None else None
        self._check(lib().tled_sur_predict(self.h, C.c_void_p(x.data_ptr()), x.shape[0], int(n_spread), float(tol),
                                           vp(mean), vp(std), vp(spread), vp(fallback)))

    def calibrate(self, x, y, n_spread, tol, coverage):
        tau, frac = C.c_float(), C.c_float()
        self._check(lib().tled_sur_calibrate(self.h, C.c_void_p(x.data_ptr()), C.c_void_p(y.data_ptr()), x.shape[0],
                                             int(n_spread), float(tol), float(coverage), C.byref(tau),
                                             C.byref(frac)))
        return float(tau.value), float(frac.value)

    def member_params(self, k):
        m = C.c_void_p()
        self._check(lib().tled_sur_member(self.h, int(k), C.byref(m)))  # dims[0] = n_feat inputs
        n = C.c_int64()
        lib().tled_mlp_num_params(m, C.byref(n))
        p = np.empty(n.value, np.float32)
        if lib().tled_mlp_get_params(m, p.ctypes.data_as(C.POINTER(C.c_float))):
            raise TledError(-4, lib().tled_mlp_last_error(m).decode())
        return p

    def set_member_params(self, k, p):
        m = C.c_void_p()
        self._check(lib().tled_sur_member(self.h, int(k), C.byref(m)))
        p = np.ascontiguousarray(p, np.float32)
        if lib().tled_mlp_set_params(m, p.ctypes.data_as(C.POINTER(C.c_float))):
            raise TledError(-4, lib().tled_mlp_last_error(m).decode())

    def sync(self):
        self._check(lib().tled_sur_sync(self.h))
