"""ctypes binding of libd2ip.so: one Python function per C entry point, same names.

Argument marshalling only: arrays may be torch tensors (device or host) or NumPy arrays
(host); they are passed as raw pointers.  A negative status raises ``D2IPError`` with the
library's message.  The library must have been built (``paper_2507_14046_gb300.build``);
importing this module without it raises at once -- there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libd2ip.so")

D2IP_FP32, D2IP_BF16, D2IP_BF16X3 = 0, 1, 2
KCLASSES = ("conv_fwd", "conv_dgrad", "conv_wgrad", "ln_fwd", "ln_bwd", "up_fwd", "up_bwd",
            "jmul", "loss", "jtmul", "adam", "misc")
STATUS = {0: "OK", -1: "BAD_ARG", -2: "BAD_SHAPE", -3: "OOM", -4: "NONFINITE", -5: "TIMEOUT",
          -6: "CUDA", -7: "STATE"}


class D2IPError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with `python -m "
                      "paper_2507_14046_gb300.build` (nvcc, sm_103a)")
_lib = C.CDLL(LIB_PATH)

_vp, _i, _ll, _f, _d, _cp = (C.c_void_p, C.c_int, C.c_longlong, C.c_float, C.c_double,
                            C.c_char_p)
_SIGS = {
    "d2ip_create": [C.POINTER(_vp), _i, _vp],
    "d2ip_destroy": [_vp],
    "d2ip_set_grid": [_vp, _i, _i, _i],
    "d2ip_set_network": [_vp, _i, _vp, _i, _i, _i],
    "d2ip_set_network_fastres": [_vp, _i, _vp, _i, _i, _i],
    "d2ip_wait_selftest": [_i, _ll, _i, C.POINTER(_i)],
    "d2ip_plan_param_table": [_i, _i, _i, _i, _i, _vp, _i, _vp, _i, C.POINTER(_i),
                              C.POINTER(_ll)],
    "d2ip_param_count": [_vp, C.POINTER(_ll)],
    "d2ip_param_table": [_vp, _vp, _i, C.POINTER(_i)],
    "d2ip_load_J": [_vp, _vp, _i, _i, _i],
    "d2ip_get_colnorms": [_vp, _vp],
    "d2ip_set_input": [_vp, _vp, _vp],
    "d2ip_set_optim": [_vp, _d, _d, _d, _d],
    "d2ip_reset_optimizer": [_vp],
    "d2ip_set_frame_reset": [_vp, _i],
    "d2ip_set_autotune": [_vp, _i],
    "d2ip_tile_plan": [_vp, _vp, _i, C.POINTER(_i), _vp],
    "d2ip_set_tile_plan": [_vp, _vp, _i],
    "d2ip_set_ln_backward_fusion": [_vp, _i],
    "d2ip_set_regularizer": [_vp, _d, _d, _d, _d],
    "d2ip_run_steps": [_vp, _vp, _i, _vp],
    "d2ip_forward": [_vp, _vp],
    "d2ip_get_grad": [_vp, _vp],
    "d2ip_fit_frame": [_vp, _vp, _i, _vp, _vp, _vp],
    "d2ip_fit_sequence": [_vp, _vp, _i, _vp, _i, _i, _i, _vp, _vp],
    "d2ip_fit_batched": [_vp, _i, _vp, _i, _vp, _i, _i, _i, _vp, _vp],
    "d2ip_get_state": [_vp, _vp, _vp, _vp, C.POINTER(_i)],
    "d2ip_set_state": [_vp, _vp, _vp, _vp, _i],
    "d2ip_err_ratio": [_vp, _vp, _vp, _vp],
    "d2ip_sync": [_vp],
    "d2ip_profile_iterations": [_vp, _vp, _i, _vp, _vp, _vp],
    "d2ip_graph_kernels": [_vp, _vp, _vp],
    "d2ip_conv3d_forward": [_vp, _vp, _vp, _vp, _i, _i, _i, _i, _i, _i, _i, _i, _ll, _vp],
    "d2ip_conv3d_dgrad": [_vp, _vp, _vp, _i, _i, _i, _i, _i, _i, _i, _i, _ll, _i, _vp],
    "d2ip_conv3d_wgrad": [_vp, _vp, _vp, _i, _i, _i, _i, _i, _i, _i, _i, _ll, _i, _vp, _ll,
                          _vp],
    "d2ip_conv3d_forward_tc": [_vp, _vp, _vp, _vp, _i, _i, _i, _i, _i, _i, _i, _i, _ll, _vp,
                               _ll, _vp],
    "d2ip_conv3d_dgrad_tc": [_vp, _vp, _vp, _i, _i, _i, _i, _i, _i, _i, _i, _ll, _i, _vp, _ll,
                             _vp],
    "d2ip_conv3d_wgrad_tc": [_vp, _vp, _vp, _i, _i, _i, _i, _i, _i, _i, _ll, _i, _vp, _ll,
                             _vp],
    "d2ip_conv3d_wgrad_noalloc": [_vp, _vp, _vp, _i, _i, _i, _i, _i, _i, _i, _i, _ll, _i,
                                  _vp],
    "d2ip_layernorm_act_forward": [_vp, _vp, _vp, _vp, _vp, _vp, _i, _ll, _i, _i, _ll, _vp],
    "d2ip_layernorm_act_backward": [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _i, _ll, _i, _ll,
                                    _i, _vp, _ll, _vp],
    "d2ip_upsample_concat_forward": [_vp, _vp, _vp, _i, _i, _i, _i, _i, _i, _i, _i, _i, _vp],
    "d2ip_upsample_concat_backward": [_vp, _vp, _vp, _i, _i, _i, _i, _i, _i, _i, _i, _i, _vp],
    "d2ip_sensitivity_residual": [_vp, _vp, _vp, _vp, _vp, _i, _i, _i, _vp, _ll, _vp],
    "d2ip_sensitivity_adjoint": [_vp, _vp, _vp, _f, _i, _i, _i, _vp],
    "d2ip_sensitivity_products_tc": [_vp, _vp, _vp, _vp, _vp, _f, _i, _i, _i, _i, _vp, _ll, _vp],
    "d2ip_normalize_columns": [_vp, _vp, _i, _i, _vp],
    "d2ip_tv4d": [_vp, _vp, _i, _vp, _vp, _i, _i, _i, _i, _d, _d, _d, _d, _vp, _ll, _vp],
    "d2ip_adam_update": [_vp, _vp, _vp, _vp, _ll, _d, _d, _d, _d, _i, _vp],
}
_SIZE_FNS = {
    "d2ip_conv3d_wgrad_workspace": [_i] * 8,
    "d2ip_conv3d_tc_workspace": [_i] * 8,
    "d2ip_conv3d_wgrad_tc_workspace": [_i] * 7,
    "d2ip_layernorm_workspace": [_i, _ll, _i],
    "d2ip_sensitivity_workspace": [_i, _i, _i],
    "d2ip_sensitivity_tc_workspace": [_i, _i, _i, _i],
    "d2ip_tv4d_workspace": [_i, _i, _i, _i],
}

for _name, _args in _SIGS.items():
    _fn = getattr(_lib, _name)
    _fn.argtypes = _args
    _fn.restype = _i
for _name, _args in _SIZE_FNS.items():
    _fn = getattr(_lib, _name)
    _fn.argtypes = _args
    _fn.restype = _ll
_lib.d2ip_last_error.argtypes = [_vp]
_lib.d2ip_last_error.restype = _cp


def exported_symbols() -> list[str]:
    return sorted(list(_SIGS) + list(_SIZE_FNS) + ["d2ip_last_error"])


def ptr(x):
    """Raw address of a torch tensor / NumPy array / int / None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("NumPy arrays passed to libd2ip must be C-contiguous")
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensors passed to libd2ip must be contiguous")
        return x.data_ptr()
    raise TypeError(f"cannot pass {type(x)} as a pointer")


def d2ip_last_error(ctx=None) -> str:
    return _lib.d2ip_last_error(ctx).decode()


def _call(name, ctx, *args):
    st = getattr(_lib, name)(*args)
    if st != 0:
        raise D2IPError(st, d2ip_last_error(ctx))
    return st


def _wrap_ctx(name):
    def f(ctx, *args):
        conv = [ptr(a) if not isinstance(a, (float, np.floating)) else a for a in args]
        return _call(name, ctx, ctx, *conv)
    f.__name__ = name
    return f


def _wrap_op(name):
    def f(*args):
        conv = [ptr(a) if not isinstance(a, (float, np.floating)) else a for a in args]
        return _call(name, None, *conv)
    f.__name__ = name
    return f


def d2ip_create(device: int = 0, stream=None):
    h = _vp()
    _call("d2ip_create", None, C.byref(h), device, ptr(stream))
    return h.value


def d2ip_destroy(ctx):
    return _lib.d2ip_destroy(ctx)


def d2ip_set_network(ctx, levels, widths, c_in, precision, batch):
    w = (C.c_int * levels)(*widths)
    return _call("d2ip_set_network", ctx, ctx, levels, C.cast(w, _vp), c_in, precision, batch)


def d2ip_set_network_fastres(ctx, levels, widths, c_in, precision, batch):
    w = (C.c_int * levels)(*widths)
    return _call("d2ip_set_network_fastres", ctx, ctx, levels, C.cast(w, _vp), c_in, precision,
                 batch)


def d2ip_plan_param_table(net, grid, levels, widths, c_in=8):
    """(rows [n, 4] int64, P) of a network's parameter table, without a context or device.
    net: "resunet" or "fastres"; grid (X, Y, Z)."""
    code = {"resunet": 0, "fastres": 1}[net]
    X, Y, Z = grid
    w = (C.c_int * levels)(*widths)
    n, P = _i(), _ll()
    _call("d2ip_plan_param_table", None, code, X, Y, Z, levels, C.cast(w, _vp), c_in, None, 0,
          C.byref(n), C.byref(P))
    rows = np.zeros((n.value, 4), dtype=np.int64)
    _call("d2ip_plan_param_table", None, code, X, Y, Z, levels, C.cast(w, _vp), c_in,
          rows.ctypes.data, n.value, C.byref(n), C.byref(P))
    return rows, P.value


def d2ip_wait_selftest(device=0, spin_limit=20000, set_flag=0):
    """Runs the bounded-wait self-test; returns the status word (raises D2IPError with
    D2IP_ERR_TIMEOUT when the wait ran out, as it does with set_flag=0)."""
    st = _i(-1)
    _call("d2ip_wait_selftest", None, device, spin_limit, set_flag, C.byref(st))
    return st.value


def d2ip_param_count(ctx) -> int:
    v = _ll()
    _call("d2ip_param_count", ctx, ctx, C.byref(v))
    return v.value


def d2ip_param_table(ctx) -> np.ndarray:
    n = _i()
    _call("d2ip_param_table", ctx, ctx, None, 0, C.byref(n))
    rows = np.zeros((n.value, 4), dtype=np.int64)
    _call("d2ip_param_table", ctx, ctx, rows.ctypes.data, n.value, C.byref(n))
    return rows


def d2ip_get_state(ctx, theta=None, adam_m=None, adam_v=None) -> int:
    t = _i()
    _call("d2ip_get_state", ctx, ctx, ptr(theta), ptr(adam_m), ptr(adam_v), C.byref(t))
    return t.value


def d2ip_tile_plan(ctx):
    """(rows [n, 15] int64, us [n, 4]) of the tensor-core tilings in use (see d2ip.h)."""
    n = _i()
    _call("d2ip_tile_plan", ctx, ctx, None, 0, C.byref(n), None)
    rows = np.zeros((n.value, 15), dtype=np.int64)
    us = np.zeros((n.value, 4), dtype=np.float64)
    _call("d2ip_tile_plan", ctx, ctx, rows.ctypes.data, n.value, C.byref(n), us.ctypes.data)
    return rows, us


def d2ip_set_tile_plan(ctx, rows):
    """Tilings saved from d2ip_tile_plan, applied when the workspace is built (see d2ip.h)."""
    r = np.ascontiguousarray(np.asarray(rows, dtype=np.int64).reshape(-1, 15))
    _call("d2ip_set_tile_plan", ctx, ctx, r.ctypes.data if r.size else None, r.shape[0])


def d2ip_conv3d_wgrad_workspace(*args) -> int:
    return int(_lib.d2ip_conv3d_wgrad_workspace(*args))


def d2ip_conv3d_tc_workspace(*args) -> int:
    return int(_lib.d2ip_conv3d_tc_workspace(*args))


def d2ip_conv3d_wgrad_tc_workspace(*args) -> int:
    return int(_lib.d2ip_conv3d_wgrad_tc_workspace(*args))


def d2ip_sensitivity_workspace(*args) -> int:
    return int(_lib.d2ip_sensitivity_workspace(*args))


def d2ip_sensitivity_tc_workspace(*args) -> int:
    return int(_lib.d2ip_sensitivity_tc_workspace(*args))


def d2ip_tv4d_workspace(*args) -> int:
    return int(_lib.d2ip_tv4d_workspace(*args))


def d2ip_layernorm_workspace(*args) -> int:
    return int(_lib.d2ip_layernorm_workspace(*args))


for _name in ("d2ip_set_grid", "d2ip_load_J", "d2ip_get_colnorms", "d2ip_set_input",
              "d2ip_set_optim", "d2ip_set_regularizer", "d2ip_reset_optimizer",
              "d2ip_set_frame_reset", "d2ip_set_autotune", "d2ip_set_ln_backward_fusion",
              "d2ip_run_steps", "d2ip_forward",
              "d2ip_get_grad", "d2ip_fit_frame", "d2ip_fit_sequence", "d2ip_set_state",
              "d2ip_err_ratio", "d2ip_sync", "d2ip_profile_iterations", "d2ip_graph_kernels"):
    globals()[_name] = _wrap_ctx(_name)
for _name in ("d2ip_conv3d_forward", "d2ip_conv3d_dgrad", "d2ip_conv3d_wgrad",
              "d2ip_conv3d_wgrad_noalloc", "d2ip_conv3d_forward_tc", "d2ip_conv3d_dgrad_tc",
              "d2ip_conv3d_wgrad_tc",
              "d2ip_layernorm_act_forward", "d2ip_layernorm_act_backward",
              "d2ip_upsample_concat_forward", "d2ip_upsample_concat_backward",
              "d2ip_sensitivity_residual", "d2ip_sensitivity_adjoint", "d2ip_normalize_columns",
              "d2ip_sensitivity_products_tc",
              "d2ip_tv4d",
              "d2ip_adam_update"):
    globals()[_name] = _wrap_op(_name)


def _ptr_array(items):
    arr = (_vp * len(items))(*[ptr(x) for x in items])
    return C.cast(arr, _vp), arr


def d2ip_fit_batched(ctxs, V, T, dV0, upws_steps, first_steps, later_steps, Sigma_out,
                     residual_out):
    """Lists of per-context handles and arrays (see d2ip.h)."""
    hc, keep1 = _ptr_array(ctxs)
    hv, keep2 = _ptr_array(V)
    hd, keep3 = _ptr_array(dV0) if dV0 is not None else (None, None)
    hs, keep4 = _ptr_array(Sigma_out) if Sigma_out is not None else (None, None)
    hr, keep5 = _ptr_array(residual_out) if residual_out is not None else (None, None)
    return _call("d2ip_fit_batched", ctxs[0], hc, len(ctxs), hv, T, hd, upws_steps,
                 first_steps, later_steps, hs, hr)


class Context:
    """Owns one d2ip_ctx (grid, network, J, batch of problems).  Methods forward to the C
    calls of the same name without the ``d2ip_`` prefix."""

    def __init__(self, grid, levels, widths, c_in=8, precision=D2IP_FP32, batch=1, device=0,
                 stream=None, net="resunet", autotune=True, tile_plan=None):
        """net: "resunet" (d2ip_set_network) or "fastres" (d2ip_set_network_fastres);
        autotune: time the tensor-core tilings when the workspace is built; tile_plan: rows
        saved from tile_plan() of a context of the same shape, applied instead of timing."""
        self.handle = d2ip_create(device, stream)
        if not autotune:
            d2ip_set_autotune(self.handle, 0)
        self.grid, self.batch, self.c_in = tuple(grid), batch, c_in
        X, Y, Z = grid
        d2ip_set_grid(self.handle, X, Y, Z)
        if net == "fastres":
            d2ip_set_network_fastres(self.handle, levels, list(widths), c_in, precision, batch)
        elif net == "resunet":
            d2ip_set_network(self.handle, levels, list(widths), c_in, precision, batch)
        else:
            raise ValueError(f"unknown network {net!r}")
        if tile_plan is not None:
            d2ip_set_tile_plan(self.handle, tile_plan)
        self.P = d2ip_param_count(self.handle)
        self.n = X * Y * Z
        self.m = 0

    def table(self):
        return d2ip_param_table(self.handle)

    def load_J(self, J, normalize=True):
        m, n = J.shape
        d2ip_load_J(self.handle, J, m, n, 1 if normalize else 0)
        self.m = m

    def colnorms(self):
        out = np.zeros(self.n, dtype=np.float64)
        d2ip_get_colnorms(self.handle, out)
        return out

    def set_input(self, Zin, theta0):
        d2ip_set_input(self.handle, Zin, theta0)

    def set_optim(self, lr, beta1=0.9, beta2=0.999, eps=1e-8):
        d2ip_set_optim(self.handle, float(lr), float(beta1), float(beta2), float(eps))

    def set_regularizer(self, lambda_tv=0.002, lambda_s=1.0, lambda_t=0.1, eps=1e-8):
        d2ip_set_regularizer(self.handle, float(lambda_tv), float(lambda_s), float(lambda_t),
                             float(eps))

    def tile_plan(self):
        return d2ip_tile_plan(self.handle)

    def set_tile_plan(self, rows):
        d2ip_set_tile_plan(self.handle, rows)

    def set_ln_backward_fusion(self, on: bool):
        d2ip_set_ln_backward_fusion(self.handle, 1 if on else 0)

    def set_frame_reset(self, reset_moments_per_frame: bool):
        d2ip_set_frame_reset(self.handle, 1 if reset_moments_per_frame else 0)

    def run_steps(self, dV, n_steps, trace=False):
        tr = np.zeros((n_steps, self.batch), dtype=np.float64) if trace else None
        d2ip_run_steps(self.handle, dV, n_steps, tr)
        return tr

    def forward(self):
        out = np.zeros((self.batch, self.n), dtype=np.float32)
        d2ip_forward(self.handle, out)
        return out

    def grad(self):
        out = np.zeros((self.batch, self.P), dtype=np.float32)
        d2ip_get_grad(self.handle, out)
        return out

    def state(self):
        th = np.zeros((self.batch, self.P), dtype=np.float32)
        m = np.zeros_like(th)
        v = np.zeros_like(th)
        t = d2ip_get_state(self.handle, th, m, v)
        return th, m, v, t

    def set_state(self, theta, m=None, v=None, t=0):
        d2ip_set_state(self.handle, theta, m, v, int(t))

    def fit_frame(self, dV, n_steps, trace=False):
        ds = np.zeros((self.batch, self.n), dtype=np.float32)
        res = np.zeros(self.batch, dtype=np.float64)
        tr = np.zeros((n_steps, self.batch), dtype=np.float64) if trace else None
        d2ip_fit_frame(self.handle, dV, n_steps, ds, res, tr)
        return ds, res, tr

    def fit_sequence(self, V, upws, first, later, dV0=None, Sigma=None, resid=None):
        T = V.shape[-2]
        if Sigma is None:
            Sigma = np.zeros((self.batch, T, self.n), dtype=np.float32)
        if resid is None:
            resid = np.zeros((self.batch, T), dtype=np.float64)
        d2ip_fit_sequence(self.handle, V, T, dV0, upws, first, later, Sigma, resid)
        return Sigma, resid

    def profile(self, dV, n_iters):
        """Per kernel class: (ms, work, launches) accumulated over n_iters eager iterations."""
        k = len(KCLASSES)
        ms, work = np.zeros(k), np.zeros(k)
        cnt = np.zeros(k, dtype=np.int64)
        d2ip_profile_iterations(self.handle, dV, n_iters, ms, work, cnt)
        return {name: (ms[i], work[i], int(cnt[i])) for i, name in enumerate(KCLASSES)}

    def graph_kernels(self):
        """Kernel launches of one training iteration and of one evaluation (graph nodes)."""
        st, ev = np.zeros(1, dtype=np.int64), np.zeros(1, dtype=np.int64)
        d2ip_graph_kernels(self.handle, st, ev)
        return int(st[0]), int(ev[0])

    def err_ratio(self, est, truth):
        out = np.zeros(self.batch, dtype=np.float64)
        d2ip_err_ratio(self.handle, est, truth, out)
        return out

    def close(self):
        if self.handle:
            d2ip_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
