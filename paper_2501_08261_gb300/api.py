"""Thin ctypes binding of include/lisa_td.h (argument marshalling only).

Every function has the C entry point's name and forwards device pointers
(``tensor.data_ptr()``) and the CUDA stream handle; all arithmetic runs in the
CUDA library.  If the library is missing, importing this module raises: there
is no CPU fallback.
"""
import ctypes
import os

from . import build as _build

LISA_TD_OK = 0
ERRORS = {-1: "EINVAL", -2: "ENOMEM", -3: "ECUDA", -4: "ETIMEOUT", -5: "ERANGE"}
EXPORTS = ("lisa_td_create", "lisa_td_create_orbits", "lisa_td_set_data", "lisa_td_waveform", "lisa_td_project",
           "lisa_td_tdi", "lisa_td_loglike_batch", "lisa_td_profile", "lisa_td_profile_read",
           "lisa_td_destroy", "lisa_td_last_error", "lisa_td_residual_loglike_noalloc",
           "lisa_td_fp32_fma_rate", "lisa_td_het_setup", "lisa_td_het_loglike",
           "lisa_td_het_deltas", "lisa_td_het_aet",
           "lisa_td_loglike_ragged", "lisa_td_ragged_graph", "lisa_td_autotune", "lisa_td_noise",
           "lisa_fisher_npoints", "lisa_fisher_points", "lisa_fisher_assemble", "lisa_cholesky",
           "lisa_gauss_draw", "lisa_gauss_logq", "lisa_gauss_walk", "lisa_mh_accept", "lisa_pt_swap",
           "flow_create", "flow_set_wait_limit", "flow_nparams", "flow_set_params", "flow_get_params", "flow_set_frame",
           "flow_logprob", "flow_propose", "flow_grad", "flow_adam", "flow_train", "flow_destroy")
NSTAGE = 7
STAGES = ("prep", "waveform", "project", "tdi", "fft_pass1", "fft_pass2_norm", "reduce")


class Config(ctypes.Structure):
    """Mirror of lisa_td_config."""
    _fields_ = [("dt", ctypes.c_double), ("n", ctypes.c_int64), ("t0", ctypes.c_double),
                ("f_lo", ctypes.c_double), ("f_hi", ctypes.c_double),
                ("tdi_gen", ctypes.c_int32), ("channel_mask", ctypes.c_int32),
                ("lagrange_order", ctypes.c_int32), ("orbit_kind", ctypes.c_int32),
                ("mode_mask", ctypes.c_int32), ("precessing", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("max_walkers", ctypes.c_int32),
                ("tdi_nested", ctypes.c_int32)]


class OrbitTable(ctypes.Structure):
    """Mirror of lisa_td_orbit_table."""
    _fields_ = [("t0", ctypes.c_double), ("dt", ctypes.c_double), ("rows", ctypes.c_int64),
                ("pos_host", ctypes.c_void_p)]


def load_library(path=None):
    path = path or _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library {path} is missing: run paper_2501_08261_gb300.build "
                           "(there is no CPU fallback)")
    lib = ctypes.CDLL(path)
    P, I32, I64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    sig = {
        "lisa_td_create": ([ctypes.POINTER(P), ctypes.POINTER(Config), P], ctypes.c_int),
        "lisa_td_create_orbits": ([ctypes.POINTER(P), ctypes.POINTER(Config),
                                   ctypes.POINTER(OrbitTable), P], ctypes.c_int),
        "lisa_td_set_data": ([P, P, P], ctypes.c_int),
        "lisa_td_waveform": ([P, P, I32, P, P], ctypes.c_int),
        "lisa_td_project": ([P, P, I32, P, P], ctypes.c_int),
        "lisa_td_tdi": ([P, P, I32, P, P], ctypes.c_int),
        "lisa_td_loglike_batch": ([P, P, I32, P, P, P], ctypes.c_int),
        "lisa_td_loglike_ragged": ([P, P, I32, P, P, P, P], ctypes.c_int),
        "lisa_td_ragged_graph": ([P, I32], ctypes.c_int),
        "lisa_td_autotune": ([P, P, I32, P, P, P], ctypes.c_int),
        "lisa_td_noise": ([P, P, P, P], ctypes.c_int),
        "lisa_td_profile": ([P, I32], ctypes.c_int),
        "lisa_td_profile_read": ([P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(I64)],
                                 ctypes.c_int),
        "lisa_td_residual_loglike_noalloc": ([ctypes.POINTER(Config), P, I32, P, P], ctypes.c_int),
        "lisa_td_fp32_fma_rate": ([ctypes.POINTER(ctypes.c_double), P], ctypes.c_int),
        "lisa_td_het_setup": ([P, P, P, I64, P], ctypes.c_int),
        "lisa_td_het_loglike": ([P, P, I32, P, P, P], ctypes.c_int),
        "lisa_td_het_deltas": ([P, P, I32, P, P], ctypes.c_int),
        "lisa_td_het_aet": ([P, P, I32, P, P], ctypes.c_int),
        "lisa_fisher_npoints": ([I32], ctypes.c_int),
        "lisa_fisher_points": ([P, P, P, I32, P, P], ctypes.c_int),
        "lisa_fisher_assemble": ([P, P, I32, P, P], ctypes.c_int),
        "lisa_cholesky": ([P, P, I32, P, P, P], ctypes.c_int),
        "lisa_gauss_draw": ([P, P, P, I32, P, I32, P, P, P], ctypes.c_int),
        "lisa_gauss_logq": ([P, P, P, I32, P, I32, P, P], ctypes.c_int),
        "lisa_gauss_walk": ([P, P, P, I32, P, I32, ctypes.c_double, P, P], ctypes.c_int),
        "lisa_mh_accept": ([I32, P, P, P, P, P, P, P, P, P, P, P, P], ctypes.c_int),
        "lisa_pt_swap": ([I32, I32, P, P, P, P, P, P, P], ctypes.c_int),
        "flow_create": ([ctypes.POINTER(P), I32, I32, I32, I32, P, P, P], ctypes.c_int),
        "flow_nparams": ([P, ctypes.POINTER(I64)], ctypes.c_int),
        "flow_set_wait_limit": ([P, I64], ctypes.c_int),
        "flow_set_params": ([P, P, P], ctypes.c_int),
        "flow_get_params": ([P, P, P], ctypes.c_int),
        "flow_set_frame": ([P, P, P, P], ctypes.c_int),
        "flow_logprob": ([P, P, I32, P, P], ctypes.c_int),
        "flow_propose": ([P, P, I32, P, P, P], ctypes.c_int),
        "flow_grad": ([P, P, I32, P, P, P], ctypes.c_int),
        "flow_adam": ([P, P, ctypes.c_float, P], ctypes.c_int),
        "flow_train": ([P, P, I64, I32, I32, ctypes.c_float, P, P], ctypes.c_int),
        "flow_destroy": ([P], None),
        "lisa_td_destroy": ([P], None),
        "lisa_td_last_error": ([], ctypes.c_char_p),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    return lib


_LIB = None


def lib():
    global _LIB
    if _LIB is None:
        _LIB = load_library()
    return _LIB


class LisaTdError(RuntimeError):
    pass


def _check(rc, what):
    if rc != LISA_TD_OK:
        msg = lib().lisa_td_last_error().decode(errors="replace")
        raise LisaTdError(f"{what} -> {ERRORS.get(rc, rc)}: {msg}")


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(getattr(stream, "cuda_stream", stream))


def make_config(dt, n, t0=0.0, f_lo=1e-4, f_hi=0.02, tdi_gen=15, channel_mask=7,
                lagrange_order=31, orbit=0, mode_mask=1, precessing=0, precision=0,
                max_walkers=32, tdi_nested=0):
    return Config(float(dt), int(n), float(t0), float(f_lo), float(f_hi), int(tdi_gen),
                  int(channel_mask), int(lagrange_order), int(orbit), int(mode_mask),
                  int(precessing), int(precision), int(max_walkers), int(tdi_nested))


def lisa_td_create(cfg, stream=None):
    h = ctypes.c_void_p()
    _check(lib().lisa_td_create(ctypes.byref(h), ctypes.byref(cfg), _stream(stream)),
           "lisa_td_create")
    return h


def lisa_td_create_orbits(cfg, t0, dt, pos, stream=None):
    """Context on the caller's spacecraft positions pos [rows][3][3] (metres,
    host array), row j at time t0 + j dt (orbit_kind 2)."""
    import numpy as np
    arr = np.ascontiguousarray(pos, dtype=np.float64)
    if arr.ndim != 3 or arr.shape[1:] != (3, 3):
        raise ValueError(f"orbit table: shape {arr.shape}, expected (rows, 3, 3)")
    tab = OrbitTable(float(t0), float(dt), int(arr.shape[0]), arr.ctypes.data)
    h = ctypes.c_void_p()
    _check(lib().lisa_td_create_orbits(ctypes.byref(h), ctypes.byref(cfg), ctypes.byref(tab),
                                       _stream(stream)), "lisa_td_create_orbits")
    return h


def lisa_td_set_data(ctx, aet, stream=None):
    _check(lib().lisa_td_set_data(ctx, _ptr(aet), _stream(stream)), "lisa_td_set_data")


def lisa_td_waveform(ctx, params, W, h, stream=None):
    _check(lib().lisa_td_waveform(ctx, _ptr(params), int(W), _ptr(h), _stream(stream)),
           "lisa_td_waveform")


def lisa_td_project(ctx, params, W, y, stream=None):
    _check(lib().lisa_td_project(ctx, _ptr(params), int(W), _ptr(y), _stream(stream)),
           "lisa_td_project")


def lisa_td_tdi(ctx, y, W, aet, stream=None):
    _check(lib().lisa_td_tdi(ctx, _ptr(y), int(W), _ptr(aet), _stream(stream)), "lisa_td_tdi")


def lisa_td_loglike_batch(ctx, params, W, logl, status=None, stream=None):
    _check(lib().lisa_td_loglike_batch(ctx, _ptr(params), int(W), _ptr(logl), _ptr(status),
                                       _stream(stream)), "lisa_td_loglike_batch")


def lisa_td_het_setup(ctx, theta0, nodes, stream=None):
    """Heterodyned likelihood set-up: fiducial theta0 [15] and node indices
    (host arrays)."""
    import numpy as np
    th = np.ascontiguousarray(theta0, dtype=np.float64).reshape(-1)
    nd = np.ascontiguousarray(nodes, dtype=np.int64).reshape(-1)
    if th.size != 15:
        raise ValueError("theta0 must hold 15 parameters")
    _check(lib().lisa_td_het_setup(ctx, th.ctypes.data_as(ctypes.c_void_p),
                                   nd.ctypes.data_as(ctypes.c_void_p), int(nd.size),
                                   _stream(stream)), "lisa_td_het_setup")


def lisa_td_het_loglike(ctx, params, W, logl, status=None, stream=None):
    _check(lib().lisa_td_het_loglike(ctx, _ptr(params), int(W), _ptr(logl), _ptr(status),
                                     _stream(stream)), "lisa_td_het_loglike")


def lisa_td_het_deltas(ctx, params, W, dz, stream=None):
    _check(lib().lisa_td_het_deltas(ctx, _ptr(params), int(W), _ptr(dz), _stream(stream)),
           "lisa_td_het_deltas")


def lisa_td_het_aet(ctx, params, W, aet, stream=None):
    _check(lib().lisa_td_het_aet(ctx, _ptr(params), int(W), _ptr(aet), _stream(stream)),
           "lisa_td_het_aet")


def lisa_td_loglike_ragged(ctx, params, W, n_per_walker, logl, status=None, stream=None):
    import numpy as np
    nh = np.ascontiguousarray(n_per_walker, dtype=np.int64)
    _check(lib().lisa_td_loglike_ragged(ctx, _ptr(params), int(W),
                                        nh.ctypes.data_as(ctypes.c_void_p), _ptr(logl),
                                        _ptr(status), _stream(stream)), "lisa_td_loglike_ragged")


def lisa_td_autotune(ctx, params, W, n_per_walker=None, stream=None):
    """-> (tile, warps, pass-1 pb, pass-2 pb, pass-1 threads, pass-2 threads)
    chosen and kept by the context."""
    import numpy as np
    ch = (ctypes.c_int32 * 6)()
    if n_per_walker is None:
        nh = None
    else:
        nh_arr = np.ascontiguousarray(n_per_walker, dtype=np.int64)
        nh = nh_arr.ctypes.data_as(ctypes.c_void_p)
    _check(lib().lisa_td_autotune(ctx, _ptr(params), int(W), nh, ch, _stream(stream)),
           "lisa_td_autotune")
    return tuple(ch)


def lisa_td_noise(ctx, z, noise, stream=None):
    _check(lib().lisa_td_noise(ctx, _ptr(z), _ptr(noise), _stream(stream)), "lisa_td_noise")


def lisa_td_ragged_graph(ctx, enable):
    _check(lib().lisa_td_ragged_graph(ctx, int(enable)), "lisa_td_ragged_graph")


def lisa_td_profile(ctx, enable):
    _check(lib().lisa_td_profile(ctx, int(enable)), "lisa_td_profile")


def lisa_td_profile_read(ctx):
    """-> (dict stage -> summed ms, number of timed calls)"""
    arr = (ctypes.c_double * NSTAGE)()
    calls = ctypes.c_int64()
    _check(lib().lisa_td_profile_read(ctx, arr, ctypes.byref(calls)), "lisa_td_profile_read")
    return dict(zip(STAGES, list(arr))), calls.value


def lisa_td_residual_loglike_noalloc(cfg, r, W, logl, stream=None):
    """-1/2 sum_c (r_c | r_c) per walker from caller-supplied residual series
    r [3][n][W] (W even) with scratch in the library's static device array:
    for callers that must not allocate device memory (see include/lisa_td.h)."""
    _check(lib().lisa_td_residual_loglike_noalloc(ctypes.byref(cfg), _ptr(r), int(W), _ptr(logl),
                                                  _stream(stream)),
           "lisa_td_residual_loglike_noalloc")


def lisa_td_fp32_fma_rate(stream=None):
    """-> the device's FP32 FMA rate in TFLOP/s (measured on the stream)."""
    v = ctypes.c_double()
    _check(lib().lisa_td_fp32_fma_rate(ctypes.byref(v), _stream(stream)), "lisa_td_fp32_fma_rate")
    return v.value


def _host_i32(a):
    import numpy as np
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a, a.ctypes.data_as(ctypes.c_void_p)


def _host_f64(a):
    import numpy as np
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(ctypes.c_void_p)


def lisa_fisher_npoints(D):
    return int(lib().lisa_fisher_npoints(int(D)))


def lisa_fisher_points(theta0, idx, eps, points, stream=None):
    (ia, ip), (ea, ep) = _host_i32(idx), _host_f64(eps)
    _check(lib().lisa_fisher_points(_ptr(theta0), ip, ep, len(ia), _ptr(points), _stream(stream)),
           "lisa_fisher_points")


def lisa_fisher_assemble(logl, eps, fisher, stream=None):
    ea, ep = _host_f64(eps)
    _check(lib().lisa_fisher_assemble(_ptr(logl), ep, len(ea), _ptr(fisher), _stream(stream)),
           "lisa_fisher_assemble")


def lisa_cholesky(a, D, l, info, diag=None, stream=None):
    if diag is None:
        dp = None
    else:
        da, dp = _host_f64(diag)
    _check(lib().lisa_cholesky(_ptr(a), dp, int(D), _ptr(l), _ptr(info), _stream(stream)),
           "lisa_cholesky")


def lisa_gauss_draw(mu, l, idx, z, W, x, logq, stream=None):
    ia, ip = _host_i32(idx)
    _check(lib().lisa_gauss_draw(_ptr(mu), _ptr(l), ip, len(ia), _ptr(z), int(W), _ptr(x),
                                 _ptr(logq), _stream(stream)), "lisa_gauss_draw")


def lisa_gauss_logq(mu, l, idx, x, W, logq, stream=None):
    ia, ip = _host_i32(idx)
    _check(lib().lisa_gauss_logq(_ptr(mu), _ptr(l), ip, len(ia), _ptr(x), int(W), _ptr(logq),
                                 _stream(stream)), "lisa_gauss_logq")


def lisa_gauss_walk(x, l, idx, z, W, step, x_prop, stream=None):
    ia, ip = _host_i32(idx)
    _check(lib().lisa_gauss_walk(_ptr(x), _ptr(l), ip, len(ia), _ptr(z), int(W), float(step),
                                 _ptr(x_prop), _stream(stream)), "lisa_gauss_walk")


def lisa_mh_accept(W, x_prop, logl_prop, logq_prop, u, lo, hi, x, logl, logq, accepted=None,
                   stream=None, beta=None):
    (la, lp), (ha, hp) = _host_f64(lo), _host_f64(hi)
    _check(lib().lisa_mh_accept(int(W), _ptr(x_prop), _ptr(logl_prop), _ptr(logq_prop), _ptr(u),
                                _ptr(beta), lp, hp, _ptr(x), _ptr(logl), _ptr(logq),
                                _ptr(accepted), _stream(stream)), "lisa_mh_accept")


def lisa_pt_swap(T, W, betas, u, x, logl, logq, swapped=None, stream=None):
    ba, bp = _host_f64(betas)
    _check(lib().lisa_pt_swap(int(T), int(W), bp, _ptr(u), _ptr(x), _ptr(logl), _ptr(logq),
                              _ptr(swapped), _stream(stream)), "lisa_pt_swap")


def flow_create(dim, layers, hidden, max_batch, idx, perms, stream=None):
    h = ctypes.c_void_p()
    (ia, ip), (pa, pp) = _host_i32(idx), _host_i32(perms)
    _check(lib().flow_create(ctypes.byref(h), int(dim), int(layers), int(hidden), int(max_batch),
                             ip, pp, _stream(stream)), "flow_create")
    return h


def flow_set_wait_limit(f, polls):
    _check(lib().flow_set_wait_limit(f, int(polls)), "flow_set_wait_limit")


def flow_nparams(f):
    n = ctypes.c_int64()
    _check(lib().flow_nparams(f, ctypes.byref(n)), "flow_nparams")
    return n.value


def flow_set_params(f, params, stream=None):
    _check(lib().flow_set_params(f, _ptr(params), _stream(stream)), "flow_set_params")


def flow_get_params(f, params, stream=None):
    _check(lib().flow_get_params(f, _ptr(params), _stream(stream)), "flow_get_params")


def flow_set_frame(f, mu, scale, stream=None):
    _check(lib().flow_set_frame(f, _ptr(mu), _ptr(scale), _stream(stream)), "flow_set_frame")


def flow_logprob(f, x, W, logq, stream=None):
    _check(lib().flow_logprob(f, _ptr(x), int(W), _ptr(logq), _stream(stream)), "flow_logprob")


def flow_propose(f, z, W, x, logq, stream=None):
    _check(lib().flow_propose(f, _ptr(z), int(W), _ptr(x), _ptr(logq), _stream(stream)),
           "flow_propose")


def flow_grad(f, x, B, loss=None, grad=None, stream=None):
    _check(lib().flow_grad(f, _ptr(x), int(B), _ptr(loss), _ptr(grad), _stream(stream)),
           "flow_grad")


def flow_adam(f, grad, lr, stream=None):
    _check(lib().flow_adam(f, _ptr(grad), float(lr), _stream(stream)), "flow_adam")


def flow_train(f, samples, S, epochs, batch, lr, loss=None, stream=None):
    _check(lib().flow_train(f, _ptr(samples), int(S), int(epochs), int(batch), float(lr),
                            _ptr(loss), _stream(stream)), "flow_train")


def flow_destroy(f):
    lib().flow_destroy(f)


def lisa_td_destroy(ctx):
    lib().lisa_td_destroy(ctx)


def _need(t, dtype, shape, what):
    """Validate a tensor before its pointer crosses the C ABI (which cannot check
    element type or size): dtype, exact shape, CUDA device, contiguity."""
    if t.dtype != dtype:
        raise TypeError(f"{what}: dtype {t.dtype}, expected {dtype}")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{what}: shape {tuple(t.shape)}, expected {tuple(shape)}")
    if not t.is_cuda:
        raise ValueError(f"{what}: must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{what}: must be contiguous")
    return t


class Likelihood:
    """Owns one context; tensors in, tensors out (torch on cuda)."""

    def __init__(self, precision=0, max_walkers=32, stream=None, orbit_table=None, **cfg):
        """orbit_table: (t0, dt, positions [rows][3][3] in metres) for orbit=2."""
        import torch
        self.torch = torch
        self.cfg = make_config(precision=precision, max_walkers=max_walkers, **cfg)
        if orbit_table is not None:
            self.ctx = lisa_td_create_orbits(self.cfg, *orbit_table, stream=stream)
        else:
            self.ctx = lisa_td_create(self.cfg, stream)
        self.dtype = torch.float64 if precision == 0 else torch.float32

    def close(self):
        if self.ctx is not None:
            lisa_td_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _params(self, params):
        params = params.to(self.torch.float64).contiguous()
        return _need(params, self.torch.float64, (params.shape[0], 15), "params")

    def set_data(self, aet):
        aet = aet.to(self.torch.float64).contiguous()
        lisa_td_set_data(self.ctx, _need(aet, self.torch.float64, (3, self.cfg.n), "data"))

    def waveform(self, params):
        params = self._params(params)
        W = params.shape[0]
        h = self.torch.empty((W, self.cfg.n, 2), dtype=self.dtype, device=params.device)
        lisa_td_waveform(self.ctx, params, W, h)
        return h

    def project(self, params):
        params = self._params(params)
        W = params.shape[0]
        y = self.torch.empty((6, self.cfg.n, W), dtype=self.dtype, device=params.device)
        lisa_td_project(self.ctx, params, W, y)
        return y

    def tdi(self, y):
        y = y.contiguous()
        W = y.shape[2]
        _need(y, self.dtype, (6, self.cfg.n, W), "y")
        aet = self.torch.empty((3, self.cfg.n, W), dtype=self.dtype, device=y.device)
        lisa_td_tdi(self.ctx, y, W, aet)
        return aet

    def loglike_ragged(self, params, n_per_walker, with_status=False, stream=None):
        params = self._params(params)
        W = params.shape[0]
        out = self.torch.empty(W, dtype=self.torch.float64, device=params.device)
        st = self.torch.empty(W, dtype=self.torch.int32, device=params.device)
        lisa_td_loglike_ragged(self.ctx, params, W, n_per_walker, out, st, stream)
        return (out, st) if with_status else out

    def loglike(self, params, with_status=False):
        params = self._params(params)
        W = params.shape[0]
        out = self.torch.empty(W, dtype=self.torch.float64, device=params.device)
        st = self.torch.empty(W, dtype=self.torch.int32, device=params.device)
        lisa_td_loglike_batch(self.ctx, params, W, out, st)
        return (out, st) if with_status else out

    # heterodyned likelihood (lisa_td_het_*)
    def het_setup(self, theta0, nodes):
        import numpy as np
        self.het_nodes = np.ascontiguousarray(nodes, dtype=np.int64)
        self.het_nm = bin(self.cfg.mode_mask).count("1")
        lisa_td_het_setup(self.ctx, theta0, self.het_nodes)

    def het_loglike(self, params, with_status=False):
        params = self._params(params)
        W = params.shape[0]
        out = self.torch.empty(W, dtype=self.torch.float64, device=params.device)
        st = self.torch.empty(W, dtype=self.torch.int32, device=params.device)
        lisa_td_het_loglike(self.ctx, params, W, out, st)
        return (out, st) if with_status else out

    def het_deltas(self, params):
        """Node differences [B][n_modes][3][W] as a complex tensor."""
        params = self._params(params)
        W = params.shape[0]
        B = self.het_nodes.size
        dz = self.torch.empty((B, self.het_nm, 3, W, 2), dtype=self.dtype, device=params.device)
        lisa_td_het_deltas(self.ctx, params, W, dz)
        return self.torch.view_as_complex(dz)

    def het_aet(self, params):
        params = self._params(params)
        W = params.shape[0]
        aet = self.torch.empty((3, self.cfg.n, W), dtype=self.dtype, device=params.device)
        lisa_td_het_aet(self.ctx, params, W, aet)
        return aet
