"""Python binding of libcpmdp, the GB300 CP-MDP library (C ABI in include/cpmdp.h).

Argument marshalling only: every step of the backup, value iteration and
policy iteration runs in the library's CUDA kernels. PyTorch supplies device
memory and streams; tensors are passed by ``data_ptr()``. There is no CPU
fallback: importing this module raises if ``libcpmdp.so`` has not been built
(``python paper_2103_00331_gb300/build.py``).

Names follow the C ABI: ``build_factors``, ``bellman_backup``,
``value_iteration``, ``policy_iteration``, ``components``, ``factors_info``.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libcpmdp.so")

MAX_DIM = 9
OK, EINVAL, ENOMEM, ECUDA, ENOCONV, ETIMEOUT = 0, 1, 2, 3, 4, 5
F32, F64, BF16X3 = 0, 1, 2
GRIDWORLD, DENSE_CP = 0, 1
SOLVER_PLAIN, SOLVER_GRID_BARRIER, SOLVER_BARRIER_FREE, SOLVER_DENSE, SOLVER_BATCH, SOLVER_MARCH_GRAPH = 0, 1, 2, 3, 4, 5
SOLVER_BATCH_RESIDENT = 6
STATUS_NAMES = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ENOCONV", 5: "ETIMEOUT"}


class CpmdpError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class Problem(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int32), ("shape", ctypes.c_int64 * MAX_DIM),
                ("nactions", ctypes.c_int32), ("kind", ctypes.c_int32),
                ("p_success", ctypes.c_double), ("cell", ctypes.c_void_p),
                ("reward", ctypes.c_void_p), ("rank", ctypes.c_int32),
                ("factors", ctypes.c_void_p), ("lambda_", ctypes.c_void_p),
                ("gamma", ctypes.c_double)]


class SolveOpts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("max_iter", ctypes.c_int32), ("certify", ctypes.c_int32),
                ("fused", ctypes.c_int32), ("eval_tol", ctypes.c_double),
                ("max_eval_iter", ctypes.c_int32), ("max_rounds", ctypes.c_int32),
                ("timeout_s", ctypes.c_double), ("trace", ctypes.c_void_p),
                ("partial_eval", ctypes.c_int32), ("inject_stall", ctypes.c_int32)]


class Result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("iterations", ctypes.c_int32),
                ("rounds", ctypes.c_int32), ("eval_sweeps", ctypes.c_int32),
                ("residual", ctypes.c_double), ("certified_residual", ctypes.c_double),
                ("error_bound", ctypes.c_double), ("backups", ctypes.c_int64),
                ("elapsed_ms", ctypes.c_double), ("solver", ctypes.c_int32), ("tail_from", ctypes.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if not k.startswith("_")}


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with "
                          "`python paper_2103_00331_gb300/build.py` (needs nvcc for sm_103a)")
    lib = ctypes.CDLL(LIB_PATH)
    vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    lib.cpmdp_default_opts.argtypes = [ctypes.POINTER(SolveOpts)]
    lib.cpmdp_default_opts.restype = None
    lib.cpmdp_build_factors.argtypes = [ctypes.POINTER(Problem), ctypes.c_int, ctypes.POINTER(vp)]
    lib.cpmdp_build_factors.restype = ctypes.c_int
    lib.cpmdp_free_factors.argtypes = [vp]
    lib.cpmdp_free_factors.restype = None
    lib.cpmdp_factors_info.argtypes = [vp, ctypes.POINTER(i64), ctypes.POINTER(i32),
                                       ctypes.POINTER(i32), ctypes.POINTER(i32)]
    lib.cpmdp_factors_info.restype = ctypes.c_int
    lib.cpmdp_components.argtypes = [vp, i64, i32, vp, vp, i32, ctypes.POINTER(i32)]
    lib.cpmdp_components.restype = ctypes.c_int
    lib.cpmdp_bellman_backup.argtypes = [vp, ctypes.c_int, vp, vp, vp, vp, vp]
    lib.cpmdp_bellman_backup.restype = ctypes.c_int
    lib.cpmdp_value_iteration.argtypes = [vp, ctypes.c_int, vp, vp, ctypes.POINTER(SolveOpts),
                                          ctypes.POINTER(Result), vp]
    lib.cpmdp_value_iteration.restype = ctypes.c_int
    lib.cpmdp_policy_iteration.argtypes = [vp, ctypes.c_int, vp, vp, ctypes.POINTER(SolveOpts),
                                           ctypes.POINTER(Result), vp]
    lib.cpmdp_policy_iteration.restype = ctypes.c_int
    lib.cpmdp_value_iteration_static.argtypes = [i32, ctypes.POINTER(i64), ctypes.c_double,
                                                 ctypes.c_double, vp, vp, vp, ctypes.c_double, i32,
                                                 ctypes.POINTER(i32), ctypes.POINTER(ctypes.c_double), vp]
    lib.cpmdp_value_iteration_static.restype = ctypes.c_int
    lib.cpmdp_batch_build.argtypes = [ctypes.POINTER(Problem), i32, ctypes.c_int, ctypes.POINTER(vp)]
    lib.cpmdp_batch_build.restype = ctypes.c_int
    lib.cpmdp_batch_free.argtypes = [vp]
    lib.cpmdp_batch_free.restype = None
    lib.cpmdp_batch_info.argtypes = [vp, ctypes.POINTER(i32), ctypes.POINTER(i64), vp]
    lib.cpmdp_batch_info.restype = ctypes.c_int
    lib.cpmdp_batch_value_iteration.argtypes = [vp, vp, ctypes.POINTER(SolveOpts), vp, vp,
                                                ctypes.POINTER(Result), vp]
    lib.cpmdp_batch_value_iteration.restype = ctypes.c_int
    lib.cpmdp_batch_certify.argtypes = [vp, vp, vp, vp, vp]
    lib.cpmdp_batch_certify.restype = ctypes.c_int
    for name, args in [
            ("cpmdp_ws_features", [vp, i32, i32, vp, vp]),
            ("cpmdp_ws_coarse_vi", [vp, i32, i32, ctypes.c_float, i32, vp, vp, vp]),
            ("cpmdp_ws_targets", [vp, vp, i32, i32, vp, vp, vp, vp]),
            ("cpmdp_ws_upsample", [vp, vp, vp, i32, i32, vp, vp]),
            ("cpmdp_ws_fine_loss_grad", [vp, vp, i32, i32, vp, vp, vp, vp, vp, vp]),
            ("cpmdp_conv3d_forward", [vp, vp, vp, vp, vp, i32, i32, i32, i32, i32, i32, vp]),
            ("cpmdp_conv3d_backward_data", [vp, vp, vp, vp, i32, i32, i32, i32, i32, vp]),
            ("cpmdp_conv3d_backward_weight", [vp, vp, vp, vp, i32, i32, i32, i32, i32, vp]),
            ("cpmdp_ws_loss_grad", [vp, vp, vp, i32, vp, vp, vp]),
            ("cpmdp_adam_step", [vp, vp, vp, vp, i64, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                 ctypes.c_float, i32, vp]),
            ("cpmdp_ws_cast_weights", [vp, vp, vp, i32, vp]),
            ("cpmdp_ws_sync", [vp])]:
        getattr(lib, name).argtypes = args
        getattr(lib, name).restype = ctypes.c_int
    lib.cpmdp_last_error.argtypes = []
    lib.cpmdp_last_error.restype = ctypes.c_char_p
    lib.cpmdp_version.argtypes = []
    lib.cpmdp_version.restype = ctypes.c_char_p
    return lib


lib = _load()

EXPORTED = ["cpmdp_default_opts", "cpmdp_build_factors", "cpmdp_free_factors", "cpmdp_factors_info",
            "cpmdp_components", "cpmdp_bellman_backup", "cpmdp_value_iteration",
            "cpmdp_policy_iteration", "cpmdp_value_iteration_static", "cpmdp_batch_build",
            "cpmdp_batch_free", "cpmdp_batch_info", "cpmdp_batch_value_iteration", "cpmdp_batch_certify",
            "cpmdp_ws_features", "cpmdp_ws_coarse_vi",
            "cpmdp_ws_targets", "cpmdp_ws_upsample", "cpmdp_ws_fine_loss_grad", "cpmdp_conv3d_forward", "cpmdp_conv3d_backward_data",
            "cpmdp_conv3d_backward_weight", "cpmdp_ws_loss_grad", "cpmdp_adam_step", "cpmdp_ws_cast_weights",
            "cpmdp_ws_sync", "cpmdp_last_error", "cpmdp_version"]


def last_error() -> str:
    return lib.cpmdp_last_error().decode()


def version() -> str:
    return lib.cpmdp_version().decode()


def _check(status):
    if status != OK:
        raise CpmdpError(status, last_error())


def default_opts(**kw) -> SolveOpts:
    o = SolveOpts()
    lib.cpmdp_default_opts(ctypes.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise TypeError(f"unknown option {k}")
        setattr(o, k, v)
    return o


def _ptr(t):
    """Device (or host) address of a tensor / numpy array / int / None."""
    if t is None:
        return None
    if isinstance(t, int):
        return t
    if isinstance(t, np.ndarray):
        return t.ctypes.data
    return t.data_ptr()


def _stream(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


class Factors:
    """Owner of a ``cpmdp_factors`` handle (freed on ``close`` / GC)."""

    def __init__(self, handle, keep):
        self.handle = handle
        self._keep = keep

    def close(self):
        if self.handle:
            lib.cpmdp_free_factors(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self):
        return factors_info(self)


def make_problem(shape, nactions, kind, reward, gamma, p_success=1.0, cell=None,
                 factors=None, lam=None, rank=0):
    """Fill a ``cpmdp_problem`` from numpy arrays (kept alive by the caller)."""
    pr = Problem()
    shape = tuple(int(n) for n in shape)
    pr.ndim = len(shape)
    for d, n in enumerate(shape[:MAX_DIM]):
        pr.shape[d] = n
    pr.nactions = int(nactions)
    pr.kind = int(kind)
    pr.p_success = float(p_success)
    pr.cell = _ptr(cell)
    pr.reward = _ptr(reward)
    pr.rank = int(rank)
    pr.factors = _ptr(factors)
    pr.lambda_ = _ptr(lam)
    pr.gamma = float(gamma)
    return pr


def build_factors(problem, device: int = 0) -> Factors:
    """``cpmdp_build_factors``. ``problem`` is a ``Problem`` or an instance
    with GridWorld / DenseCP fields (``cpmdp_inputs``)."""
    keep = []
    if not isinstance(problem, Problem):
        inst = problem
        reward = np.ascontiguousarray(np.asarray(inst.reward, dtype=np.float64).reshape(-1))
        keep.append(reward)
        if hasattr(inst, "cell"):
            cell = np.ascontiguousarray(np.asarray(inst.cell, dtype=np.uint8).reshape(-1))
            keep.append(cell)
            problem = make_problem(inst.shape, 2 * len(inst.shape), GRIDWORLD, reward, inst.gamma,
                                   p_success=inst.p, cell=cell)
        else:
            fac = np.ascontiguousarray(inst.packed_factors())
            lam = np.ascontiguousarray(np.asarray(inst.lam, dtype=np.float64).reshape(-1))
            keep += [fac, lam]
            problem = make_problem(inst.shape, inst.nactions, DENSE_CP, reward, inst.gamma,
                                   factors=fac, lam=lam, rank=inst.rank)
    h = ctypes.c_void_p()
    _check(lib.cpmdp_build_factors(ctypes.byref(problem), int(device), ctypes.byref(h)))
    return Factors(h, None)


def factors_info(f: Factors):
    ns, na, rk, nd = ctypes.c_int64(), ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    _check(lib.cpmdp_factors_info(f.handle, ctypes.byref(ns), ctypes.byref(na), ctypes.byref(rk),
                                  ctypes.byref(nd)))
    return {"nstates": ns.value, "nactions": na.value, "rank": rk.value, "ndim": nd.value}


def components(f: Factors, state: int, action: int, cap: int = 64):
    """Definition 3 components of (state, action): list of (s', P(s'|s,a))."""
    nxt = np.zeros(cap, dtype=np.int64)
    prob = np.zeros(cap, dtype=np.float64)
    cnt = ctypes.c_int32()
    _check(lib.cpmdp_components(f.handle, int(state), int(action), nxt.ctypes.data,
                                prob.ctypes.data, cap, ctypes.byref(cnt)))
    n = cnt.value
    if n > cap:
        return components(f, state, action, cap=n)
    return list(zip(nxt[:n].tolist(), prob[:n].tolist()))


def bellman_backup(f: Factors, precision, V_in, V_out, policy_out=None, residual_out=None,
                   stream=None):
    """``cpmdp_bellman_backup`` on device tensors (asynchronous)."""
    _check(lib.cpmdp_bellman_backup(f.handle, int(precision), _ptr(V_in), _ptr(V_out),
                                    _ptr(policy_out), _ptr(residual_out), _stream(stream)))


def value_iteration(f: Factors, precision, V, policy_out=None, opts=None, stream=None,
                    raise_on_noconv=True):
    """``cpmdp_value_iteration``: returns the ``Result`` as a dict."""
    res = Result()
    st = lib.cpmdp_value_iteration(f.handle, int(precision), _ptr(V), _ptr(policy_out),
                                   ctypes.byref(opts) if opts is not None else None,
                                   ctypes.byref(res), _stream(stream))
    if st != OK and not (st == ENOCONV and not raise_on_noconv):
        _check(st)
    return res.as_dict()


def policy_iteration(f: Factors, precision, V, policy, opts=None, stream=None,
                     raise_on_noconv=True):
    """``cpmdp_policy_iteration``: returns the ``Result`` as a dict."""
    res = Result()
    st = lib.cpmdp_policy_iteration(f.handle, int(precision), _ptr(V), _ptr(policy),
                                    ctypes.byref(opts) if opts is not None else None,
                                    ctypes.byref(res), _stream(stream))
    if st != OK and not (st == ENOCONV and not raise_on_noconv):
        _check(st)
    return res.as_dict()


def value_iteration_static(shape, p_success, gamma, cell, reward, V, tol=1e-6, max_iter=1000,
                           stream=None):
    """``cpmdp_value_iteration_static``: FP32 GridWorld value iteration with no
    device allocation (scratch in a fixed static device array). ``cell`` (uint8
    or None), ``reward`` (float32) and ``V`` (float32) are device tensors.
    Returns (iterations, residual); raises on any status but OK."""
    shape = tuple(int(n) for n in shape)
    sh = (ctypes.c_int64 * len(shape))(*shape)
    it, res = ctypes.c_int32(), ctypes.c_double()
    _check(lib.cpmdp_value_iteration_static(len(shape), sh, float(p_success), float(gamma),
                                            _ptr(cell), _ptr(reward), _ptr(V), float(tol),
                                            int(max_iter), ctypes.byref(it), ctypes.byref(res),
                                            _stream(stream)))
    return it.value, res.value


class Batch:
    """Owner of a ``cpmdp_batch`` handle (freed on ``close`` / GC)."""

    def __init__(self, handle):
        self.handle = handle
        n, tot = ctypes.c_int32(), ctypes.c_int64()
        _check(lib.cpmdp_batch_info(handle, ctypes.byref(n), ctypes.byref(tot), None))
        self.count, self.total_states = n.value, tot.value
        self.offsets = np.zeros(self.count + 1, dtype=np.int64)
        _check(lib.cpmdp_batch_info(handle, None, None, self.offsets.ctypes.data))

    def close(self):
        if self.handle:
            lib.cpmdp_batch_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def batch_build(instances, device: int = 0) -> Batch:
    """``cpmdp_batch_build`` from a list of GridWorld instances (``cpmdp_inputs``)."""
    n = len(instances)
    arr = (Problem * n)()
    keep = []
    for i, inst in enumerate(instances):
        reward = np.ascontiguousarray(np.asarray(inst.reward, dtype=np.float64).reshape(-1))
        cell = np.ascontiguousarray(np.asarray(inst.cell, dtype=np.uint8).reshape(-1))
        keep += [reward, cell]
        arr[i] = make_problem(inst.shape, 2 * len(inst.shape), GRIDWORLD, reward, inst.gamma,
                              p_success=inst.p, cell=cell)
    h = ctypes.c_void_p()
    _check(lib.cpmdp_batch_build(arr, n, int(device), ctypes.byref(h)))
    return Batch(h)


def batch_value_iteration(batch: Batch, V, opts=None, stream=None, raise_on_noconv=True):
    """``cpmdp_batch_value_iteration``: returns (result dict, sweeps per
    instance, last residual per instance)."""
    it = np.zeros(batch.count, dtype=np.int32)
    rs = np.zeros(batch.count, dtype=np.float64)
    res = Result()
    st = lib.cpmdp_batch_value_iteration(batch.handle, _ptr(V),
                                         ctypes.byref(opts) if opts is not None else None,
                                         it.ctypes.data, rs.ctypes.data, ctypes.byref(res),
                                         _stream(stream))
    if st != OK and not (st == ENOCONV and not raise_on_noconv):
        _check(st)
    return res.as_dict(), it, rs


def batch_certify(batch: Batch, V, policy_out=None, stream=None):
    """``cpmdp_batch_certify``: one FP64 backup of every instance of the
    packed values V; writes the FP64 argmax policy to ``policy_out`` (packed
    uint8 device tensor, optional) and returns the certified residual
    max |T(V) - V| per instance (numpy float64)."""
    cert = np.zeros(batch.count, dtype=np.float64)
    _check(lib.cpmdp_batch_certify(batch.handle, _ptr(V), _ptr(policy_out), cert.ctypes.data, _stream(stream)))
    return cert


def ws_features(batch, first, count, feat, stream=None):
    _check(lib.cpmdp_ws_features(batch.handle, int(first), int(count), _ptr(feat), _stream(stream)))


def ws_coarse_vi(batch, first, count, coarse_v, feat=None, tol=1e-4, max_sweeps=4000, stream=None):
    _check(lib.cpmdp_ws_coarse_vi(batch.handle, int(first), int(count), float(tol), int(max_sweeps), _ptr(coarse_v),
                                  _ptr(feat), _stream(stream)))


def ws_targets(batch, V, first, count, target, mask, base=None, stream=None):
    _check(lib.cpmdp_ws_targets(batch.handle, _ptr(V), int(first), int(count), _ptr(base), _ptr(target),
                                _ptr(mask), _stream(stream)))


def ws_upsample(batch, coarse, first, count, V, base=None, stream=None):
    _check(lib.cpmdp_ws_upsample(batch.handle, _ptr(coarse), _ptr(base), int(first), int(count), _ptr(V),
                                 _stream(stream)))


def ws_fine_loss_grad(batch, V_target, first, count, pred, base, resid, dy, loss=None, stream=None):
    """``cpmdp_ws_fine_loss_grad``: loss of upsample(pred + base) against
    V_target on the full grid (added to ``loss``) and its gradient with
    respect to pred in channel 0 of ``dy``."""
    _check(lib.cpmdp_ws_fine_loss_grad(batch.handle, _ptr(V_target), int(first), int(count), _ptr(pred), _ptr(base),
                                       _ptr(resid), _ptr(dy), _ptr(loss), _stream(stream)))


def conv3d_forward(x, wf, bias, y, y0, dims, dilation, relu, stream=None):
    n, z, yy, xx = dims
    _check(lib.cpmdp_conv3d_forward(_ptr(x), _ptr(wf), _ptr(bias), _ptr(y), _ptr(y0), n, z, yy, xx,
                                    int(dilation), int(relu), _stream(stream)))


def conv3d_backward_data(dy, wb, act_in, dx, dims, dilation, stream=None):
    n, z, yy, xx = dims
    _check(lib.cpmdp_conv3d_backward_data(_ptr(dy), _ptr(wb), _ptr(act_in), _ptr(dx), n, z, yy, xx,
                                          int(dilation), _stream(stream)))


def conv3d_backward_weight(x, dy, dw, db, dims, dilation, stream=None):
    n, z, yy, xx = dims
    _check(lib.cpmdp_conv3d_backward_weight(_ptr(x), _ptr(dy), _ptr(dw), _ptr(db), n, z, yy, xx,
                                            int(dilation), _stream(stream)))


def ws_loss_grad(pred, target, mask, nvox, dy, loss, stream=None):
    _check(lib.cpmdp_ws_loss_grad(_ptr(pred), _ptr(target), _ptr(mask), int(nvox), _ptr(dy), _ptr(loss),
                                  _stream(stream)))


def adam_step(p, g, m, v, n, lr, beta1, beta2, eps, step, stream=None):
    _check(lib.cpmdp_adam_step(_ptr(p), _ptr(g), _ptr(m), _ptr(v), int(n), lr, beta1, beta2, eps, int(step),
                               _stream(stream)))


def ws_cast_weights(w, wf, wb, layers, stream=None):
    _check(lib.cpmdp_ws_cast_weights(_ptr(w), _ptr(wf), _ptr(wb), int(layers), _stream(stream)))


def ws_sync(stream=None):
    """``cpmdp_ws_sync``: wait for the queued warm-start work; raises on a
    tensor-core wait that ran out."""
    _check(lib.cpmdp_ws_sync(_stream(stream)))
