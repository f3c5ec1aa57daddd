"""Python binding of the C ABI in include/tc.h (argument marshalling only).

Every computation runs in libtc_b300.so; if the library cannot be loaded this module raises
instead of falling back to anything else.  Arrays are numpy (host) arrays; device pointers are
plain integers (e.g. ``torch.Tensor.data_ptr()``), streams are ``cudaStream_t`` integers (e.g.
``torch.cuda.current_stream().cuda_stream``).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

TC_OK, TC_ERR_ARG, TC_ERR_MESH, TC_ERR_STATE = 0, -1, -2, -3
TC_ERR_CUDA, TC_ERR_NOMEM, TC_ERR_TIMEOUT, TC_ERR_NAN = -4, -5, -6, -7
TC_MODEL_MS, TC_MODEL_TP06 = 0, 1
TC_FP64, TC_FP32 = 0, 1
TC_OP_M, TC_OP_K, TC_OP_A = 0, 1, 2
TC_FIELD_V, TC_FIELD_V_PREV, TC_FIELD_STATE = 0, 1, 16

_STATUS_NAMES = {0: "TC_OK", -1: "TC_ERR_ARG", -2: "TC_ERR_MESH", -3: "TC_ERR_STATE",
                 -4: "TC_ERR_CUDA", -5: "TC_ERR_NOMEM", -6: "TC_ERR_TIMEOUT", -7: "TC_ERR_NAN"}


class TcError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{_STATUS_NAMES.get(status, status)}: {message}")
        self.status = status
        self.message = message


class StepStats(C.Structure):
    _fields_ = [("steps", C.c_int64), ("step_index", C.c_int64), ("cg_iterations", C.c_int64),
                ("max_iterations", C.c_int32), ("not_converged", C.c_int32),
                ("last_znorm", C.c_double), ("last_z0norm", C.c_double), ("graph_steps", C.c_int64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class Profile(C.Structure):
    _fields_ = [("ionic_ms", C.c_double), ("ionic_launches", C.c_int64),
                ("pcg_ms", C.c_double), ("pcg_launches", C.c_int64),
                ("pcg_iterations", C.c_int64), ("surrogate_ms", C.c_double),
                ("surrogate_windows", C.c_int64), ("mlp_ms", C.c_double), ("surrogate_rows", C.c_int64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_P = C.c_void_p
_D = C.POINTER(C.c_double)
_I32 = C.POINTER(C.c_int32)
_I64 = C.POINTER(C.c_int64)
_SIGS = {
    "tc_mesh_create": [_D, C.c_int64, _I32, C.c_int64, _D, _I32, C.POINTER(_P)],
    "tc_mesh_nnz": [_P, _I64],
    "tc_mesh_matrices": [_P, _D, _D, C.c_int32, _I64, _I32, _D, _D],
    "tc_mesh_ordering": [_P, C.c_int32, _I32, _I32],
    "tc_mesh_set_sell_sigma": [_P, C.c_int32],
    "tc_assemble": [_P, _D, _D, C.c_int32, C.c_double, C.c_double, C.c_double, C.c_double,
                    C.c_int32, _P, C.POINTER(_P)],
    "tc_sim_size": [_P, _I64, _I64, _I64, _I32],
    "tc_sim_layout": [_P, _I32, _I64, _I32, _I32],
    "tc_sim_staging": [_P, _I32, _I32, _I32, _I64, _I32],
    "tc_set_launch": [_P, C.c_int32, C.c_int32],
    "tc_autotune": [_P, C.c_int32, _I32, _I32, _D],
    "tc_set_graphs": [_P, C.c_int32],
    "tc_mesh_layout_size": [_P, _I32, _I64],
    "tc_monodomain_conductivity": [_D, _D, _D, _D, C.c_int32, _D, _D],
    "tc_set_ionic": [_P, C.c_int32, _D, C.c_int32, _D],
    "tc_add_stimulus": [_P, _I32, C.c_int64, C.c_double, C.c_double, C.c_double],
    "tc_set_solver": [_P, C.c_double, C.c_double, C.c_int32],
    "tc_set_activation_threshold": [_P, C.c_double],
    "tc_step": [_P, C.c_int64, C.POINTER(StepStats)],
    "tc_read_state": [_P, C.c_int32, _D, C.c_int64],
    "tc_write_state": [_P, C.c_int32, _D, C.c_int64],
    "tc_activation_times": [_P, C.c_double, _D, C.c_int64],
    "tc_set_repolarisation_threshold": [_P, C.c_double],
    "tc_repolarisation_times": [_P, _D, C.c_int64],
    "tc_apd90": [_P, _D, C.c_int64],
    "tc_get_step_index": [_P, _I64],
    "tc_set_step_index": [_P, C.c_int64],
    "tc_apply_operator": [_P, C.c_int32, _D, _D, C.c_int64],
    "tc_apply_operator_dev": [_P, C.c_int32, _P, _P],
    "tc_apply_operator_static": [_P, C.c_int32, _D, _D, C.c_int64],
    "tc_set_profiling": [_P, C.c_int32],
    "tc_get_profile": [_P, C.POINTER(Profile)],
    "tc_reset_profile": [_P],
    "tc_set_wait_limit": [_P, C.c_int64],
    "tc_selftest_exp": [_D, _D, _D, C.c_int64],
    "tc_selftest_log": [_D, _D, _D, C.c_int64],
    "tc_selftest_rcp": [_D, _D, _D, C.c_int64],
    "tc_selftest_exp2": [_D, _D, _D, C.c_int64],
    "tc_measure_fp64_rate": [_D],
    "tc_mlp_create": [C.c_uint64, C.POINTER(_P)],
    "tc_mlp_n_params": [_P, _I64],
    "tc_mlp_get_params": [_P, C.POINTER(C.c_float), C.c_int64],
    "tc_mlp_set_params": [_P, C.POINTER(C.c_float), C.c_int64],
    "tc_mlp_set_normalization": [_P, C.POINTER(C.c_float), C.c_int64],
    "tc_mlp_set_gemm": [_P, C.c_int32],
    "tc_mlp_fit_normalization": [_P, _P, _P, C.c_int64],
    "tc_mlp_get_normalization": [_P, C.POINTER(C.c_float), C.c_int64],
    "tc_mlp_forward": [_P, C.POINTER(C.c_float), C.c_int64, C.POINTER(C.c_float)],
    "tc_mlp_gradients": [_P, C.POINTER(C.c_float), C.POINTER(C.c_float), C.c_int64,
                         C.POINTER(C.c_float), C.POINTER(C.c_float)],
    "tc_mlp_train": [_P, _P, _P, C.c_int64, C.c_int32, C.c_int32, C.c_float, C.c_uint64, _P,
                     C.POINTER(C.c_float)],
    "tc_mlp_diagnostics": [_P, _P],
    "tc_gemm_bf16_nt": [_P, _P, _P, C.c_int32, C.c_int32, C.c_int32, _P],
    "tc_tp06_window": [_P, _P, C.c_int64, C.c_double, C.c_int32, C.c_int32, C.c_int32, _P, _P],
    "tc_set_surrogate": [_P, _P, C.c_int32, C.c_double, C.c_double, C.c_double, C.c_double],
    "tc_surrogate_usage": [_P, _I64, _I64],
    "tc_surrogate_sample": [_P, C.c_int32, C.c_double, C.c_double, C.c_double, C.c_double, C.c_uint64, _P, _P,
                            C.c_int64, _I64],
}
_VOID = {"tc_mesh_destroy": [_P], "tc_sim_destroy": [_P], "tc_mlp_destroy": [_P]}
_STR = {"tc_last_error": [], "tc_version": []}

_lib = None


def lib():
    """Load (building first if needed) the in-tree libtc_b300.so and declare its signatures."""
    global _lib
    if _lib is None:
        path = _build.LIB
        if not os.path.exists(path):
            path = _build.build()
        L = C.CDLL(path)
        for name, args in _SIGS.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = C.c_int
        for name, args in _VOID.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = None
        for name, args in _STR.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = C.c_char_p
        _lib = L
    return _lib


def exported_symbols():
    return list(_SIGS) + list(_VOID) + list(_STR)


def _check(status):
    if status != TC_OK:
        raise TcError(status, lib().tc_last_error().decode())


def _d(a):
    return a.ctypes.data_as(_D)


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


class Mesh:
    """tc_mesh: a copied tetrahedral mesh (coordinates mm, 0-based tets, unit fibres)."""

    def __init__(self, xyz, tets, fibres=None, region=None):
        xyz = _f64(xyz).reshape(-1, 3)
        tets = _i32(tets).reshape(-1, 4)
        fib = None if fibres is None else _f64(fibres).reshape(-1, 3)
        reg = None if region is None else _i32(region)
        h = _P()
        _check(lib().tc_mesh_create(_d(xyz), xyz.shape[0], tets.ctypes.data_as(_I32), tets.shape[0],
                                    None if fib is None else _d(fib),
                                    None if reg is None else reg.ctypes.data_as(_I32), C.byref(h)))
        self._h = h
        self.n_nodes = xyz.shape[0]
        self.n_tets = tets.shape[0]

    @classmethod
    def from_inputs(cls, m):
        return cls(m.xyz, m.tets, m.fibres, m.region)

    @property
    def nnz(self):
        v = C.c_int64()
        _check(lib().tc_mesh_nnz(self._h, C.byref(v)))
        return v.value

    def matrices(self, sigma_l, sigma_t):
        """Host-assembled (row_ptr, col, M values, K values) in the caller's node order."""
        sl = _f64(np.atleast_1d(sigma_l))
        st = _f64(np.atleast_1d(sigma_t))
        nnz = self.nnz
        rp = np.empty(self.n_nodes + 1, dtype=np.int64)
        col = np.empty(nnz, dtype=np.int32)
        mv = np.empty(nnz)
        kv = np.empty(nnz)
        _check(lib().tc_mesh_matrices(self._h, _d(sl), _d(st), sl.size, rp.ctypes.data_as(_I64),
                                      col.ctypes.data_as(_I32), _d(mv), _d(kv)))
        return rp, col, mv, kv

    def layout_size(self):
        nc, ni = C.c_int32(), C.c_int64()
        _check(lib().tc_mesh_layout_size(self._h, C.byref(nc), C.byref(ni)))
        return nc.value, ni.value

    def ordering(self, sell_sigma=1):
        perm = np.empty(self.n_nodes, dtype=np.int32)
        sw = np.empty(self.layout_size()[1] // 32, dtype=np.int32)
        _check(lib().tc_mesh_ordering(self._h, sell_sigma, perm.ctypes.data_as(_I32),
                                      sw.ctypes.data_as(_I32)))
        return perm, sw

    def set_sell_sigma(self, sigma):
        """SELL row-sorting window for simulations assembled from this mesh afterwards."""
        _check(lib().tc_mesh_set_sell_sigma(self._h, int(sigma)))

    def close(self):
        if getattr(self, "_h", None):
            lib().tc_mesh_destroy(self._h)
            self._h = None

    __del__ = close


class Simulation:
    """tc_sim: the device-resident monodomain simulation."""

    def __init__(self, mesh: Mesh, sigma_l, sigma_t, chi, cm, theta, dt, precision=TC_FP64,
                 stream=None):
        sl = _f64(np.atleast_1d(sigma_l))
        st = _f64(np.atleast_1d(sigma_t))
        h = _P()
        _check(lib().tc_assemble(mesh._h, _d(sl), _d(st), sl.size, chi, cm, theta, dt, precision,
                                 None if stream is None else _P(int(stream)), C.byref(h)))
        self._h = h
        self.n_nodes = mesh.n_nodes

    # -- configuration
    def set_ionic(self, model, params, init_state=None):
        p = _f64(np.atleast_1d(params))
        s = None if init_state is None else _f64(init_state)
        _check(lib().tc_set_ionic(self._h, model, _d(p), p.size, None if s is None else _d(s)))

    def add_stimulus(self, nodes, start, duration, intensity):
        nd = _i32(nodes)
        _check(lib().tc_add_stimulus(self._h, nd.ctypes.data_as(_I32), nd.size, start, duration,
                                     intensity))

    def set_solver(self, atol, rtol, max_iter):
        _check(lib().tc_set_solver(self._h, atol, rtol, max_iter))

    def set_activation_threshold(self, v):
        _check(lib().tc_set_activation_threshold(self._h, v))

    def set_wait_limit(self, polls):
        _check(lib().tc_set_wait_limit(self._h, polls))

    # -- stepping and I/O
    def step(self, n_steps=1):
        st = StepStats()
        _check(lib().tc_step(self._h, n_steps, C.byref(st)))
        return st.as_dict()

    def read(self, field=TC_FIELD_V, out=None):
        """Field in caller node order; with `out` (a C-contiguous float64 array of n entries,
        ideally page-locked) the values land there directly."""
        if out is None:
            out = np.empty(self.n_nodes)
        elif out.dtype != np.float64 or not out.flags["C_CONTIGUOUS"] or out.size != self.n_nodes:
            raise TcError(TC_ERR_ARG, "out must be a C-contiguous float64 array of n_nodes entries")
        _check(lib().tc_read_state(self._h, field, _d(out), self.n_nodes))
        return out

    def write(self, field, values):
        v = _f64(values)
        _check(lib().tc_write_state(self._h, field, _d(v), v.size))

    def activation_times(self, v_threshold=0.0):
        out = np.empty(self.n_nodes)
        _check(lib().tc_activation_times(self._h, v_threshold, _d(out), self.n_nodes))
        return out

    def set_repolarisation_threshold(self, v):
        _check(lib().tc_set_repolarisation_threshold(self._h, v))

    def repolarisation_times(self):
        out = np.empty(self.n_nodes)
        _check(lib().tc_repolarisation_times(self._h, _d(out), self.n_nodes))
        return out

    def apd90(self):
        out = np.empty(self.n_nodes)
        _check(lib().tc_apd90(self._h, _d(out), self.n_nodes))
        return out

    @property
    def step_index(self):
        v = C.c_int64()
        _check(lib().tc_get_step_index(self._h, C.byref(v)))
        return v.value

    @step_index.setter
    def step_index(self, k):
        _check(lib().tc_set_step_index(self._h, k))

    def apply(self, op, x):
        x = _f64(x)
        y = np.empty(self.n_nodes)
        _check(lib().tc_apply_operator(self._h, op, _d(x), _d(y), x.size))
        return y

    def apply_static(self, op, x):
        """tc_apply_operator_static: y = Op x with no device allocation (static staging)."""
        x = _f64(x)
        y = np.empty(self.n_nodes)
        _check(lib().tc_apply_operator_static(self._h, op, _d(x), _d(y), x.size))
        return y

    def apply_dev(self, op, x_ptr: int, y_ptr: int):
        _check(lib().tc_apply_operator_dev(self._h, op, _P(x_ptr), _P(y_ptr)))

    def size(self):
        n, nnz, pad = C.c_int64(), C.c_int64(), C.c_int64()
        nb = C.c_int32()
        _check(lib().tc_sim_size(self._h, C.byref(n), C.byref(nnz), C.byref(pad), C.byref(nb)))
        return {"n_nodes": n.value, "nnz": nnz.value, "padded_nnz": pad.value, "n_blocks": nb.value}

    def layout(self):
        nc, ni, th, bps = C.c_int32(), C.c_int64(), C.c_int32(), C.c_int32()
        _check(lib().tc_sim_layout(self._h, C.byref(nc), C.byref(ni), C.byref(th), C.byref(bps)))
        return {"n_components": nc.value, "n_internal": ni.value, "pcg_threads": th.value,
                "blocks_per_sm": bps.value}

    def staging(self):
        nb, ns, mw, sm, i16 = C.c_int32(), C.c_int32(), C.c_int32(), C.c_int64(), C.c_int32()
        _check(lib().tc_sim_staging(self._h, C.byref(nb), C.byref(ns), C.byref(mw), C.byref(sm), C.byref(i16)))
        return {"blocks": nb.value, "staged_blocks": ns.value, "max_window": mw.value, "smem_bytes": sm.value,
                "idx16": bool(i16.value)}

    def set_launch(self, pcg_threads, blocks_per_sm):
        _check(lib().tc_set_launch(self._h, pcg_threads, blocks_per_sm))

    def autotune(self, trial_steps=20):
        th, bps, ms = C.c_int32(), C.c_int32(), C.c_double()
        _check(lib().tc_autotune(self._h, trial_steps, C.byref(th), C.byref(bps), C.byref(ms)))
        return {"pcg_threads": th.value, "blocks_per_sm": bps.value, "ms_per_step": ms.value}

    def set_graphs(self, on=True):
        _check(lib().tc_set_graphs(self._h, int(bool(on))))

    def set_surrogate(self, mlp, window=10, dv_max=2.0, dvdt_max=1.0, dv_neighbour=0.3, rest_band=0.5):
        """Attach a trained Mlp (or None to detach) as the learned ionic surrogate."""
        _check(lib().tc_set_surrogate(self._h, None if mlp is None else mlp._h, window, dv_max, dvdt_max,
                                      dv_neighbour, rest_band))
        self._mlp = mlp

    def surrogate_sample(self, x_dev, y_dev, capacity, count, window=10, rest_band=1.0, rest_keep=0.05,
                         dv_keep=0.0, dvdt_keep=0.0, seed=0):
        """Append training pairs from the current state to device arrays [capacity][20] and
        [capacity][19] (pointers); returns the new count."""
        c = C.c_int64(count)
        _check(lib().tc_surrogate_sample(self._h, window, rest_band, rest_keep, dv_keep, dvdt_keep, seed,
                                         _P(x_dev), _P(y_dev), capacity, C.byref(c)))
        return c.value

    def surrogate_usage(self):
        a, b = C.c_int64(), C.c_int64()
        _check(lib().tc_surrogate_usage(self._h, C.byref(a), C.byref(b)))
        return {"surrogate": a.value, "exact": b.value}

    def set_profiling(self, on=True):
        _check(lib().tc_set_profiling(self._h, int(bool(on))))

    def profile(self):
        p = Profile()
        _check(lib().tc_get_profile(self._h, C.byref(p)))
        return p.as_dict()

    def reset_profile(self):
        _check(lib().tc_reset_profile(self._h))

    def close(self):
        if getattr(self, "_h", None):
            lib().tc_sim_destroy(self._h)
            self._h = None

    __del__ = close


def set_model(sim, w):
    """tc_set_ionic with the workload's model and parameters (also resets to rest, step 0)."""
    if w.model == "ms":
        sim.set_ionic(TC_MODEL_MS, w.ms.as_array())
    elif w.model == "tp06":
        sim.set_ionic(TC_MODEL_TP06, [float(w.tp06_cell)])
    else:
        raise TcError(TC_ERR_ARG, f"model {w.model!r} is not available")


_F = C.POINTER(C.c_float)


def _f32(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float32)
    return a if shape is None else a.reshape(shape)


class Mlp:
    """tc_mlp: the learned ionic surrogate's network (device-resident)."""
    N_IN, N_OUT = 20, 19
    GEMM_TC, GEMM_SIMT = 0, 1

    def __init__(self, seed=0):
        h = _P()
        _check(lib().tc_mlp_create(seed, C.byref(h)))
        self._h = h
        n = C.c_int64()
        _check(lib().tc_mlp_n_params(self._h, C.byref(n)))
        self.n_params = n.value

    def params(self):
        out = np.empty(self.n_params, dtype=np.float32)
        _check(lib().tc_mlp_get_params(self._h, out.ctypes.data_as(_F), out.size))
        return out

    def set_params(self, p):
        p = _f32(p)
        _check(lib().tc_mlp_set_params(self._h, p.ctypes.data_as(_F), p.size))

    def set_normalization(self, in_mean, in_scale, out_mean, out_scale):
        v = _f32(np.concatenate([in_mean, in_scale, out_mean, out_scale]))
        _check(lib().tc_mlp_set_normalization(self._h, v.ctypes.data_as(_F), v.size))

    def fit_normalization(self, x_dev, y_dev, n):
        """Normalization from a device training set (pointers to [n][20] and [n][19] FP32)."""
        _check(lib().tc_mlp_fit_normalization(self._h, _P(x_dev), _P(y_dev), n))

    def normalization(self):
        v = np.empty(2 * self.N_IN + 2 * self.N_OUT, dtype=np.float32)
        _check(lib().tc_mlp_get_normalization(self._h, v.ctypes.data_as(_F), v.size))
        return v

    def set_gemm(self, impl):
        _check(lib().tc_mlp_set_gemm(self._h, impl))

    def forward(self, x):
        x = _f32(x).reshape(-1, self.N_IN)
        y = np.empty((x.shape[0], self.N_OUT), dtype=np.float32)
        _check(lib().tc_mlp_forward(self._h, x.ctypes.data_as(_F), x.shape[0], y.ctypes.data_as(_F)))
        return y

    def gradients(self, x, t):
        x = _f32(x).reshape(-1, self.N_IN)
        t = _f32(t).reshape(-1, self.N_OUT)
        g = np.empty(self.n_params, dtype=np.float32)
        loss = C.c_float()
        _check(lib().tc_mlp_gradients(self._h, x.ctypes.data_as(_F), t.ctypes.data_as(_F), x.shape[0],
                                      g.ctypes.data_as(_F), C.byref(loss)))
        return loss.value, g

    def train(self, x_dev, y_dev, n, epochs, batch, lr, seed=0, stream=None):
        """x_dev, y_dev: device pointers of [n][20] and [n][19] FP32 (e.g. torch data_ptr())."""
        hist = np.zeros(epochs, dtype=np.float32)
        _check(lib().tc_mlp_train(self._h, _P(x_dev), _P(y_dev), n, epochs, batch, lr, seed,
                                  None if stream is None else _P(int(stream)), hist.ctypes.data_as(_F)))
        return hist

    def close(self):
        if getattr(self, "_h", None):
            lib().tc_mlp_destroy(self._h)
            self._h = None

    __del__ = close


def tp06_window(in_ptr, istim_ptr, n, dt, nsub, cell, precision=TC_FP64, out_ptr=None, stream=None):
    """Exact single-cell windows on device arrays ([19][n] in and out, istim [n] or None)."""
    _check(lib().tc_tp06_window(_P(in_ptr), None if istim_ptr is None else _P(istim_ptr), n, dt, nsub, cell,
                                precision, _P(out_ptr), None if stream is None else _P(int(stream))))


def gemm_bf16_nt(a_ptr, b_ptr, c_ptr, M, N, K, stream=None):
    """c [M][N] = a [M][K] . b [N][K]^T on the tensor cores (device pointers; BF16 in, FP32 out)."""
    _check(lib().tc_gemm_bf16_nt(_P(a_ptr), _P(b_ptr), _P(c_ptr), M, N, K,
                                 None if stream is None else _P(int(stream))))


def monodomain_conductivity(il, it, el, et):
    """Per-region monodomain (sigma_l, sigma_t) from intra-/extracellular conductivities (S/m)."""
    il, it, el, et = (_f64(v) for v in (il, it, el, et))
    sl, st = np.empty_like(il), np.empty_like(il)
    _check(lib().tc_monodomain_conductivity(_d(il), _d(it), _d(el), _d(et), il.size, _d(sl), _d(st)))
    return sl, st


def selftest_log(x):
    """(device log used by the ionic kernels, CUDA library log) at x."""
    x = _f64(x)
    a = np.empty_like(x)
    b = np.empty_like(x)
    _check(lib().tc_selftest_log(_d(x), _d(a), _d(b), x.size))
    return a, b


def selftest_rcp(x):
    """(device reciprocal used by the ionic kernels, IEEE 1.0 / x) at x."""
    x = _f64(x)
    a = np.empty_like(x)
    b = np.empty_like(x)
    _check(lib().tc_selftest_rcp(_d(x), _d(a), _d(b), x.size))
    return a, b


def selftest_exp2(x):
    """(device base-2 exponential used by the ionic kernels, CUDA library exp2) at x."""
    x = _f64(x)
    a = np.empty_like(x)
    b = np.empty_like(x)
    _check(lib().tc_selftest_exp2(_d(x), _d(a), _d(b), x.size))
    return a, b


def selftest_exp(x):
    """(device exp used by the ionic kernels, CUDA library exp) at x."""
    x = _f64(x)
    a = np.empty_like(x)
    b = np.empty_like(x)
    _check(lib().tc_selftest_exp(_d(x), _d(a), _d(b), x.size))
    return a, b


def from_workload(w, stream=None, precision=TC_FP64, mesh=None):
    """Build a Simulation from an ``inputs.Workload`` (mesh, tissue, model, stimuli, solver);
    `mesh` may pass an already created Mesh of w.mesh (e.g. with a chosen SELL window)."""
    mesh = Mesh.from_inputs(w.mesh) if mesh is None else mesh
    sim = Simulation(mesh, w.sigma_l, w.sigma_t, w.chi, w.cm, w.theta, w.dt, precision, stream)
    sim.mesh = mesh
    sim.set_activation_threshold(w.v_threshold)
    set_model(sim, w)
    for s in w.stimuli:
        sim.add_stimulus(s.nodes, s.start, s.duration, s.intensity)
    sim.set_solver(w.atol, w.rtol, w.max_iter)
    return sim


def measure_fp64_rate():
    """tc_measure_fp64_rate: FP64 FMA instructions per second the current device sustains."""
    v = C.c_double()
    _check(lib().tc_measure_fp64_rate(C.byref(v)))
    return v.value
