"""Python binding of libsvm (include/svm.h): argument marshalling only.

Every function here has the name of the C entry point it calls and passes
its arguments through ctypes: device buffers are torch CUDA tensors (their
``data_ptr()``), host arrays are numpy arrays, the stream is a
``torch.cuda.Stream`` (default: the current stream).  All computation runs in
the library's CUDA kernels; there is no CPU fallback, and importing a
function raises if ``libsvm.so`` has not been built (``build()``).
"""
from __future__ import annotations

import ctypes as C
import os
import platform
import struct

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", platform.machine(), "libsvm.so")

SVM_OK, SVM_E_INVALID, SVM_E_CUDA, SVM_E_OOM, SVM_E_TIMEOUT, SVM_E_WEIGHTS, SVM_E_UNSUPPORTED = range(7)
SVM_FP32, SVM_BF16, SVM_FP8_E4M3 = 0, 1, 2
SVM_RELU, SVM_SILU = 0, 1
SVM_STRICT, SVM_NO_EARLY_EXIT, SVM_VERIFY_ALL, SVM_PATHS3, SVM_PREDICT_ONLY, SVM_PATHS2 = 1, 2, 4, 8, 16, 32
SVM_SEARCH_GCC0, SVM_SEARCH_SORTED, SVM_SEARCH_PATHS2, SVM_SEARCH_PATHS3 = 1, 2, 4, 8

RESULT_DTYPE = np.dtype([("collision", "u1"), ("early_exit", "u1"), ("status", "<u2"),
                         ("d_min", "<f4"), ("dhat_min", "<f4"), ("n_flagged", "<u4"),
                         ("n_verified", "<u4"), ("witness_point", "<i4"), ("witness_step", "<i4"),
                         ("n_ambiguous", "<u4")])
assert RESULT_DTYPE.itemsize == 32


class svm_model_desc(C.Structure):
    _fields_ = [("dh", (C.c_double * 4) * 6), ("radius", C.c_double * 7), ("tool_len", C.c_double),
                ("width", C.c_int32), ("n_hidden", C.c_int32), ("act", C.c_int32), ("prec", C.c_int32),
                ("arch", C.c_int32)]


class SvmError(RuntimeError):
    def __init__(self, fn, status, text):
        super().__init__(f"{fn} failed: status {status} ({text})")
        self.status = status


_lib = None


def build() -> str:
    """Compile libsvm.so for sm_103a (nvcc, in-tree)."""
    from . import buildlib
    return buildlib.build()


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libsvm.so not built ({LIB_PATH}); run paper_2402_15281_gb300.build()")
        L = C.CDLL(LIB_PATH)
        vp, i32, i64, u32, f32, sz = C.c_void_p, C.c_int32, C.c_int64, C.c_uint32, C.c_float, C.c_size_t
        L.svm_status_string.argtypes = [C.c_int]
        L.svm_status_string.restype = C.c_char_p
        L.svm_last_error.argtypes = [vp]
        L.svm_last_error.restype = C.c_char_p
        L.svm_create_model.argtypes = [C.POINTER(svm_model_desc), C.c_int, C.POINTER(vp)]
        L.svm_destroy_model.argtypes = [vp]
        L.svm_load_weights.argtypes = [vp, C.c_char_p, sz]
        L.svm_export_weights.argtypes = [vp, vp, sz, C.POINTER(sz)]
        L.svm_set_gate.argtypes = [vp, f32]
        L.svm_test_set_tie_cap.argtypes = [vp, i32]
        L.svm_set_act_scales.argtypes = [vp, vp, i32]
        L.svm_check_motions.argtypes = [vp, vp, vp, i32, vp, i64, f32, i32, u32, vp, vp]
        L.svm_check_batch.argtypes = [vp, vp, vp, i32, vp, vp, vp, i32, f32, i32, u32, vp, vp]
        L.svm_eval_pairs.argtypes = [vp, vp, vp, i32, vp, i64, vp, vp]
        L.svm_label_pairs.argtypes = [vp, vp, vp, i32, vp, i64, i32, vp, vp]
        L.svm_plan_create.argtypes = [vp, vp, vp, i32, vp, vp, i32, f32, i32, u32, C.POINTER(vp)]
        L.svm_plan_destroy.argtypes = [vp]
        L.svm_plan_launch.argtypes = [vp, vp, vp, vp]
        L.svm_plan_graph_launch.argtypes = [vp, vp, vp, vp]
        L.svm_plan_set_verify_shape.argtypes = [vp, i32, i32]
        L.svm_plan_set_network_grid.argtypes = [vp, i32]
        L.svm_plan_autotune.argtypes = [vp, vp, vp, vp, C.c_char_p, sz]
        for f in ("svm_plan_create", "svm_plan_destroy", "svm_plan_launch", "svm_plan_graph_launch",
                  "svm_plan_set_verify_shape", "svm_plan_autotune"):
            getattr(L, f).restype = C.c_int
        L.svm_calibrate_act_scales.argtypes = [vp, vp, vp, i32, vp, i64, f32, vp]
        L.svm_calibrate_act_scales.restype = C.c_int
        L.svm_calibrate_gate.argtypes = [vp, vp, vp, i32, vp, i64, f32, i32, f32, f32, vp, vp, vp, vp]
        L.svm_calibrate_gate.restype = C.c_int
        L.svm_check_motions_noalloc.argtypes = [vp, vp, vp, i32, vp, i64, f32, i32, u32, vp, vp]
        L.svm_check_motions_noalloc.restype = C.c_int
        L.svm_train_create.argtypes = [C.POINTER(svm_model_desc), C.c_int, i32, C.POINTER(vp)]
        L.svm_train_destroy.argtypes = [vp]
        L.svm_train_last_error.argtypes = [vp]
        L.svm_train_last_error.restype = C.c_char_p
        L.svm_train_param_count.argtypes = [vp]
        L.svm_train_param_count.restype = C.c_int64
        L.svm_train_set_weights.argtypes = [vp, C.c_char_p, sz]
        L.svm_train_get_weights.argtypes = [vp, vp, sz, C.POINTER(sz)]
        L.svm_train_make_data.argtypes = [vp, vp, vp, i32, i32, i32, C.c_uint64]
        L.svm_train_set_box.argtypes = [vp, vp, vp]
        L.svm_train_set_box.restype = C.c_int
        L.svm_train_set_samples.argtypes = [vp, vp, vp, i32, vp, vp, i64]
        L.svm_train_copy_samples.argtypes = [vp, vp, vp, i64]
        L.svm_train_gradient.argtypes = [vp, i64, vp, vp]
        L.svm_train_adam.argtypes = [vp, f32]
        L.svm_train_epoch.argtypes = [vp, i64, i64, f32, C.c_uint64, vp]
        L.svm_train_evaluate.argtypes = [vp, i64, i64, vp]
        L.svm_train_state.argtypes = [vp, vp, vp, vp, vp, i64]
        L.svm_train_restore.argtypes = [vp, vp, vp, vp, i64, i64]
        for f in ("svm_train_create", "svm_train_destroy", "svm_train_set_weights", "svm_train_get_weights",
                  "svm_train_make_data", "svm_train_set_samples", "svm_train_copy_samples", "svm_train_gradient",
                  "svm_train_adam", "svm_train_epoch", "svm_train_evaluate", "svm_train_state",
                  "svm_train_restore"):
            getattr(L, f).restype = C.c_int
        L.svm_search_free_motion.argtypes = [vp, vp, vp, i32, vp, i64, f32, i32, i32, u32,
                                             C.POINTER(svm_search_result), vp]
        L.svm_search_free_motion.restype = C.c_int
        L.svm_test_expire_wait.argtypes = [vp, i32]
        L.svm_test_expire_wait.restype = C.c_int
        L.svm_profile_enable.argtypes = [vp, C.c_int]
        L.svm_profile_read.argtypes = [vp, vp, i32]
        for f in ("svm_profile_enable", "svm_profile_read", "svm_create_model", "svm_destroy_model", "svm_load_weights", "svm_export_weights",
                  "svm_set_gate", "svm_set_act_scales", "svm_check_motions", "svm_check_batch",
                  "svm_eval_pairs", "svm_label_pairs"):
            getattr(L, f).restype = C.c_int
        _lib = L
    return _lib


def _check(fn, status, model=None):
    if status != SVM_OK:
        text = lib().svm_status_string(status).decode()
        if model is not None:
            text += ": " + lib().svm_last_error(model).decode()
        raise SvmError(fn, status, text)


def _stream(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _host_f64(a, cols=6):
    a = np.ascontiguousarray(a, dtype=np.float64).reshape(-1, cols)
    return a, a.ctypes.data_as(C.c_void_p)


def _dev(t):
    if t is None:
        return C.c_void_p(0)
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("device arguments must be contiguous CUDA tensors")
    return C.c_void_p(t.data_ptr())


def _points(t):
    """A point cloud: contiguous (P, 4) float32 CUDA tensor."""
    if t.dtype != _torch().float32 or t.dim() != 2 or t.shape[1] != 4:
        raise ValueError("points must be a (P, 4) float32 CUDA tensor")
    return _dev(t)


def _out(t, nbytes, what):
    """An output buffer the call writes `nbytes` into (checked before the
    launch: a short buffer would be overrun on the device)."""
    have = t.numel() * t.element_size()
    if have < nbytes:
        raise ValueError(f"{what} holds {have} bytes; the call writes {nbytes}")
    return _dev(t)


def _n_records(n_motions, flags):
    """Result records a check call writes: one per motion, or per path."""
    return n_motions // 3 if flags & SVM_PATHS3 else n_motions // 2 if flags & SVM_PATHS2 else n_motions


# ------------------------------------------------------------------ entry points

SVM_ARCH_MLP, SVM_ARCH_BLOCKS = 0, 1


def svm_create_model(robot, width=256, n_hidden=4, act=SVM_RELU, prec=SVM_FP32, device=0, arch=SVM_ARCH_MLP):
    d = svm_model_desc()
    for j in range(6):
        for c in range(4):
            d.dh[j][c] = float(robot.dh[j, c])
    for j in range(7):
        d.radius[j] = float(robot.radius[j])
    d.tool_len = float(robot.tool_len)
    d.width, d.n_hidden, d.act, d.prec, d.arch = int(width), int(n_hidden), int(act), int(prec), int(arch)
    h = C.c_void_p()
    _check("svm_create_model", lib().svm_create_model(C.byref(d), int(device), C.byref(h)))
    return h


def svm_destroy_model(model):
    _check("svm_destroy_model", lib().svm_destroy_model(model))


def make_blob(layers, act=SVM_RELU, tau=float("inf")) -> bytes:
    """Serialise [(W, b), ...] (15 -> W, ..., W -> 1) in the blob format of svm_load_weights."""
    width = layers[0][0].shape[0]
    out = [b"SVMW", struct.pack("<IIIIIf", 1, len(layers), 15, width, act, tau)]
    for W, b in layers:
        W = np.ascontiguousarray(W, dtype="<f4")
        b = np.ascontiguousarray(b, dtype="<f4")
        out.append(struct.pack("<II", W.shape[0], W.shape[1]))
        out.append(W.tobytes())
        out.append(b.tobytes())
    return b"".join(out)


def make_block_blob(params, tau=float("inf"), bn_eps=1e-5) -> bytes:
    """Serialise the block architecture (synth.block_weights layout) in the
    version-2 blob format of svm_load_weights."""
    W0, b0 = params["init"]
    width = W0.shape[0]
    f4 = lambda a: np.ascontiguousarray(a, dtype="<f4").tobytes()
    out = [b"SVMW", struct.pack("<IIIIIff", 2, len(params["blocks"]), 15, width, SVM_RELU, tau, bn_eps)]
    out += [struct.pack("<II", *W0.shape), f4(W0), f4(b0)]
    for (W, b, gamma, beta, mean, var) in params["blocks"]:
        out += [struct.pack("<II", *W.shape), f4(W), f4(b), f4(gamma), f4(beta), f4(mean), f4(var)]
    Wf, bf = params["final"]
    out += [struct.pack("<II", *Wf.shape), f4(Wf), f4(bf)]
    return b"".join(out)


def parse_blob(blob: bytes):
    """[(W, b), ...] of a weight blob (inverse of make_blob)."""
    n_layers = struct.unpack("<I", blob[8:12])[0]
    off, out = 28, []
    for _ in range(n_layers):
        o, i = struct.unpack("<II", blob[off:off + 8])
        off += 8
        W = np.frombuffer(blob, "<f4", o * i, off).reshape(o, i).copy()
        off += 4 * o * i
        b = np.frombuffer(blob, "<f4", o, off).copy()
        off += 4 * o
        out.append((W, b))
    return out


def svm_load_weights(model, blob: bytes):
    _check("svm_load_weights", lib().svm_load_weights(model, blob, len(blob)), model)


def svm_export_weights(model) -> np.ndarray:
    need = C.c_size_t()
    _check("svm_export_weights", lib().svm_export_weights(model, None, 0, C.byref(need)), model)
    out = np.zeros(need.value, dtype=np.float32)
    _check("svm_export_weights", lib().svm_export_weights(model, out.ctypes.data_as(C.c_void_p),
                                                          out.shape[0], None), model)
    return out


def svm_test_expire_wait(model, n_calls: int = 1):
    _check("svm_test_expire_wait", lib().svm_test_expire_wait(model, int(n_calls)), model)


def svm_test_set_tie_cap(model, cap: int):
    _check("svm_test_set_tie_cap", lib().svm_test_set_tie_cap(model, int(cap)), model)


def svm_set_gate(model, tau: float):
    _check("svm_set_gate", lib().svm_set_gate(model, float(tau)), model)


def svm_set_act_scales(model, scales):
    s = np.ascontiguousarray(scales, dtype=np.float32)
    _check("svm_set_act_scales", lib().svm_set_act_scales(model, s.ctypes.data_as(C.c_void_p), s.shape[0]), model)


def svm_calibrate_act_scales(model, q0, q1, points_dev, headroom=2.0) -> np.ndarray:
    """FP8: set (and return) the per-layer activation scales from data."""
    q0, p0 = _host_f64(q0)
    q1, p1 = _host_f64(q1)
    out = np.zeros(64, dtype=np.float32)
    _check("svm_calibrate_act_scales", lib().svm_calibrate_act_scales(
        model, p0, p1, q0.shape[0], _dev(points_dev), points_dev.shape[0], float(headroom),
        out.ctypes.data_as(C.c_void_p)), model)
    return out


def svm_calibrate_gate(model, q0, q1, points_dev, margin, steps, band=0.05, safety=1.25, stream=None):
    """Set the gate from calibration motions (host (M, 6)) against a device
    cloud; returns (tau, largest overestimate, number of near pairs)."""
    q0, p0 = _host_f64(q0)
    q1, p1 = _host_f64(q1)
    tau, over, n_near = C.c_float(0.0), C.c_float(0.0), C.c_int64(0)
    _check("svm_calibrate_gate", lib().svm_calibrate_gate(
        model, p0, p1, q0.shape[0], _points(points_dev), points_dev.shape[0], float(margin), int(steps),
        float(band), float(safety), C.byref(tau), C.byref(over), C.byref(n_near), _stream(stream)), model)
    return float(tau.value), float(over.value), int(n_near.value)


def svm_check_motions(model, q0, q1, points_dev, margin, steps, flags, results_dev, stream=None):
    """q0, q1: host (M, 6); points_dev: CUDA float32 (P, 4); results_dev: CUDA uint8 (M, 32)."""
    q0, p0 = _host_f64(q0)
    q1, p1 = _host_f64(q1)
    _check("svm_check_motions", lib().svm_check_motions(
        model, p0, p1, q0.shape[0], _points(points_dev), points_dev.shape[0], float(margin), int(steps),
        int(flags), _out(results_dev, 32 * _n_records(q0.shape[0], int(flags)), "results"), _stream(stream)),
        model)


def svm_check_motions_noalloc(model, q0_dev, q1_dev, points_dev, margin, steps, flags, results_dev, stream=None):
    """Allocation-free check: q0_dev, q1_dev are CUDA float64 (M, 6) tensors."""
    if q0_dev.dtype != _torch().float64 or q1_dev.dtype != _torch().float64:
        raise ValueError("q0_dev and q1_dev must be float64 CUDA tensors")
    if q0_dev.shape != q1_dev.shape or q0_dev.shape[-1] != 6:
        raise ValueError("q0_dev and q1_dev must both be (M, 6)")
    _check("svm_check_motions_noalloc", lib().svm_check_motions_noalloc(
        model, _dev(q0_dev), _dev(q1_dev), q0_dev.shape[0], _points(points_dev), points_dev.shape[0],
        float(margin), int(steps), int(flags), _out(results_dev, 32 * _n_records(q0_dev.shape[0], int(flags)),
                                                    "results"), _stream(stream)), model)


def _torch():
    import torch
    return torch


class svm_search_result(C.Structure):
    _fields_ = [("motion", C.c_int32), ("loop", C.c_int32), ("delta", C.c_float), ("delta_hat", C.c_float),
                ("n_exact", C.c_int32), ("n_exact_run", C.c_int32), ("n_nn", C.c_int32),
                ("n_nn_seq", C.c_int32)]


def svm_search_free_motion(model, q0, q1, points_dev, margin, steps, wave=1, flags=0, stream=None):
    """Algorithm 1: the first collision-free motion found with the network as a
    proxy (flags = SVM_SEARCH_GCC0: exact checks in the given order).  Returns a
    dict of the svm_search_result fields."""
    q0, p0 = _host_f64(q0)
    q1, p1 = _host_f64(q1)
    out = svm_search_result()
    _check("svm_search_free_motion", lib().svm_search_free_motion(
        model, p0, p1, q0.shape[0], _points(points_dev), points_dev.shape[0], float(margin), int(steps),
        int(wave), int(flags), C.byref(out), _stream(stream)), model)
    return {f: getattr(out, f) for f, _ in svm_search_result._fields_}


def svm_check_batch(model, q0, q1, motion_scene, points_dev, scene_offsets, margin, steps, flags,
                    results_dev, stream=None):
    q0, p0 = _host_f64(q0)
    q1, p1 = _host_f64(q1)
    ms = np.ascontiguousarray(motion_scene, dtype=np.int32)
    so = np.ascontiguousarray(scene_offsets, dtype=np.int64)
    _check("svm_check_batch", lib().svm_check_batch(
        model, p0, p1, q0.shape[0], ms.ctypes.data_as(C.c_void_p), _points(points_dev),
        so.ctypes.data_as(C.c_void_p), so.shape[0] - 1, float(margin), int(steps), int(flags),
        _out(results_dev, 32 * _n_records(q0.shape[0], int(flags)), "results"), _stream(stream)), model)


class Plan:
    """A prepared batch (svm_plan_*); `model` must stay alive."""

    def __init__(self, model, q0, q1, motion_scene, scene_offsets, margin, steps, flags):
        q0, p0 = _host_f64(q0)
        q1, p1 = _host_f64(q1)
        ms = np.ascontiguousarray(motion_scene, dtype=np.int32)
        so = np.ascontiguousarray(scene_offsets, dtype=np.int64)
        self.model = model
        self.n_records = _n_records(q0.shape[0], int(flags))
        self.h = C.c_void_p()
        _check("svm_plan_create", lib().svm_plan_create(
            model, p0, p1, q0.shape[0], ms.ctypes.data_as(C.c_void_p), so.ctypes.data_as(C.c_void_p),
            so.shape[0] - 1, float(margin), int(steps), int(flags), C.byref(self.h)), model)

    def _bufs(self, points_dev, results_dev):
        return _points(points_dev), _out(results_dev, 32 * self.n_records, "results")

    def launch(self, points_dev, results_dev, stream=None):
        _check("svm_plan_launch", lib().svm_plan_launch(self.h, *self._bufs(points_dev, results_dev),
                                                        _stream(stream)), self.model)

    def graph_launch(self, points_dev, results_dev, stream):
        _check("svm_plan_graph_launch", lib().svm_plan_graph_launch(self.h, *self._bufs(points_dev, results_dev),
                                                                    _stream(stream)), self.model)

    def set_verify_shape(self, points_per_thread, ctas_per_sm):
        _check("svm_plan_set_verify_shape", lib().svm_plan_set_verify_shape(self.h, int(points_per_thread),
                                                                            int(ctas_per_sm)), self.model)

    def set_network_grid(self, ctas):
        _check("svm_plan_set_network_grid", lib().svm_plan_set_network_grid(self.h, int(ctas)), self.model)

    def autotune(self, points_dev, results_dev, stream=None) -> str:
        buf = C.create_string_buffer(4096)
        _check("svm_plan_autotune", lib().svm_plan_autotune(self.h, *self._bufs(points_dev, results_dev),
                                                            _stream(stream), buf, 4096), self.model)
        return buf.value.decode()

    def close(self):
        if self.h:
            _check("svm_plan_destroy", lib().svm_plan_destroy(self.h))
            self.h = C.c_void_p()


def svm_eval_pairs(model, q0, q1, points_dev, f_dev, stream=None):
    q0, p0 = _host_f64(q0)
    q1, p1 = _host_f64(q1)
    _check("svm_eval_pairs", lib().svm_eval_pairs(
        model, p0, p1, q0.shape[0], _points(points_dev), points_dev.shape[0],
        _out(f_dev, 4 * q0.shape[0] * points_dev.shape[0], "f"), _stream(stream)), model)


def svm_label_pairs(model, q0, q1, points_dev, steps, delta_dev, stream=None):
    q0, p0 = _host_f64(q0)
    q1, p1 = _host_f64(q1)
    _check("svm_label_pairs", lib().svm_label_pairs(
        model, p0, p1, q0.shape[0], _points(points_dev), points_dev.shape[0], int(steps),
        _out(delta_dev, 4 * q0.shape[0] * points_dev.shape[0], "delta"), _stream(stream)), model)


def svm_profile_enable(model, on=True):
    _check("svm_profile_enable", lib().svm_profile_enable(model, int(bool(on))), model)


def svm_profile_read(model, n=4) -> np.ndarray:
    """Phase durations (ms) of the last profiled check call."""
    out = np.zeros(n, dtype=np.float32)
    _check("svm_profile_read", lib().svm_profile_read(model, out.ctypes.data_as(C.c_void_p), n), model)
    return out


def results_to_numpy(results_dev) -> np.ndarray:
    """Copy result records (CUDA uint8 tensor of n x 32 bytes) to a structured numpy array."""
    raw = results_dev.cpu().numpy().reshape(-1)
    return raw.view(RESULT_DTYPE)


def new_results(n, device="cuda"):
    import torch
    return torch.empty((max(n, 1), 32), dtype=torch.uint8, device=device)


# ------------------------------------------------------------------ training

def _tcheck(fn, status, trainer=None):
    if status != SVM_OK:
        text = lib().svm_status_string(status).decode()
        if trainer is not None:
            text += ": " + lib().svm_train_last_error(trainer).decode()
        raise SvmError(fn, status, text)


def _desc(robot, width, n_hidden, act, prec=SVM_FP32):
    d = svm_model_desc()
    for j in range(6):
        for c in range(4):
            d.dh[j][c] = float(robot.dh[j, c])
    for j in range(7):
        d.radius[j] = float(robot.radius[j])
    d.tool_len = float(robot.tool_len)
    d.width, d.n_hidden, d.act, d.prec = int(width), int(n_hidden), int(act), int(prec)
    return d


def svm_train_create(robot, width, n_hidden, act, batch, device=0):
    d = _desc(robot, width, n_hidden, act)
    h = C.c_void_p()
    _tcheck("svm_train_create", lib().svm_train_create(C.byref(d), int(device), int(batch), C.byref(h)))
    return h


def svm_train_destroy(t):
    _tcheck("svm_train_destroy", lib().svm_train_destroy(t))


def svm_train_param_count(t) -> int:
    return int(lib().svm_train_param_count(t))


def svm_train_set_weights(t, blob: bytes):
    _tcheck("svm_train_set_weights", lib().svm_train_set_weights(t, blob, len(blob)), t)


def svm_train_get_weights(t) -> bytes:
    need = C.c_size_t()
    _tcheck("svm_train_get_weights", lib().svm_train_get_weights(t, None, 0, C.byref(need)), t)
    buf = C.create_string_buffer(need.value)
    _tcheck("svm_train_get_weights", lib().svm_train_get_weights(t, buf, need.value, None), t)
    return buf.raw


def svm_train_make_data(t, q0, q1, samples_per_motion, steps, seed):
    q0, p0 = _host_f64(q0)
    q1, p1 = _host_f64(q1)
    _tcheck("svm_train_make_data", lib().svm_train_make_data(t, p0, p1, q0.shape[0], int(samples_per_motion),
                                                             int(steps), int(seed)), t)


def svm_train_set_box(t, lo, hi):
    lo = np.ascontiguousarray(lo, dtype=np.float64).reshape(3)
    hi = np.ascontiguousarray(hi, dtype=np.float64).reshape(3)
    _tcheck("svm_train_set_box", lib().svm_train_set_box(t, lo.ctypes.data_as(C.c_void_p),
                                                         hi.ctypes.data_as(C.c_void_p)), t)


def svm_train_set_samples(t, q0, q1, x4, motion):
    q0, p0 = _host_f64(q0)
    q1, p1 = _host_f64(q1)
    x4 = np.ascontiguousarray(x4, dtype=np.float32).reshape(-1, 4)
    mo = np.ascontiguousarray(motion, dtype=np.int32)
    _tcheck("svm_train_set_samples", lib().svm_train_set_samples(
        t, p0, p1, q0.shape[0], x4.ctypes.data_as(C.c_void_p), mo.ctypes.data_as(C.c_void_p), x4.shape[0]), t)


def svm_train_copy_samples(t, n):
    x4 = np.zeros((n, 4), dtype=np.float32)
    mo = np.zeros(n, dtype=np.int32)
    _tcheck("svm_train_copy_samples", lib().svm_train_copy_samples(
        t, x4.ctypes.data_as(C.c_void_p), mo.ctypes.data_as(C.c_void_p), n), t)
    return x4, mo


def svm_train_gradient(t, sample_begin=0):
    g = np.zeros(svm_train_param_count(t), dtype=np.float32)
    loss = C.c_float()
    _tcheck("svm_train_gradient", lib().svm_train_gradient(t, int(sample_begin), g.ctypes.data_as(C.c_void_p),
                                                           C.byref(loss)), t)
    return g, loss.value


def svm_train_adam(t, lr):
    _tcheck("svm_train_adam", lib().svm_train_adam(t, float(lr)), t)


def svm_train_epoch(t, begin, end, lr, shuffle_seed) -> float:
    loss = C.c_float()
    _tcheck("svm_train_epoch", lib().svm_train_epoch(t, int(begin), int(end), float(lr), int(shuffle_seed),
                                                     C.byref(loss)), t)
    return loss.value


def svm_train_evaluate(t, begin, end) -> float:
    mae = C.c_float()
    _tcheck("svm_train_evaluate", lib().svm_train_evaluate(t, int(begin), int(end), C.byref(mae)), t)
    return mae.value


def svm_train_state(t):
    n = svm_train_param_count(t)
    P, M1, M2 = (np.zeros(n, dtype=np.float32) for _ in range(3))
    step = C.c_int64()
    _tcheck("svm_train_state", lib().svm_train_state(t, P.ctypes.data_as(C.c_void_p), M1.ctypes.data_as(C.c_void_p),
                                                     M2.ctypes.data_as(C.c_void_p), C.byref(step), n), t)
    return P, M1, M2, step.value


def svm_train_restore(t, P, M1, M2, step):
    P, M1, M2 = (np.ascontiguousarray(a, dtype=np.float32) for a in (P, M1, M2))
    _tcheck("svm_train_restore", lib().svm_train_restore(t, P.ctypes.data_as(C.c_void_p), M1.ctypes.data_as(C.c_void_p),
                                                         M2.ctypes.data_as(C.c_void_p), int(step), P.shape[0]), t)
