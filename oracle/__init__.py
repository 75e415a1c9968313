"""Python access to the FP64 CPU oracle (``svm_oracle.c``), and Algorithm 1
(the motion search of Sec. IV-B) written out in plain Python on top of it.

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's
CPU-baseline leg use this module to state what the GPU path must compute.
The CUDA library never imports it, and it never imports the CUDA library.

Every function takes and returns numpy arrays in float64 (points as (n, 3)).
``build()`` compiles the C source with gcc and OpenMP; it runs on first use.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "svm_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lib = None

DOF = 6
NCAPS = 7


def build(force: bool = False) -> str:
    """Compile the oracle (plain C, -O2, no fast-math, no FMA contraction)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-std=gnu11", "-O2", "-fPIC", "-shared", "-fopenmp",
               "-ffp-contract=off", "-fno-fast-math", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_D = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_F = np.ctypeslib.ndpointer(dtype=np.float32, flags="C_CONTIGUOUS")
_I32 = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_I64 = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        L = _lib
        L.orc_num_threads.restype = C.c_int
        L.orc_set_num_threads.argtypes = [C.c_int]
        L.orc_fk.argtypes = [_D, _D, _D]
        L.orc_capsules.argtypes = [_D, C.c_double, _D, _D, _D]
        L.orc_point_capsule.argtypes = [_D, _D, _D, C.c_double]
        L.orc_point_capsule.restype = C.c_double
        L.orc_robot_sdf.argtypes = [_D, C.c_double, _D, _D, _D]
        L.orc_robot_sdf.restype = C.c_double
        L.orc_swept_sdf.argtypes = [_D, C.c_double, _D, _D, _D, C.c_int, _D]
        L.orc_swept_sdf.restype = C.c_double
        L.orc_swept_sdf_batch.argtypes = [_D, C.c_double, _D, _D, _D, C.c_int, C.c_int, _D, C.c_long, _D]
        L.orc_gcc_motion.argtypes = [_D, C.c_double, _D, _D, _D, C.c_int, C.c_int, _D, C.c_long,
                                     C.c_double, _D, _I32]
        L.orc_param_count.argtypes = [C.c_int, C.c_int]
        L.orc_param_count.restype = C.c_long
        L.orc_mlp_forward.argtypes = [_D, C.c_int, C.c_int, C.c_int, _D, C.c_long, _D]
        L.orc_mlp_pairs.argtypes = [_D, C.c_int, C.c_int, C.c_int, _D, _D, C.c_int, _D, C.c_long, _D]
        L.orc_mlp_pairs_rounded.argtypes = [_D, C.c_int, C.c_int, C.c_int, C.c_int, _D, _D, _D, C.c_int,
                                            _D, C.c_long, _D]
        L.orc_mlp_forward_rounded.argtypes = [_D, C.c_int, C.c_int, C.c_int, _I32, _D, _D, C.c_long, _D]
        L.orc_mlp_loss_grad.argtypes = [_D, C.c_int, C.c_int, C.c_int, _D, _D, C.c_long, _D]
        L.orc_mlp_loss_grad.restype = C.c_double
        L.orc_mlp_loss_grad_bf16.argtypes = [_D, C.c_int, C.c_int, C.c_int, _D, _D, C.c_long, _D]
        L.orc_mlp_loss_grad_bf16.restype = C.c_double
        L.orc_adam_step.argtypes = [_D, _D, _D, _D, C.c_long, C.c_long, C.c_double, C.c_double,
                                    C.c_double, C.c_double]
        L.orc_check_motions.argtypes = [_D, C.c_int, C.c_int, C.c_int, _D, C.c_double, _D,
                                        _D, _D, C.c_int, C.c_int, _D, C.c_long, C.c_double,
                                        C.c_double, C.c_int, C.c_void_p, _I32, _D, _D, _I64]
        L.orc_round_bf16.argtypes = [C.c_float]
        L.orc_round_bf16.restype = C.c_float
        L.orc_round_bf16_array.argtypes = [_F, C.c_long]
        L.orc_round_e4m3.argtypes = [C.c_double]
        L.orc_round_e4m3.restype = C.c_double
        L.orc_quantize_e4m3.argtypes = [_F, C.c_long, _F]
        L.orc_quantize_e4m3.restype = C.c_float
        L.orc_training_points.argtypes = [_D, C.c_double, _D, _D, _D, C.c_int, C.c_uint64, C.c_int, C.c_int, _D]
        L.orc_training_points_region.argtypes = [_D, C.c_double, _D, _D, _D, C.c_int, C.c_uint64, C.c_int,
                                                 C.c_int, _D, _D, _D]
        L.orc_splitmix64_u01.argtypes = [C.c_uint64, C.c_uint64, C.c_uint64]
        L.orc_splitmix64_u01.restype = C.c_double
    return _lib


def _d(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def num_threads() -> int:
    return lib().orc_num_threads()


def set_num_threads(n: int) -> None:
    lib().orc_set_num_threads(int(n))


# ----------------------------------------------------------------- robot

class RobotArrays:
    """The oracle's view of a robot: DH table, radii, tool length."""

    def __init__(self, robot):
        self.dh = _d(robot.dh).reshape(6, 4)
        self.radius = _d(robot.radius).reshape(7)
        self.tool_len = float(robot.tool_len)


def fk(robot, q) -> np.ndarray:
    """Frames T_0..T_6 as (7, 4, 4)."""
    R = RobotArrays(robot)
    T = np.zeros(7 * 16)
    lib().orc_fk(R.dh, _d(q), T)
    return T.reshape(7, 4, 4)


def capsules(robot, q):
    """Capsule axes (a, b), each (7, 3)."""
    R = RobotArrays(robot)
    a = np.zeros(21)
    b = np.zeros(21)
    lib().orc_capsules(R.dh, R.tool_len, _d(q), a, b)
    return a.reshape(7, 3), b.reshape(7, 3)


def point_capsule(x, a, b, r) -> float:
    return lib().orc_point_capsule(_d(x), _d(a), _d(b), float(r))


def robot_sdf(robot, q, x) -> float:
    R = RobotArrays(robot)
    return lib().orc_robot_sdf(R.dh, R.tool_len, R.radius, _d(q), _d(x))


def swept_sdf(robot, q0, q1, N, x) -> float:
    R = RobotArrays(robot)
    return lib().orc_swept_sdf(R.dh, R.tool_len, R.radius, _d(q0), _d(q1), int(N), _d(x))


def _xyz(points) -> np.ndarray:
    p = np.asarray(points)
    return _d(p[:, :3])


def swept_sdf_batch(robot, q0, q1, N, points) -> np.ndarray:
    """delta[m, i] for every motion m and point i (points (n, 3) or (n, 4))."""
    R = RobotArrays(robot)
    q0 = _d(q0).reshape(-1, 6)
    q1 = _d(q1).reshape(-1, 6)
    pts = _xyz(points)
    M, n = q0.shape[0], pts.shape[0]
    out = np.zeros(M * n)
    lib().orc_swept_sdf_batch(R.dh, R.tool_len, R.radius, q0, q1, M, int(N), pts, n, out)
    return out.reshape(M, n)


def gcc_motion(robot, q0, q1, N, points, eps):
    """Eq. 5 per motion: (dmin (M,), collision (M,) int32)."""
    R = RobotArrays(robot)
    q0 = _d(q0).reshape(-1, 6)
    q1 = _d(q1).reshape(-1, 6)
    pts = _xyz(points)
    M = q0.shape[0]
    dmin = np.zeros(M)
    coll = np.zeros(M, dtype=np.int32)
    lib().orc_gcc_motion(R.dh, R.tool_len, R.radius, q0, q1, M, int(N), pts, pts.shape[0],
                         float(eps), dmin, coll)
    return dmin, coll


# ------------------------------------------------------------------- MLP

def flatten_params(layers) -> np.ndarray:
    """[(W, b), ...] -> one float64 vector, W row-major then b per layer."""
    return np.concatenate([np.concatenate([_d(W).ravel(), _d(b).ravel()]) for W, b in layers])


def unflatten_params(P, width, n_hidden):
    """Inverse of flatten_params for the 15 -> W, L x (W -> W), W -> 1 net."""
    shapes = [(width, 15)] + [(width, width)] * n_hidden + [(1, width)]
    out, off = [], 0
    for (o, i) in shapes:
        W = P[off:off + o * i].reshape(o, i)
        off += o * i
        b = P[off:off + o]
        off += o
        out.append((W.copy(), b.copy()))
    return out


def quantized_params(layers, prec) -> np.ndarray:
    """Flat float64 parameters of [(W, b), ...] as a model of precision `prec`
    uses them, rounded by the oracle's own quantisers: 0 = FP32 (unchanged);
    1 = BF16 (every weight matrix to nearest-even bfloat16); 2 = FP8 (hidden
    matrices to E4M3 with scale max|W| / 448, first and last layers BF16).
    Biases are never rounded."""
    out = []
    n = len(layers)
    for li, (W, b) in enumerate(layers):
        W = np.ascontiguousarray(W, dtype=np.float32)
        if prec == 1 or (prec == 2 and (li == 0 or li == n - 1)):
            Wq = round_bf16(W)
        elif prec == 2:
            _, Wq = quantize_e4m3(W)
            Wq = Wq.reshape(W.shape)
        else:
            Wq = W
        out.append((Wq, np.asarray(b, dtype=np.float32)))
    return flatten_params(out)


def param_count(width, n_hidden) -> int:
    return int(lib().orc_param_count(width, n_hidden))


def mlp_forward(P, width, n_hidden, act, inputs) -> np.ndarray:
    inputs = _d(inputs).reshape(-1, 15)
    out = np.zeros(inputs.shape[0])
    lib().orc_mlp_forward(_d(P), width, n_hidden, act, inputs, inputs.shape[0], out)
    return out


def mlp_pairs(P, width, n_hidden, act, q0, q1, points) -> np.ndarray:
    """f_theta(x_i, q0_m, q1_m) for all pairs: (M, n)."""
    q0 = _d(q0).reshape(-1, 6)
    q1 = _d(q1).reshape(-1, 6)
    pts = _xyz(points)
    M, n = q0.shape[0], pts.shape[0]
    out = np.zeros(M * n)
    lib().orc_mlp_pairs(_d(P), width, n_hidden, act, q0, q1, M, pts, n, out)
    return out.reshape(M, n)


def mlp_pairs_rounded(P, width, n_hidden, act, fmt, scales, q0, q1, points) -> np.ndarray:
    """Like mlp_pairs, with the input of each hidden layer rounded to the
    activation format fmt (1 bfloat16, 2 E4M3 with per-layer scales)."""
    q0 = _d(q0).reshape(-1, 6)
    q1 = _d(q1).reshape(-1, 6)
    pts = _xyz(points)
    M, n = q0.shape[0], pts.shape[0]
    sc = _d(scales if scales is not None else np.ones(max(1, n_hidden)))
    out = np.zeros(M * n)
    lib().orc_mlp_pairs_rounded(_d(P), width, n_hidden, act, int(fmt), sc, q0, q1, M, pts, n, out)
    return out.reshape(M, n)


def mlp_forward_rounded(P, width, n_hidden, act, fmts, scales, inputs) -> np.ndarray:
    """The network on input rows (n, 15) with the input of hidden layer l
    rounded to format fmts[l] (0 none, 1 bfloat16, 2 E4M3 with scale
    scales[l]): the error of a precision taken apart layer by layer."""
    X = _d(inputs).reshape(-1, 15)
    f = np.ascontiguousarray(fmts, dtype=np.int32).reshape(n_hidden)
    sc = _d(scales if scales is not None else np.ones(max(1, n_hidden)))
    out = np.zeros(X.shape[0])
    lib().orc_mlp_forward_rounded(_d(P), width, n_hidden, act, f, sc, X, X.shape[0], out)
    return out


def mlp_loss_grad(P, width, n_hidden, act, inputs, target):
    inputs = _d(inputs).reshape(-1, 15)
    G = np.zeros(param_count(width, n_hidden))
    loss = lib().orc_mlp_loss_grad(_d(P), width, n_hidden, act, inputs, _d(target),
                                   inputs.shape[0], G)
    return loss, G


def mlp_loss_grad_bf16(P, width, n_hidden, act, inputs, target):
    """mlp_loss_grad with bfloat16 rounding where a BF16 training step stores
    values (hidden weights in the products, act(z) and act'(z) of every
    layer's unrounded pre-activation, every layer's gradient G); (loss,
    gradient)."""
    inputs = _d(inputs).reshape(-1, 15)
    G = np.zeros(param_count(width, n_hidden))
    loss = lib().orc_mlp_loss_grad_bf16(_d(P), width, n_hidden, act, inputs, _d(target), inputs.shape[0], G)
    return loss, G


def adam_step(P, G, M1, V1, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """In-place Adam step on float64 arrays P, M1, V1."""
    lib().orc_adam_step(P, _d(G), M1, V1, P.shape[0], int(t), lr, b1, b2, eps)


def check_motions(P, width, n_hidden, act, robot, q0, q1, N, points, eps, gate,
                  strict=False, f=None):
    """Margin-gated combined check; returns dict of per-motion arrays."""
    R = RobotArrays(robot)
    q0 = _d(q0).reshape(-1, 6)
    q1 = _d(q1).reshape(-1, 6)
    pts = _xyz(points)
    M, n = q0.shape[0], pts.shape[0]
    coll = np.zeros(M, dtype=np.int32)
    dmin = np.zeros(M)
    dhat = np.zeros(M)
    nf = np.zeros(M, dtype=np.int64)
    fptr = None
    if f is not None:
        f = _d(f).reshape(M, n)
        fptr = f.ctypes.data_as(C.c_void_p)
    Pd = _d(P) if P is not None else np.zeros(1)
    lib().orc_check_motions(Pd, width, n_hidden, act, R.dh, R.tool_len, R.radius, q0, q1,
                            M, int(N), pts, n, float(eps), float(gate), int(bool(strict)),
                            fptr, coll, dmin, dhat, nf)
    return {"collision": coll, "d_min": dmin, "dhat_min": dhat, "n_flagged": nf}


# ------------------------------------------------------------ quantisers

def round_bf16(a) -> np.ndarray:
    """Nearest-even bfloat16 of every element, returned as float32."""
    a = np.ascontiguousarray(a, dtype=np.float32)
    flat = a.ravel().copy()
    lib().orc_round_bf16_array(flat, flat.shape[0])
    return flat.reshape(a.shape)


def round_e4m3(v: float) -> float:
    return lib().orc_round_e4m3(float(v))


def quantize_e4m3(w):
    """(scale, dequantised float32 copy) of a weight tensor."""
    w = np.ascontiguousarray(w, dtype=np.float32).ravel()
    q = np.zeros_like(w)
    s = lib().orc_quantize_e4m3(w, w.shape[0], q)
    return s, q


def splitmix64_u01(seed, stream, i) -> float:
    return lib().orc_splitmix64_u01(int(seed), int(stream), int(i))


def training_points(robot, q0, q1, N, seed, m, spm, lo=None, hi=None) -> np.ndarray:
    """The data generator's points and labels for motion index m: (spm, 4).
    lo, hi: the box of the uniform points (default [-0.75,0.75]^2 x [0,1.5])."""
    R = RobotArrays(robot)
    out = np.zeros(spm * 4)
    if lo is None and hi is None:
        lib().orc_training_points(R.dh, R.tool_len, R.radius, _d(q0).reshape(6), _d(q1).reshape(6), int(N),
                                  int(seed), int(m), int(spm), out)
    else:
        lib().orc_training_points_region(R.dh, R.tool_len, R.radius, _d(q0).reshape(6), _d(q1).reshape(6),
                                         int(N), int(seed), int(m), int(spm), _d(lo).reshape(3),
                                         _d(hi).reshape(3), out)
    return out.reshape(spm, 4)


# ------------------------------------------------------------ Algorithm 1

def motion_dhat(P, width, n_hidden, act, q0, q1, points, fmt=0, scales=None) -> np.ndarray:
    """Eq. 6 per motion: d_hat(X, m) = min over the cloud of f(x, m); fmt 0
    evaluates the network in FP64, 1/2 with the hidden-layer inputs rounded
    as the BF16 / FP8 model stores them."""
    if len(_xyz(points)) == 0:
        return np.full(_d(q0).reshape(-1, 6).shape[0], np.inf)
    if fmt == 0:
        f = mlp_pairs(P, width, n_hidden, act, q0, q1, points)
    else:
        f = mlp_pairs_rounded(P, width, n_hidden, act, fmt, scales, q0, q1, points)
    return f.min(axis=1)


def search_first_free(dhat, delta, eps):
    """Algorithm 1 (Sec. IV-B), sequentially, on given per-motion values:
    dhat[m] the network's estimate d_hat(X, m), delta[m] the exact distance
    d(X, m); a motion is free iff its distance > eps.
      first loop:  for m in the given order, if dhat[m] > eps, check m exactly
                   (count it); return m if delta[m] > eps;
      second loop: the motions not checked, by decreasing dhat (ties in the
                   given order), check each exactly; return the first free.
    Returns dict(motion, loop, n_exact, n_nn_seq); motion -1 if none is free.
    n_nn_seq counts the network evaluations of the first loop."""
    dhat = np.asarray(dhat, dtype=np.float64)
    delta = np.asarray(delta, dtype=np.float64)
    M = len(dhat)
    done = np.zeros(M, dtype=bool)
    n_exact = 0
    for m in range(M):                                  # first loop
        if dhat[m] > eps:
            n_exact += 1
            done[m] = True
            if delta[m] > eps:
                return {"motion": m, "loop": 1, "n_exact": n_exact, "n_nn_seq": m + 1}
    rest = [m for m in range(M) if not done[m]]
    rest.sort(key=lambda m: -dhat[m])                   # stable: ties keep the given order
    for m in rest:                                      # second loop
        n_exact += 1
        if delta[m] > eps:
            return {"motion": m, "loop": 2, "n_exact": n_exact, "n_nn_seq": M}
    return {"motion": -1, "loop": 0, "n_exact": n_exact, "n_nn_seq": M}


def search_sorted(dhat, delta, eps):
    """The second loop of Algorithm 1 alone (its use in Sec. V-C): every
    candidate checked exactly by decreasing dhat (ties in the given order)
    until one is free.  Returns dict(motion, n_exact)."""
    dhat = np.asarray(dhat, dtype=np.float64)
    delta = np.asarray(delta, dtype=np.float64)
    order = sorted(range(len(dhat)), key=lambda m: -dhat[m])
    for n, m in enumerate(order):
        if delta[m] > eps:
            return {"motion": m, "n_exact": n + 1}
    return {"motion": -1, "n_exact": len(dhat)}


def search_gcc0(delta, eps):
    """GCC_0 of Sec. V-B: the exact check of each motion in the given order
    until one is free.  Returns dict(motion, n_exact)."""
    for m, d in enumerate(np.asarray(delta, dtype=np.float64)):
        if d > eps:
            return {"motion": m, "n_exact": m + 1}
    return {"motion": -1, "n_exact": len(delta)}


# ------------------------------------------------------------ block architecture

def block_forward(params, inputs, bn_eps=1e-5) -> np.ndarray:
    """The network of Sec. IV-A in FP64, BatchNorm at inference (running
    statistics), written from its definition:
      h_0 = W_0 u + b_0                      (initial linear layer, u = [x; q0; q1])
      block l: v = h_{l-1} (l = 1) or [h_{l-1}; u] (l > 1, jump connection)
               h_l = BN_l(ReLU(W_l v + b_l)) + h_{l-1}   (skip connection)
               BN(y) = gamma (y - mean) / sqrt(var + eps) + beta
      f = w_f [h_L; u] + b_f                 (final layer)
    inputs: (n, 15).  Returns (n,)."""
    u = np.asarray(inputs, dtype=np.float64).reshape(-1, 15)
    W0, b0 = (np.asarray(a, dtype=np.float64) for a in params["init"])
    h = u @ W0.T + b0
    for l, blk in enumerate(params["blocks"]):
        W, b, gamma, beta, mean, var = (np.asarray(a, dtype=np.float64) for a in blk)
        v = h if l == 0 else np.concatenate([h, u], axis=1)
        y = np.maximum(v @ W.T + b, 0.0)
        h = gamma * (y - mean) / np.sqrt(var + bn_eps) + beta + h
    Wf, bf = (np.asarray(a, dtype=np.float64) for a in params["final"])
    return (np.concatenate([h, u], axis=1) @ Wf.T + bf)[:, 0]


def block_pairs(params, q0, q1, points, bn_eps=1e-5) -> np.ndarray:
    """block_forward for every (motion, point) pair: (M, n)."""
    q0 = _d(q0).reshape(-1, 6)
    q1 = _d(q1).reshape(-1, 6)
    pts = _xyz(points)
    M, n = q0.shape[0], pts.shape[0]
    out = np.empty((M, n))
    for m in range(M):
        u = np.concatenate([pts, np.repeat(q0[m][None], n, 0), np.repeat(q1[m][None], n, 0)], axis=1)
        out[m] = block_forward(params, u, bn_eps)
    return out


def quantized_block_params(params, prec):
    """The block architecture's parameters as a model of precision `prec`
    uses them: 1 = BF16 rounds every weight matrix (initial layer, blocks,
    final layer) to nearest-even bfloat16 with the oracle's quantiser; biases
    and BatchNorm statistics are not rounded.  0 leaves everything as is."""
    if prec == 0:
        return params
    init = (round_bf16(params["init"][0]), np.asarray(params["init"][1], dtype=np.float32))
    blocks = [(round_bf16(W),) + tuple(np.asarray(a, dtype=np.float32) for a in rest)
              for W, *rest in params["blocks"]]
    final = (round_bf16(params["final"][0]), np.asarray(params["final"][1], dtype=np.float32))
    return {"init": init, "blocks": blocks, "final": final}


def block_forward_rounded(params, inputs, bn_eps=1e-5, fmt=1) -> np.ndarray:
    """block_forward with the activations stored in a 16-bit format between
    layers (fmt 1: nearest-even bfloat16; fmt 0: not rounded, block_forward
    itself): h_0 and every h_l that a later block reads -- as its input and
    as its skip term -- are rounded; the last block's output enters the final
    layer unrounded.  Everything else in double.  inputs: (n, 15)."""
    u = np.asarray(inputs, dtype=np.float64).reshape(-1, 15)

    def rnd(h):
        return round_bf16(h).astype(np.float64) if fmt == 1 else h

    W0, b0 = (np.asarray(a, dtype=np.float64) for a in params["init"])
    h = rnd(u @ W0.T + b0)
    nb = len(params["blocks"])
    for l, blk in enumerate(params["blocks"]):
        W, b, gamma, beta, mean, var = (np.asarray(a, dtype=np.float64) for a in blk)
        v = h if l == 0 else np.concatenate([h, u], axis=1)
        y = np.maximum(v @ W.T + b, 0.0)
        h = gamma * (y - mean) / np.sqrt(var + bn_eps) + beta + h
        if l + 1 < nb:
            h = rnd(h)
    Wf, bf = (np.asarray(a, dtype=np.float64) for a in params["final"])
    return (np.concatenate([h, u], axis=1) @ Wf.T + bf)[:, 0]


def block_pairs_rounded(params, q0, q1, points, bn_eps=1e-5, fmt=1) -> np.ndarray:
    """block_forward_rounded for every (motion, point) pair: (M, n)."""
    q0 = _d(q0).reshape(-1, 6)
    q1 = _d(q1).reshape(-1, 6)
    pts = _xyz(points)
    M, n = q0.shape[0], pts.shape[0]
    out = np.empty((M, n))
    for m in range(M):
        u = np.concatenate([pts, np.repeat(q0[m][None], n, 0), np.repeat(q1[m][None], n, 0)], axis=1)
        out[m] = block_forward_rounded(params, u, bn_eps, fmt)
    return out
