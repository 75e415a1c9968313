"""The block architecture of Sec. IV-A in the oracle, pinned on hand-worked
and closed-form cases."""
import numpy as np
import pytest

import oracle
from paper_2402_15281_gb300 import synth as S


def _params(width, n_blocks, init, blocks, final):
    return {"init": init, "blocks": blocks, "final": final}


def test_hand_worked_two_wide_network():
    # width 2, two blocks; input u = (x, y, z, q0.., q1..) with only x = 1, y = 2 nonzero
    u = np.zeros((1, 15)); u[0, 0], u[0, 1] = 1.0, 2.0
    W0 = np.zeros((2, 15)); W0[0, 0], W0[1, 1] = 1.0, -1.0          # h0 = (1, -2) + b0
    b0 = np.array([0.5, 0.0])                                         # h0 = (1.5, -2)
    # block 1: W = I, b = 0 -> relu(h0) = (1.5, 0); BN with gamma 2, beta 0.1, mean 0.5, var 1 - eps
    eps = 1e-5
    blk1 = (np.eye(2), np.zeros(2), np.array([2.0, 2.0]), np.array([0.1, 0.1]), np.array([0.5, 0.5]),
            np.array([1 - eps, 1 - eps]))
    # a1 = 2 (y - 0.5) + 0.1 = (2.1, -0.9); h1 = a1 + h0 = (3.6, -2.9)
    # block 2 sees [h1; u]: W picks h1[1] and x: z = (-h1[1], x) = (2.9, 1); identity BN
    W2 = np.zeros((2, 17)); W2[0, 1], W2[1, 2] = -1.0, 1.0
    blk2 = (W2, np.zeros(2), np.ones(2), np.zeros(2), np.zeros(2), np.full(2, 1 - eps))
    # h2 = (2.9, 1) + h1 = (6.5, -1.9)
    Wf = np.zeros((1, 17)); Wf[0, 0], Wf[0, 1], Wf[0, 3] = 1.0, 2.0, 10.0   # 6.5 - 3.8 + 20 (y)
    P = _params(2, 2, (W0, b0), [blk1, blk2], (Wf, np.array([0.25])))
    f = oracle.block_forward(P, u, eps)
    assert abs(f[0] - (6.5 - 3.8 + 20.0 + 0.25)) < 1e-12


def test_identity_blocks_reduce_to_the_initial_layer():
    """Zero block weights and an identity BatchNorm leave h = h0 + relu(b) per
    block: f = w_f [h0 + sum relu(b_l); u] + b_f."""
    P = S.block_weights(64, 3, seed=4)
    eps = 1e-5
    blocks = []
    relu_sum = np.zeros(64)
    for (W, b, g, be, m, v) in P["blocks"]:
        blocks.append((np.zeros_like(W), b, np.sqrt(v.astype(np.float64) + eps), m.astype(np.float64), m, v))
        relu_sum += np.maximum(b.astype(np.float64), 0.0)
    Q = {"init": P["init"], "blocks": blocks, "final": P["final"]}
    rng = np.random.default_rng(0)
    u = rng.uniform(-1, 1, (50, 15))
    W0, b0 = (a.astype(np.float64) for a in P["init"])
    h = u @ W0.T + b0 + relu_sum
    Wf, bf = (a.astype(np.float64) for a in P["final"])
    want = np.concatenate([h, u], axis=1) @ Wf[0] + bf[0]
    np.testing.assert_allclose(oracle.block_forward(Q, u, eps), want, rtol=1e-12, atol=1e-12)


def test_jump_path_carries_the_input():
    """A second block that reads only the jump input: h2 - h1 = BN(relu(W_u u + b))."""
    P = S.block_weights(32, 2, seed=5)
    W, b, g, be, m, v = P["blocks"][1]
    W = W.copy(); W[:, :32] = 0.0                        # only the [u] part remains
    Q = {"init": P["init"], "blocks": [P["blocks"][0], (W, b, g, be, m, v)], "final": P["final"]}
    Q1 = {"init": P["init"], "blocks": [P["blocks"][0]], "final": (P["final"][0], P["final"][1])}
    rng = np.random.default_rng(1)
    u = rng.uniform(-1, 1, (20, 15))
    y = np.maximum(u @ W[:, 32:].astype(np.float64).T + b, 0.0)
    a2 = g * (y - m) / np.sqrt(v.astype(np.float64) + 1e-5) + be
    Wf = P["final"][0].astype(np.float64)[0]
    np.testing.assert_allclose(oracle.block_forward(Q, u) - oracle.block_forward(Q1, u), a2 @ Wf[:32], rtol=1e-10,
                               atol=1e-10)


def test_block_blob_round_trip():
    import struct
    import paper_2402_15281_gb300 as svm
    P = S.block_weights(64, 2, seed=1)
    blob = svm.make_block_blob(P, tau=0.5)
    magic, ver, nb, ind, w, act, tau, eps = struct.unpack("<4sIIIIIff", blob[:32])
    assert (magic, ver, nb, ind, w, act, tau) == (b"SVMW", 2, 2, 15, 64, 0, 0.5) and abs(eps - 1e-5) < 1e-12
    n = 8 + 64 * 15 * 4 + 64 * 4                          # initial
    n += 8 + 64 * 64 * 4 + 5 * 64 * 4 + 8 + 64 * 79 * 4 + 5 * 64 * 4
    n += 8 + 79 * 4 + 4
    assert len(blob) == 32 + n


def test_block_forward_rounded():
    """The 16-bit emulation of the block architecture: with fmt 0 it is
    block_forward bitwise; with fmt 1 it equals torch's bfloat16 conversions
    applied to h_0 and to every block output a later block reads (a library
    routine), and the BF16 weight rounding equals torch's conversion."""
    torch = pytest.importorskip("torch")
    P = S.block_weights(64, 3, seed=11)
    rng = np.random.default_rng(3)
    X = rng.uniform(-1, 1, (50, 15))
    np.testing.assert_array_equal(oracle.block_forward_rounded(P, X, fmt=0), oracle.block_forward(P, X))
    Q = oracle.quantized_block_params(P, 1)
    for (Wq, *_), (W, *_) in zip(Q["blocks"], P["blocks"]):
        np.testing.assert_array_equal(Wq, torch.from_numpy(np.asarray(W, np.float32)).to(torch.bfloat16).float().numpy())

    def bf(h):
        return torch.from_numpy(h.astype(np.float32)).to(torch.bfloat16).double().numpy()

    W0, b0 = (np.asarray(a, np.float64) for a in Q["init"])
    h = bf(X @ W0.T + b0)
    for l, (W, b, g, be, mu, var) in enumerate(Q["blocks"]):
        W, b, g, be, mu, var = (np.asarray(a, np.float64) for a in (W, b, g, be, mu, var))
        v = h if l == 0 else np.concatenate([h, X], axis=1)
        y = np.maximum(v @ W.T + b, 0.0)
        h = g * (y - mu) / np.sqrt(var + 1e-5) + be + h
        if l < 2:
            h = bf(h)
    Wf, bfin = (np.asarray(a, np.float64) for a in Q["final"])
    want = (np.concatenate([h, X], axis=1) @ Wf.T + bfin)[:, 0]
    np.testing.assert_allclose(oracle.block_forward_rounded(Q, X, fmt=1), want, rtol=1e-12, atol=1e-12)
