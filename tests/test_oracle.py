"""Pins of the FP64 CPU oracle against closed forms, invariants, brute force
and library routines -- never against the oracle's own formulas retyped.

Each test names the part of the oracle it pins and the fact that pins it.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_2402_15281_gb300 import synth as S

GOLD = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def robot():
    return S.make_robot(1)


# --------------------------------------------------------------- capsules

def test_point_capsule_closed_forms():
    a = np.array([0.1, -0.2, 0.3])
    b = np.array([0.1, -0.2, 0.9])
    r = 0.05
    # beyond the b end, on the axis: distance to the end point minus r
    assert oracle.point_capsule([0.1, -0.2, 1.4], a, b, r) == pytest.approx(0.5 - r, abs=1e-15)
    # before the a end, on the axis
    assert oracle.point_capsule([0.1, -0.2, 0.0], a, b, r) == pytest.approx(0.3 - r, abs=1e-15)
    # perpendicular foot inside the segment: radial distance minus r
    assert oracle.point_capsule([0.1 + 0.3, -0.2 + 0.4, 0.5], a, b, r) == pytest.approx(0.5 - r, abs=1e-15)
    # on the axis inside: -r (deepest point)
    assert oracle.point_capsule([0.1, -0.2, 0.6], a, b, r) == pytest.approx(-r, abs=1e-15)
    # zero-length axis is a sphere
    c = np.array([1.0, 2.0, 3.0])
    assert oracle.point_capsule([1.0, 2.0, 5.0], c, c, 0.5) == pytest.approx(1.5, abs=1e-15)


def test_point_capsule_brute_force():
    """Distance to the segment = min over densely sampled segment points; the
    sampled minimum converges to the closed-form projection from above."""
    rng = np.random.default_rng(7)
    ts = np.linspace(0.0, 1.0, 200001)
    for _ in range(50):
        a, b, x = rng.normal(size=3), rng.normal(size=3), rng.normal(size=3) * 2
        r = rng.uniform(0.01, 0.2)
        seg = a[None, :] + ts[:, None] * (b - a)[None, :]
        brute = np.min(np.linalg.norm(seg - x[None, :], axis=1)) - r
        exact = oracle.point_capsule(x, a, b, r)
        h = np.linalg.norm(b - a) / (len(ts) - 1)
        assert exact <= brute + 1e-15
        assert brute - exact <= h / 2 + 1e-12


# --------------------------------------------------------------------- FK

def test_fk_home_pose_closed_form(robot):
    """At q = 0 the chain with alpha = (-pi/2, 0, -pi/2, pi/2, -pi/2, 0) puts
    the origins at sums of the DH lengths (derived by hand):
    o1 = (a1, 0, d1), o2 = (a1+a2, 0, d1), o3 = (a1+a2+a3, 0, d1),
    o4 = o5 = (a1+a2+a3, 0, d1-d4), o6 = (a1+a2+a3, 0, d1-d4-d6), z6 = -z."""
    d1, a1 = robot.dh[0, 0], robot.dh[0, 1]
    a2, a3 = robot.dh[1, 1], robot.dh[2, 1]
    d4, d6 = robot.dh[3, 0], robot.dh[5, 0]
    T = oracle.fk(robot, np.zeros(6))
    s = a1 + a2 + a3
    want = [(0, 0, 0), (a1, 0, d1), (a1 + a2, 0, d1), (s, 0, d1), (s, 0, d1 - d4),
            (s, 0, d1 - d4), (s, 0, d1 - d4 - d6)]
    for j, o in enumerate(want):
        np.testing.assert_allclose(T[j, :3, 3], o, atol=1e-15)
    np.testing.assert_allclose(T[6, :3, 2], (0, 0, -1), atol=1e-15)
    a, b = oracle.capsules(robot, np.zeros(6))
    np.testing.assert_allclose(b[6], (s, 0, d1 - d4 - d6 - robot.tool_len), atol=1e-15)


def test_fk_rotations_orthonormal(robot):
    rng = np.random.default_rng(1)
    for _ in range(20):
        T = oracle.fk(robot, rng.uniform(-3, 3, 6))
        for j in range(7):
            R = T[j, :3, :3]
            assert np.abs(R.T @ R - np.eye(3)).max() < 1e-14
            assert np.linalg.det(R) == pytest.approx(1.0, abs=1e-14)
            np.testing.assert_array_equal(T[j, 3], [0, 0, 0, 1])


def test_fk_planar_two_link():
    """alpha = 0 and d = 0: a planar arm with o2 = (a1 c1 + a2 c12, a1 s1 + a2 s12, 0)."""
    R = S.Robot(dh=np.array([[0, 0.7, 0, 0], [0, 0.4, 0, 0]] + [[0, 0, 0, 0]] * 4, float),
                radius=np.full(7, 0.05), tool_len=0.0, qmin=-np.ones(6), qmax=np.ones(6))
    for q1, q2 in [(0.3, -1.1), (2.0, 0.5), (-2.5, 3.0)]:
        T = oracle.fk(R, np.array([q1, q2, 0, 0, 0, 0]))
        want = (0.7 * math.cos(q1) + 0.4 * math.cos(q1 + q2),
                0.7 * math.sin(q1) + 0.4 * math.sin(q1 + q2), 0.0)
        np.testing.assert_allclose(T[2, :3, 3], want, atol=1e-15)


def _rodrigues(w, th):
    K = np.array([[0, -w[2], w[1]], [w[2], 0, -w[0]], [-w[1], w[0], 0]])
    return np.eye(3) + math.sin(th) * K + (1 - math.cos(th)) * K @ K


def test_fk_product_of_exponentials(robot):
    """Independent formulation: each joint j turns everything after it about
    the fixed line (axis z_{j-1}, through o_{j-1}) of the home pose, applied
    from the tool end inwards.  The origins must agree with the DH chain."""
    T0 = oracle.fk(robot, np.zeros(6))
    axes = [T0[j, :3, 2] for j in range(6)]
    pivots = [T0[j, :3, 3] for j in range(6)]
    rng = np.random.default_rng(3)
    for _ in range(10):
        q = rng.uniform(-2.9, 2.9, 6)
        T = oracle.fk(robot, q)
        for k in range(1, 7):
            p = T0[k, :3, 3].copy()
            for j in reversed(range(k)):
                p = pivots[j] + _rodrigues(axes[j], q[j]) @ (p - pivots[j])
            np.testing.assert_allclose(T[k, :3, 3], p, atol=1e-13)


# ------------------------------------------------------------- swept SDF

def test_swept_static_motion_equals_robot_sdf(robot):
    """q0 = q1: every sample is q0 bitwise when q0 is dyadic, so the swept SDF
    is the static robot SDF bitwise; otherwise within rounding."""
    rng = np.random.default_rng(5)
    for _ in range(20):
        q = np.round(rng.uniform(-2.9, 2.9, 6) * 2 ** 20) / 2 ** 20
        x = rng.uniform(-0.8, 0.8, 3)
        assert oracle.swept_sdf(robot, q, q, 64, x) == oracle.robot_sdf(robot, q, x)
        q = rng.uniform(-2.9, 2.9, 6)
        assert oracle.swept_sdf(robot, q, q, 64, x) == pytest.approx(oracle.robot_sdf(robot, q, x), abs=1e-12)


def test_swept_symmetry_bitwise(robot):
    """f_d(x, q0, q1) = f_d(x, q1, q0): the swept volume does not depend on
    the direction of travel; the sampled form keeps this bitwise."""
    q0, q1 = S.uniform_motions(robot, 6, seed=11)
    pts = S.cube_cloud(300, seed=4)
    d01 = oracle.swept_sdf_batch(robot, q0, q1, 37, pts)
    d10 = oracle.swept_sdf_batch(robot, q1, q0, 37, pts)
    np.testing.assert_array_equal(d01, d10)


def test_swept_refinement_monotone_and_converges(robot):
    """Nested grids N, 2N, 4N, ...: the sampled union only grows, so the
    sampled SDF never increases, and it converges."""
    q0, q1 = S.uniform_motions(robot, 3, seed=12)
    pts = S.cube_cloud(200, seed=5)
    prev = None
    gaps = []
    ref = oracle.swept_sdf_batch(robot, q0, q1, 2048, pts)
    for N in (4, 8, 16, 32, 64, 128, 256):
        d = oracle.swept_sdf_batch(robot, q0, q1, N, pts)
        if prev is not None:
            assert np.all(d <= prev)
        assert np.all(d >= ref)
        gaps.append(np.max(d - ref))
        prev = d
    assert gaps[-1] < gaps[0] / 20


def test_swept_sphere_along_arc_closed_form():
    """A sphere of radius r carried on a single revolute joint sweeps a tube
    around a circular arc; its SDF is (distance to the arc) - r.  The sampled
    SDF is above it by at most half the arc spacing."""
    R, r = 0.6, 0.05
    far = -1e6    # capsules with this radius are never the minimum
    rob = S.Robot(dh=np.array([[0, R, 0, 0]] + [[0, 0, 0, 0]] * 5, float),
                  radius=np.array([far, r, far, far, far, far, far]), tool_len=0.0,
                  qmin=-np.ones(6) * 3, qmax=np.ones(6) * 3)
    th0, th1 = -0.4, 1.3
    q0 = np.array([th0, 0, 0, 0, 0, 0])
    q1 = np.array([th1, 0, 0, 0, 0, 0])
    rng = np.random.default_rng(9)
    X = rng.uniform(-1, 1, (300, 3))

    def arc_sdf(x):
        rho, phi = math.hypot(x[0], x[1]), math.atan2(x[1], x[0])
        cands = [np.array([R * math.cos(t), R * math.sin(t), 0.0]) for t in (th0, th1)]
        if th0 <= phi <= th1:
            cands.append(np.array([R * math.cos(phi), R * math.sin(phi), 0.0]))
        return min(np.linalg.norm(x - c) for c in cands) - r

    for N in (8, 64, 512):
        h = R * (th1 - th0) / N
        d = oracle.swept_sdf_batch(rob, q0, q1, N, X)[0]
        exact = np.array([arc_sdf(x) for x in X])
        assert np.all(d >= exact - 1e-12)
        assert np.all(d - exact <= h / 2 + 1e-12)


def test_swept_brute_force_tiny(robot):
    """Tiny cases by explicit enumeration of samples, capsules and a dense
    point-on-segment search (no projection formula)."""
    q0, q1 = S.uniform_motions(robot, 2, seed=13)
    pts = S.cube_cloud(4, seed=6)[:, :3].astype(np.float64)
    N = 4
    ts = np.linspace(0, 1, 20001)
    d = oracle.swept_sdf_batch(robot, q0, q1, N, pts)
    for m in range(2):
        for i in range(4):
            best = np.inf
            for k in range(N + 1):
                qk = ((N - k) * q0[m] + k * q1[m]) / N
                a, b = oracle.capsules(robot, qk)
                for j in range(7):
                    seg = a[j][None, :] + ts[:, None] * (b[j] - a[j])[None, :]
                    best = min(best, np.min(np.linalg.norm(seg - pts[i], axis=1)) - robot.radius[j])
            assert d[m, i] <= best + 1e-15
            assert best - d[m, i] < 2e-5


def test_gcc_motion_is_min_over_cloud(robot):
    q0, q1 = S.uniform_motions(robot, 4, seed=14, max_step_deg=15)
    pts = S.cube_cloud(500, seed=7)
    dmin, coll = oracle.gcc_motion(robot, q0, q1, 16, pts, 0.05)
    d = oracle.swept_sdf_batch(robot, q0, q1, 16, pts)
    np.testing.assert_array_equal(dmin, d.min(axis=1))
    np.testing.assert_array_equal(coll, (d.min(axis=1) <= 0.05).astype(np.int32))


# -------------------------------------------------------------------- MLP

def _numpy_forward(layers, X, act):
    """Library-matmul formulation of the same network, for comparison."""
    h = X
    for W, b in layers[:-1]:
        z = h @ W.T + b
        h = np.maximum(z, 0) if act == 0 else z / (1 + np.exp(-z))
    W, b = layers[-1]
    return (h @ W.T + b)[:, 0]


def test_mlp_hand_computed():
    # width 1, one hidden layer: f = wo * relu(w2 * relu(w1 . x + b1) + b2) + bo
    w1 = np.arange(1, 16, dtype=float) / 10.0
    layers = [(w1[None, :], np.array([-1.0])), (np.array([[2.0]]), np.array([0.5])),
              (np.array([[-3.0]]), np.array([0.25]))]
    P = oracle.flatten_params(layers)
    x = np.linspace(-1, 1, 15)
    h1 = max(0.0, float(w1 @ x) - 1.0)
    want = -3.0 * max(0.0, 2.0 * h1 + 0.5) + 0.25
    assert oracle.mlp_forward(P, 1, 1, S.ACT_RELU, x[None, :])[0] == pytest.approx(want, abs=1e-15)
    # all-zero weights: the output is the output bias
    zero = [(np.zeros_like(W), np.zeros_like(b)) for W, b in S.xavier_weights(8, 2)]
    zero[-1] = (zero[-1][0], np.array([0.75]))
    assert np.all(oracle.mlp_forward(oracle.flatten_params(zero), 8, 2, 0, np.ones((3, 15))) == 0.75)


@pytest.mark.parametrize("act", [S.ACT_RELU, S.ACT_SILU])
def test_mlp_matches_library_matmul(act):
    layers = S.xavier_weights(64, 3, seed=21)
    layers = [(W.astype(np.float64), np.random.default_rng(0).normal(size=b.shape) * 0.1) for W, b in layers]
    X = np.random.default_rng(1).uniform(-2, 2, (200, 15))
    f = oracle.mlp_forward(oracle.flatten_params(layers), 64, 3, act, X)
    np.testing.assert_allclose(f, _numpy_forward(layers, X, act), rtol=1e-12, atol=1e-12)


def test_mlp_pairs_input_order(robot):
    """Input row = [x, y, z, q0, q1] in that column order."""
    layers = S.xavier_weights(16, 1, seed=3)
    P = oracle.flatten_params(layers)
    q0, q1 = S.uniform_motions(robot, 2, seed=1)
    pts = S.cube_cloud(5, seed=1)
    f = oracle.mlp_pairs(P, 16, 1, 0, q0, q1, pts)
    for m in range(2):
        X = np.concatenate([pts[:, :3].astype(np.float64), np.repeat(q0[m][None], 5, 0),
                            np.repeat(q1[m][None], 5, 0)], axis=1)
        np.testing.assert_allclose(f[m], _numpy_forward(layers, X, 0), rtol=1e-12, atol=1e-13)


def test_mlp_gradient_finite_differences():
    width, L, act = 8, 2, S.ACT_SILU
    layers = S.xavier_weights(width, L, seed=31)
    P = oracle.flatten_params(layers)
    P = P + np.random.default_rng(2).normal(size=P.shape) * 0.05
    X = np.random.default_rng(3).uniform(-1, 1, (16, 15))
    target = oracle.mlp_forward(P, width, L, act, X) + np.random.default_rng(4).choice([-1, 1], 16) * 0.5
    loss, G = oracle.mlp_loss_grad(P, width, L, act, X, target)
    f = oracle.mlp_forward(P, width, L, act, X)
    assert loss == pytest.approx(np.mean(np.abs(f - target)), rel=1e-14)
    h = 1e-6
    for i in range(P.shape[0]):
        Pp, Pm = P.copy(), P.copy()
        Pp[i] += h
        Pm[i] -= h
        lp = np.mean(np.abs(oracle.mlp_forward(Pp, width, L, act, X) - target))
        lm = np.mean(np.abs(oracle.mlp_forward(Pm, width, L, act, X) - target))
        fd = (lp - lm) / (2 * h)
        assert abs(fd - G[i]) <= 1e-6 * max(1.0, abs(G[i])) + 1e-9, i


def test_mlp_gradient_relu_finite_differences():
    width, L, act = 6, 1, S.ACT_RELU
    P = oracle.flatten_params(S.xavier_weights(width, L, seed=32))
    P = P + np.random.default_rng(5).normal(size=P.shape) * 0.2
    X = np.random.default_rng(6).uniform(-1, 1, (8, 15))
    target = oracle.mlp_forward(P, width, L, act, X) - 1.0
    _, G = oracle.mlp_loss_grad(P, width, L, act, X, target)
    h = 1e-7
    for i in range(P.shape[0]):
        Pp, Pm = P.copy(), P.copy()
        Pp[i] += h
        Pm[i] -= h
        fd = (np.mean(np.abs(oracle.mlp_forward(Pp, width, L, act, X) - target))
              - np.mean(np.abs(oracle.mlp_forward(Pm, width, L, act, X) - target))) / (2 * h)
        assert abs(fd - G[i]) <= 1e-6 * max(1.0, abs(G[i])), i


def test_adam_first_step_closed_form():
    """At t = 1 the bias-corrected moments are g and g^2, so each parameter
    moves by -lr * g / (|g| + eps)."""
    rng = np.random.default_rng(8)
    P = rng.normal(size=100)
    G = rng.normal(size=100)
    P0 = P.copy()
    m, v = np.zeros(100), np.zeros(100)
    oracle.adam_step(P, G, m, v, 1, lr=1e-3)
    np.testing.assert_allclose(P, P0 - 1e-3 * G / (np.abs(G) + 1e-8), rtol=0, atol=1e-15)
    np.testing.assert_allclose(m, 0.1 * G, rtol=1e-14)
    np.testing.assert_allclose(v, 0.001 * G * G, rtol=1e-14)
    # a constant gradient keeps moving by lr * sign(g) (bias correction exact)
    for t in range(2, 6):
        oracle.adam_step(P, G, m, v, t, lr=1e-3)
    np.testing.assert_allclose(P, P0 - 5e-3 * G / (np.abs(G) + 1e-8), rtol=0, atol=1e-12)


def test_mlp_rounded_activations_match_library_emulation(robot):
    """fmt 0 is the plain network; fmt 1 and 2 round each hidden layer's input
    like torch's bfloat16 / float8_e4m3fn conversions (a library routine)."""
    torch = pytest.importorskip("torch")
    layers = S.xavier_weights(32, 2, seed=4)
    P = oracle.flatten_params(layers)
    q0, q1 = S.uniform_motions(robot, 2, seed=2)
    pts = S.cube_cloud(100, seed=2)
    np.testing.assert_array_equal(oracle.mlp_pairs_rounded(P, 32, 2, 0, 0, None, q0, q1, pts),
                                  oracle.mlp_pairs(P, 32, 2, 0, q0, q1, pts))
    Ls = [(W.astype(np.float64), b.astype(np.float64)) for W, b in layers]
    sc = np.array([1 / 16, 1 / 32])

    def emulate(fmt):
        out = []
        for m in range(2):
            X = np.concatenate([pts[:, :3].astype(np.float64), np.repeat(q0[m][None], 100, 0),
                                np.repeat(q1[m][None], 100, 0)], 1)
            h = np.maximum(X @ Ls[0][0].T + Ls[0][1], 0)
            for l in (1, 2):
                if fmt == 1:
                    h = torch.from_numpy(h.astype(np.float32)).to(torch.bfloat16).double().numpy()
                else:
                    h = torch.from_numpy(h / sc[l - 1]).to(torch.float8_e4m3fn).double().numpy() * sc[l - 1]
                h = np.maximum(h @ Ls[l][0].T + Ls[l][1], 0)
            out.append((h @ Ls[3][0].T + Ls[3][1])[:, 0])
        return np.array(out)

    for fmt in (1, 2):
        got = oracle.mlp_pairs_rounded(P, 32, 2, 0, fmt, sc, q0, q1, pts)
        np.testing.assert_allclose(got, emulate(fmt), rtol=1e-12, atol=1e-12)


def test_mlp_forward_rounded_per_layer_formats(robot):
    """The per-layer form: all-zero formats are the plain network, a uniform
    format equals mlp_pairs_rounded bitwise, and a mix (E4M3 in one layer,
    bfloat16 in another) equals torch's conversions applied layer by layer."""
    torch = pytest.importorskip("torch")
    layers = S.xavier_weights(32, 2, seed=5)
    P = oracle.flatten_params(layers)
    q0, q1 = S.uniform_motions(robot, 1, seed=4)
    pts = S.cube_cloud(200, seed=4)
    X = np.concatenate([pts[:, :3].astype(np.float64), np.repeat(q0, 200, 0), np.repeat(q1, 200, 0)], 1)
    sc = np.array([1 / 16, 1 / 32])
    np.testing.assert_array_equal(oracle.mlp_forward_rounded(P, 32, 2, 0, [0, 0], sc, X),
                                  oracle.mlp_forward(P, 32, 2, 0, X))
    for fmt in (1, 2):
        np.testing.assert_array_equal(oracle.mlp_forward_rounded(P, 32, 2, 0, [fmt, fmt], sc, X),
                                      oracle.mlp_pairs_rounded(P, 32, 2, 0, fmt, sc, q0, q1, pts)[0])
    Ls = [(W.astype(np.float64), b.astype(np.float64)) for W, b in layers]
    h = np.maximum(X @ Ls[0][0].T + Ls[0][1], 0)
    h = torch.from_numpy(h / sc[0]).to(torch.float8_e4m3fn).double().numpy() * sc[0]
    h = np.maximum(h @ Ls[1][0].T + Ls[1][1], 0)
    h = torch.from_numpy(h.astype(np.float32)).to(torch.bfloat16).double().numpy()
    h = np.maximum(h @ Ls[2][0].T + Ls[2][1], 0)
    want = (h @ Ls[3][0].T + Ls[3][1])[:, 0]
    np.testing.assert_allclose(oracle.mlp_forward_rounded(P, 32, 2, 0, [2, 1], sc, X), want, rtol=1e-12,
                               atol=1e-12)


# ---------------------------------------------------------- combined check

def test_check_open_gate_reduces_to_gcc(robot):
    """With the gate wide open every point is verified, so the combined check
    is exactly the geometric check of Eq. 5 (GCC alone)."""
    q0, q1 = S.uniform_motions(robot, 8, seed=15, max_step_deg=15)
    pts = S.cube_cloud(64, seed=8)
    P = oracle.flatten_params(S.xavier_weights(16, 1, seed=2))
    r = oracle.check_motions(P, 16, 1, 0, robot, q0, q1, 32, pts, 0.05, np.inf)
    dmin, coll = oracle.gcc_motion(robot, q0, q1, 32, pts, 0.05)
    np.testing.assert_array_equal(r["collision"], coll)
    np.testing.assert_array_equal(r["d_min"], dmin)
    assert np.all(r["n_flagged"] == 64)
    assert 0 < coll.sum() < 8     # both verdicts occur in this case


def test_check_closed_gate_and_strict(robot):
    q0, q1 = S.uniform_motions(robot, 6, seed=15, max_step_deg=15)
    pts = S.cube_cloud(300, seed=8)
    P = oracle.flatten_params(S.xavier_weights(16, 1, seed=2))
    r = oracle.check_motions(P, 16, 1, 0, robot, q0, q1, 32, pts, 0.05, -np.inf)
    assert np.all(r["collision"] == 0) and np.all(np.isinf(r["d_min"])) and np.all(r["n_flagged"] == 0)
    # strict mode re-checks every point of a motion declared free
    s = oracle.check_motions(P, 16, 1, 0, robot, q0, q1, 32, pts, 0.05, -np.inf, strict=True)
    dmin, coll = oracle.gcc_motion(robot, q0, q1, 32, pts, 0.05)
    np.testing.assert_array_equal(s["collision"], coll)
    np.testing.assert_array_equal(s["d_min"], dmin)


def test_check_gate_from_given_f(robot):
    """Flagging is f <= gate with ties flagged; dhat is the minimum of f (Eq. 6)."""
    q0, q1 = S.uniform_motions(robot, 2, seed=16, max_step_deg=10)
    pts = S.cube_cloud(50, seed=9)
    f = np.tile(np.linspace(-1, 1, 50), (2, 1))
    r = oracle.check_motions(None, 1, 1, 0, robot, q0, q1, 8, pts, 0.05, f[0, 10], f=f)
    assert np.all(r["n_flagged"] == 11)
    assert np.all(r["dhat_min"] == -1.0)
    d = oracle.swept_sdf_batch(robot, q0, q1, 8, pts)
    np.testing.assert_array_equal(r["d_min"], d[:, :11].min(axis=1))


# ------------------------------------------------------------- quantisers

def test_bf16_matches_library_and_ties():
    rng = np.random.default_rng(10)
    v = np.concatenate([rng.normal(size=20000).astype(np.float32) * 3,
                        np.array([1 + 2 ** -8, 1 + 3 * 2 ** -8, -(1 + 2 ** -8)], dtype=np.float32)])
    torch = pytest.importorskip("torch")
    lib = torch.from_numpy(v).to(torch.bfloat16).float().numpy()
    np.testing.assert_array_equal(oracle.round_bf16(v), lib)
    q = oracle.round_bf16(v[-3:])
    assert list(q) == [1.0, 1.015625, -1.0]    # ties go to the even mantissa


def _e4m3_table():
    spec = json.load(open(os.path.join(GOLD, "e4m3_format.json")))
    vals = []
    for e in range(16):
        for m in range(8):
            if e == 15 and m == 7:
                continue                             # NaN code
            if e == 0:
                vals.append(m * 2.0 ** (1 - spec["bias"] - spec["mantissa_bits"]))
            else:
                vals.append((1 + m / 8.0) * 2.0 ** (e - spec["bias"]))
    vals = np.array(sorted(set(vals)))
    assert vals.max() == spec["max_finite"] and vals[1] == spec["min_subnormal"]
    return vals


def test_e4m3_nearest_even_by_enumeration():
    """Every result is the nearest code of the format table (built from the
    OCP definition), ties to the code with an even mantissa, saturating."""
    table = _e4m3_table()
    rng = np.random.default_rng(11)
    vs = np.concatenate([rng.normal(size=3000) * 10, rng.uniform(-0.02, 0.02, 2000),
                         (table[:-1] + table[1:]) / 2, [500.0, -1e4, 448.0, 464.0]])
    for v in vs:
        r = oracle.round_e4m3(v)
        a = min(abs(v), 448.0)
        dist = np.abs(table - a)
        cands = table[dist == dist.min()]
        if len(cands) == 1:
            assert abs(r) == cands[0], v
        else:   # tie: the code whose own 3-bit mantissa field is even
            def mant(c):
                if c < 2 ** -6:
                    return int(round(c / 2 ** -9))
                e = math.floor(math.log2(c))
                return int(round(c / 2.0 ** (e - 3))) - 8
            even = [c for c in cands if mant(c) % 2 == 0]
            assert len(even) == 1 and abs(r) == even[0], v
        assert math.copysign(1.0, r) == math.copysign(1.0, v) or r == 0


def test_e4m3_matches_library():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(12)
    v = np.concatenate([rng.normal(size=20000) * 40, rng.uniform(-0.05, 0.05, 5000)])
    v = v[np.abs(v) <= 448]
    lib = torch.from_numpy(v.astype(np.float32)).to(torch.float8_e4m3fn).float().numpy()
    ours = np.array([oracle.round_e4m3(float(np.float32(x))) for x in v])
    np.testing.assert_array_equal(ours, lib.astype(np.float64))


def test_quantize_e4m3_scale():
    w = np.random.default_rng(13).normal(size=1000).astype(np.float32)
    s, q = oracle.quantize_e4m3(w)
    assert s == np.float32(np.abs(w).max()) / np.float32(448.0)
    assert np.abs(q).max() == pytest.approx(np.abs(w).max(), rel=1e-6)
    assert np.all(np.abs(q - w) <= np.abs(w) * 2 ** -4 + s * 2 ** -9 + 1e-12)


# -------------------------------------------------------------------- RNG

def test_splitmix64_published_vector():
    gold = json.load(open(os.path.join(GOLD, "splitmix64.json")))
    g = np.uint64(int(gold["gamma"], 16))
    with np.errstate(over="ignore"):
        z = np.arange(1, 5, dtype=np.uint64) * g
    got = [hex(int(x)) for x in S._fin(z)]
    assert got == [hex(int(h, 16)) for h in gold["outputs_from_state_0"]]


def test_splitmix64_oracle_matches_generator():
    r = S.Rng(17, 9)
    u = r.uniform(50)
    for i in range(50):
        assert oracle.splitmix64_u01(17, 9, i) == u[i]


def test_training_points_box():
    """The uniform training draws fill the requested box: the default box gives
    the default generator's points bit for bit; a wider box moves only the
    uniform draws (the near-surface ones stay), and those fill the wider box."""
    robot = S.make_robot(1)
    q0, q1 = S.uniform_motions(robot, 1, seed=5, max_step_deg=30)
    a = oracle.training_points(robot, q0[0], q1[0], 16, 3, 0, 4000)
    b = oracle.training_points(robot, q0[0], q1[0], 16, 3, 0, 4000, [-0.75, -0.75, 0.0], [0.75, 0.75, 1.5])
    np.testing.assert_array_equal(a, b)
    c = oracle.training_points(robot, q0[0], q1[0], 16, 3, 0, 4000, S.BOX_LO, S.BOX_HI)
    moved = np.any(a[:, :3] != c[:, :3], axis=1)
    assert 0.25 < moved.mean() < 0.35                       # the 30 % uniform draws
    # a uniform draw keeps its unit coordinates: x' = lo' + (x - lo) / (hi - lo) * (hi' - lo')
    lo0, hi0 = np.array([-0.75, -0.75, 0.0]), np.array([0.75, 0.75, 1.5])
    u = (a[moved, :3] - lo0) / (hi0 - lo0)
    np.testing.assert_allclose(c[moved, :3], S.BOX_LO + u * (S.BOX_HI - S.BOX_LO), atol=1e-12)
    assert np.all(c[moved, :3] >= S.BOX_LO) and np.all(c[moved, :3] <= S.BOX_HI)


def test_training_points_near_surface_branch():
    """The near-surface draws of the training sampler (Sec. IV-C data recipe
    on capsules), pinned by geometry rather than by its own formula: with the
    draws u_0..u_6 recomputed from the (separately pinned) SplitMix64 stream,
    every draw with u_0 < 0.7 lies at distance exactly |r_c + off| from the
    point a + u_3 (b - a) of the axis of capsule c = floor(7 u_2) at sample
    k = floor((N + 1) u_1) (axes from the pinned FK), off = -0.1 + 0.2 u_6;
    its label is at most that distance minus r_c (the capsule it was drawn
    near bounds the minimum) and equals the pinned swept-volume distance; the
    offset directions are uniform on the sphere (mean 0, second moment I / 3);
    about 70 % of the draws take this branch."""
    robot = S.make_robot(1)
    q0, q1 = S.uniform_motions(robot, 1, seed=9, max_step_deg=40)
    q0, q1 = q0[0], q1[0]
    N, seed, m, spm = 24, 11, 3, 3000
    pts = oracle.training_points(robot, q0, q1, N, seed, m, spm)
    dirs, near = [], 0
    for j in range(spm):
        u = [oracle.splitmix64_u01(seed, m, 8 * j + i) for i in range(7)]
        if u[0] >= 0.7:
            continue
        near += 1
        k = min(int(u[1] * (N + 1)), N)
        c = min(int(u[2] * 7), 6)
        qk = ((N - k) * q0 + k * q1) / N
        A, B = oracle.capsules(robot, qk)
        foot = A[c] + u[3] * (B[c] - A[c])
        off = -0.1 + 0.2 * u[6]
        rc = robot.radius[c]
        v = pts[j, :3] - foot
        dist = np.linalg.norm(v)
        assert abs(dist - abs(rc + off)) <= 1e-12, (j, dist, rc + off)
        assert pts[j, 3] <= abs(rc + off) - rc + 1e-12
        assert pts[j, 3] == oracle.swept_sdf(robot, q0, q1, N, pts[j, :3])
        if abs(rc + off) > 1e-3:
            dirs.append(v / (rc + off))
    d = np.array(dirs)
    n = len(d)
    assert abs(near / spm - 0.7) <= 4 * np.sqrt(0.21 / spm)
    np.testing.assert_allclose(np.linalg.norm(d, axis=1), 1.0, atol=1e-9)
    assert np.abs(d.mean(axis=0)).max() <= 4 / np.sqrt(3 * n)
    assert np.abs(d.T @ d / n - np.eye(3) / 3).max() <= 0.05


def test_bf16_training_gradient_emulation():
    """The BF16 training-gradient emulation (orc_mlp_loss_grad_bf16):
    * with dyadic weights and inputs of few bits every value it rounds is
      already a bfloat16, so it equals the FP64 backpropagation (itself pinned
      by finite differences) bit for bit, in both activations;
    * on a random network it equals torch's bfloat16 conversions applied at
      the same places (act(z) and act'(z) of the unrounded pre-activation,
      the hidden weights in their products, every layer's gradient G) -- a
      library routine for the rounding;
    * and it stays within the bfloat16 error of the FP64 gradient."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    W, L, n = 4, 2, 8
    npar = oracle.param_count(W, L)
    P = rng.choice([-1.0, -0.5, -0.25, 0.25, 0.5, 1.0], npar) * rng.integers(0, 2, npar)
    X = rng.choice([-1.0, -0.5, 0.0, 0.5, 1.0], (n, 15))
    T = rng.choice([-2.0, 0.0, 2.0], n)
    # ReLU: all values dyadic with few bits; SiLU values are not, so only ReLU is exact
    l0, g0 = oracle.mlp_loss_grad(P, W, L, 0, X, T)
    l1, g1 = oracle.mlp_loss_grad_bf16(P, W, L, 0, X, T)
    assert l0 == l1
    np.testing.assert_array_equal(g0, g1)
    assert np.abs(g0).sum() > 0

    def bf(a):
        return torch.from_numpy(np.asarray(a, dtype=np.float32)).to(torch.bfloat16).double().numpy()

    for act in (0, 1):
        W, L, n = 16, 2, 32
        layers = S.xavier_weights(W, L, seed=7 + act)
        P = oracle.flatten_params(layers)
        X = rng.uniform(-1, 1, (n, 15))
        T = rng.uniform(-0.2, 0.5, n)
        loss, G = oracle.mlp_loss_grad_bf16(P, W, L, act, X, T)
        Ls = [(w.astype(np.float64), b.astype(np.float64)) for w, b in layers]
        fa = (lambda z: np.maximum(z, 0)) if act == 0 else (lambda z: z / (1 + np.exp(-z)))
        da = (lambda z: (z > 0).astype(np.float64)) if act == 0 else \
             (lambda z: (1 / (1 + np.exp(-z))) * (1 + z * (1 - 1 / (1 + np.exp(-z)))))
        Ds, Hs = [], []
        z = X @ Ls[0][0].T + Ls[0][1]
        Ds.append(bf(da(z))); Hs.append(bf(fa(z)))
        Wr = [bf(Ls[l][0]) for l in range(1, L + 1)]
        for l in range(1, L + 1):
            z = Hs[-1] @ Wr[l - 1].T + Ls[l][1]
            Ds.append(bf(da(z))); Hs.append(bf(fa(z)))
        wo, bo = Ls[L + 1][0][0], Ls[L + 1][1][0]
        f = Hs[-1] @ wo + bo
        e = f - T
        df = np.sign(e) / n
        grads = [None] * (L + 2)
        grads[L + 1] = (df @ Hs[-1], np.array([df.sum()]))
        g = bf(df[:, None] * wo[None, :] * Ds[-1])
        for l in range(L, 0, -1):
            grads[l] = (g.T @ Hs[l - 1], g.sum(axis=0))
            g = bf((g @ Wr[l - 1]) * Ds[l - 1])
        grads[0] = (g.T @ X, g.sum(axis=0))
        want = np.concatenate([np.concatenate([gw.ravel(), gb.ravel()]) for gw, gb in grads])
        np.testing.assert_allclose(G, want, rtol=1e-9, atol=1e-12)
        assert abs(loss - np.abs(e).mean()) <= 1e-12
        _, G64 = oracle.mlp_loss_grad(P, W, L, act, X, T)
        assert np.linalg.norm(G - G64) <= 0.15 * np.linalg.norm(G64)     # rounding can flip a row's sign(e)
