"""GPU parity of the check path through the C ABI against the FP64 oracle.

Tolerances: per-pair network output within 1e-5 m (FP32), exact distances
within 1e-5 m, verdicts identical; counts of flagged pairs identical except
for pairs whose oracle prediction lies within 1e-4 m of the gate (where FP32
and FP64 may decide differently, and then only those may differ).
"""
import numpy as np
import pytest

import oracle
from paper_2402_15281_gb300 import synth as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

F32_TOL = 1e-5
DIST_TOL = 1e-5


@pytest.fixture(scope="module")
def svm():
    import paper_2402_15281_gb300 as svm
    svm.build()
    assert torch.cuda.is_available()
    return svm


@pytest.fixture(scope="module")
def robot():
    return S.make_robot(1)


def _layers(width=256, n_hidden=4, seed=2, bout=0.0):
    layers = S.xavier_weights(width, n_hidden, seed=seed)
    layers[-1] = (layers[-1][0], np.array([bout], dtype=np.float32))
    return layers


class Model:
    def __init__(self, svm, robot, layers, prec=0, act=0, tau=float("inf")):
        self.svm = svm
        self.width = layers[0][0].shape[0]
        self.n_hidden = len(layers) - 2
        self.act = act
        self.h = svm.svm_create_model(robot, self.width, self.n_hidden, act, prec, 0)
        svm.svm_load_weights(self.h, svm.make_blob(layers, act=act, tau=tau))
        # the oracle rounds the weights itself; the library's copy is only compared
        self.used = oracle.quantized_params(layers, prec)

    def close(self):
        self.svm.svm_destroy_model(self.h)


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _check(svm, model, q0, q1, pts, eps, N, flags):
    n_out = len(q0) // 3 if flags & svm.SVM_PATHS3 else len(q0) // 2 if flags & svm.SVM_PATHS2 else len(q0)
    res = svm.new_results(n_out)
    svm.svm_check_motions(model.h, q0, q1, _dev(pts), eps, N, flags, res)
    torch.cuda.synchronize()
    return svm.results_to_numpy(res)[:n_out]


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_weight_rounding_matches_oracle_bitwise(svm, robot, prec):
    """The device rounding at load (cvt to bfloat16 / E4M3) equals the oracle's
    quantisers written from the format definitions, bit for bit."""
    layers = _layers()
    m = Model(svm, robot, layers, prec=prec)
    try:
        np.testing.assert_array_equal(svm.svm_export_weights(m.h).astype(np.float64), m.used)
    finally:
        m.close()


def test_eval_pairs_fp32_8x4096(svm, robot):
    """Small uniform workload: 8 motions x 4096 points in the 1.5 m cube,
    15 -> 256 x 4 -> 1 ReLU."""
    q0, q1 = S.uniform_motions(robot, 8, seed=0)
    pts = S.cube_cloud(4096, seed=0)
    m = Model(svm, robot, _layers())
    try:
        f = torch.empty((8, 4096), device="cuda")
        svm.svm_eval_pairs(m.h, q0, q1, _dev(pts), f)
        torch.cuda.synchronize()
        ref = oracle.mlp_pairs(m.used, 256, 4, 0, q0, q1, pts)
        err = np.abs(f.cpu().numpy() - ref)
        assert err.max() <= F32_TOL, err.max()
    finally:
        m.close()


@pytest.mark.parametrize("width,n_hidden,act", [(64, 1, 0), (128, 2, 1), (512, 2, 1), (1024, 2, 1), (256, 0, 0)])
def test_eval_pairs_fp32_shapes(svm, robot, width, n_hidden, act):
    q0, q1 = S.uniform_motions(robot, 3, seed=1)
    pts = S.cube_cloud(1000, seed=1)         # ragged: 1000 = 15 * 64 + 40
    m = Model(svm, robot, _layers(width, n_hidden, seed=5), act=act)
    try:
        f = torch.empty((3, 1000), device="cuda")
        svm.svm_eval_pairs(m.h, q0, q1, _dev(pts), f)
        torch.cuda.synchronize()
        ref = oracle.mlp_pairs(m.used, width, n_hidden, act, q0, q1, pts)
        assert np.abs(f.cpu().numpy() - ref).max() <= F32_TOL
    finally:
        m.close()


@pytest.mark.parametrize("N", [1, 7, 64, 128])
def test_label_pairs_exact_distance(svm, robot, N):
    q0, q1 = S.uniform_motions(robot, 5, seed=2)
    pts = S.cube_cloud(777, seed=2)
    m = Model(svm, robot, _layers())
    try:
        d = torch.empty((5, 777), device="cuda")
        svm.svm_label_pairs(m.h, q0, q1, _dev(pts), N, d)
        torch.cuda.synchronize()
        ref = oracle.swept_sdf_batch(robot, q0, q1, N, pts)
        assert np.abs(d.cpu().numpy() - ref).max() <= DIST_TOL
    finally:
        m.close()


def _compare(r, ref, pts_f=None, gate=None, exact_dmin=True):
    np.testing.assert_array_equal(r["collision"], ref["collision"])
    if exact_dmin:
        both_inf = np.isinf(r["d_min"]) & np.isinf(ref["d_min"])
        with np.errstate(invalid="ignore"):
            close = np.abs(r["d_min"] - ref["d_min"]) <= DIST_TOL
        assert np.all(both_inf | close)
    if pts_f is not None:
        near = (np.abs(pts_f - gate) < 1e-4).sum(axis=1)
        assert np.all(np.abs(r["n_flagged"].astype(np.int64) - ref["n_flagged"]) <= near)
    fin = np.isfinite(ref["dhat_min"])
    assert np.all(np.abs(r["dhat_min"][fin] - ref["dhat_min"][fin]) <= F32_TOL)


@pytest.mark.parametrize("strict", [False, True])
def test_check_balanced_gated(svm, robot, strict):
    """8 short motions (|q1 - q0| <= 15 deg, both verdicts) x 4096 points with a gate
    in the middle of the prediction range, so some points are not flagged."""
    q0, q1 = S.uniform_motions(robot, 8, seed=15, max_step_deg=15)
    pts = S.cube_cloud(4096, seed=8)
    m = Model(svm, robot, _layers(bout=0.1), tau=0.0)
    eps, N = 0.05, 64
    try:
        flags = svm.SVM_NO_EARLY_EXIT | (svm.SVM_STRICT if strict else 0)
        r = _check(svm, m, q0, q1, pts, eps, N, flags)
        f = oracle.mlp_pairs(m.used, 256, 4, 0, q0, q1, pts)
        ref = oracle.check_motions(m.used, 256, 4, 0, robot, q0, q1, N, pts, eps, eps, strict=strict)
        assert 0 < ref["n_flagged"].sum() < 8 * 4096
        _compare(r, ref, f, eps)
        assert 0 < r["collision"].sum() <= 8
    finally:
        m.close()


def test_check_open_gate_equals_geometric_check(svm, robot):
    q0, q1 = S.uniform_motions(robot, 8, seed=15, max_step_deg=15)
    pts = S.cube_cloud(64, seed=8)
    m = Model(svm, robot, _layers())
    try:
        r = _check(svm, m, q0, q1, pts, 0.05, 32, svm.SVM_NO_EARLY_EXIT)
        dmin, coll = oracle.gcc_motion(robot, q0, q1, 32, pts, 0.05)
        np.testing.assert_array_equal(r["collision"], coll)
        assert np.abs(r["d_min"] - dmin).max() <= DIST_TOL
        assert np.all(r["n_flagged"] == 64) and np.all(r["n_verified"] == 64)
        assert 0 < coll.sum() < 8
        # the verify-all mode (no network) gives the same answer
        r2 = _check(svm, m, q0, q1, pts, 0.05, 32, svm.SVM_NO_EARLY_EXIT | svm.SVM_VERIFY_ALL)
        np.testing.assert_array_equal(r2["collision"], coll)
        assert np.abs(r2["d_min"] - dmin).max() <= DIST_TOL
        assert np.all(np.isinf(r2["dhat_min"]))
    finally:
        m.close()


def test_check_early_exit_verdicts_and_witness(svm, robot):
    q0, q1 = S.uniform_motions(robot, 8, seed=0)
    pts = S.cube_cloud(4096, seed=0)
    m = Model(svm, robot, _layers())
    eps, N = 0.05, 64
    try:
        r = _check(svm, m, q0, q1, pts, eps, N, 0)
        dmin, coll = oracle.gcc_motion(robot, q0, q1, N, pts, eps)
        np.testing.assert_array_equal(r["collision"], coll)
        for i in np.nonzero(coll)[0]:
            # the witness is a real collision at the reported sample
            p, k = r["witness_point"][i], r["witness_step"][i]
            assert 0 <= p < 4096 and 0 <= k <= N
            qk = ((N - k) * q0[i] + k * q1[i]) / N
            assert oracle.robot_sdf(robot, qk, pts[p, :3].astype(np.float64)) <= eps + DIST_TOL
            assert r["early_exit"][i] == 1 and r["d_min"][i] <= eps + DIST_TOL
    finally:
        m.close()


def test_check_edge_cases(svm, robot):
    m = Model(svm, robot, _layers())
    try:
        q0, q1 = S.uniform_motions(robot, 3, seed=4, max_step_deg=10)
        # no motions: nothing to do, no error
        res = svm.new_results(1)
        svm.svm_check_motions(m.h, np.zeros((0, 6)), np.zeros((0, 6)), _dev(S.cube_cloud(10)), 0.05, 8, 0, res)
        # empty cloud: every motion is free with d_min = +inf
        empty = torch.empty((0, 4), device="cuda")
        r = _check(svm, m, q0, q1, empty.cpu().numpy(), 0.05, 8, 0)
        assert np.all(r["collision"] == 0) and np.all(np.isinf(r["d_min"])) and np.all(r["n_flagged"] == 0)
        # one point, one motion, one step
        pts = S.cube_cloud(1, seed=9)
        r = _check(svm, m, q0[:1], q1[:1], pts, 0.05, 1, svm.SVM_NO_EARLY_EXIT)
        ref = oracle.check_motions(m.used, 256, 4, 0, robot, q0[:1], q1[:1], 1, pts, 0.05, np.inf)
        _compare(r, ref)
        # ragged tile counts: 63, 65, 129 points
        for n in (63, 65, 129):
            pts = S.cube_cloud(n, seed=n)
            r = _check(svm, m, q0, q1, pts, 0.05, 16, svm.SVM_NO_EARLY_EXIT)
            ref = oracle.check_motions(m.used, 256, 4, 0, robot, q0, q1, 16, pts, 0.05, np.inf)
            _compare(r, ref)
        # closed gate: nothing flagged, all free
        svm.svm_set_gate(m.h, 0.0)
        pts = S.cube_cloud(300, seed=3)
        r = _check(svm, m, q0, q1, pts, 0.0, 16, 0)
        f = oracle.mlp_pairs(m.used, 256, 4, 0, q0, q1, pts)
        assert np.all(r["n_flagged"] == (f <= 0.0).sum(axis=1))
    finally:
        m.close()


def test_max_steps_and_static_motions(svm, robot):
    """The largest sample count a call takes (900 steps: a 201 KB capsule
    table in shared memory) against the oracle; 901 steps are rejected.  A
    motion with q0 = q1 sweeps nothing: its sampled distance is the static
    robot's distance at every step count (the oracle pins this bitwise), so
    its check at 1 and at 900 steps gives the same verdict and d_min."""
    m = Model(svm, robot, _layers())
    try:
        q0, q1 = S.uniform_motions(robot, 3, seed=24, max_step_deg=40)
        q1[2] = q0[2]                                  # a static motion
        pts = S.cube_cloud(60, seed=24)                # motion 1 collides, 0 and 2 are free
        r = _check(svm, m, q0, q1, pts, 0.05, 900, svm.SVM_NO_EARLY_EXIT)
        ref = oracle.check_motions(m.used, 256, 4, 0, robot, q0, q1, 900, pts, 0.05, np.inf)
        _compare(r, ref)
        np.testing.assert_array_equal(r["collision"], [0, 1, 0])
        assert np.all(r["n_verified"] == 60)
        r1 = _check(svm, m, q0[2:], q1[2:], pts, 0.05, 1, svm.SVM_NO_EARLY_EXIT)
        assert r1["collision"][0] == r["collision"][2]
        assert abs(float(r1["d_min"][0]) - float(r["d_min"][2])) <= DIST_TOL
        with pytest.raises(svm.SvmError) as e:
            _check(svm, m, q0, q1, pts, 0.05, 901, 0)
        assert e.value.status == svm.SVM_E_INVALID
    finally:
        m.close()


def test_workspace_limit_reports_out_of_memory(svm, robot, monkeypatch):
    """The out-of-memory path without exhausting the GPU: with
    SVM_WORKSPACE_LIMIT below what a call needs, the call returns
    SVM_E_OOM before it allocates, and the model stays usable -- the same call
    without the limit gives the oracle's verdicts."""
    m = Model(svm, robot, _layers())
    try:
        q0, q1 = S.uniform_motions(robot, 3, seed=4, max_step_deg=10)
        pts = S.cube_cloud(500, seed=4)
        monkeypatch.setenv("SVM_WORKSPACE_LIMIT", "65536")
        with pytest.raises(svm.SvmError) as e:
            _check(svm, m, q0, q1, pts, 0.05, 16, svm.SVM_NO_EARLY_EXIT)
        assert e.value.status == svm.SVM_E_OOM and "SVM_WORKSPACE_LIMIT" in str(e.value)
        monkeypatch.delenv("SVM_WORKSPACE_LIMIT")
        r = _check(svm, m, q0, q1, pts, 0.05, 16, svm.SVM_NO_EARLY_EXIT)
        _compare(r, oracle.check_motions(m.used, 256, 4, 0, robot, q0, q1, 16, pts, 0.05, np.inf))
    finally:
        m.close()


def test_invalid_arguments_are_rejected(svm, robot):
    m = Model(svm, robot, _layers())
    try:
        q0, q1 = S.uniform_motions(robot, 3, seed=4)
        pts = _dev(S.cube_cloud(100))
        res = svm.new_results(3)
        bad = q0.copy()
        bad[0, 0] = np.nan
        for args in [(bad, q1, pts, 0.05, 8, 0), (q0, q1, pts, -1.0, 8, 0), (q0, q1, pts, 0.05, 0, 0),
                     (q0, q1, pts, 0.05, 8, svm.SVM_PATHS3 if len(q0) % 3 else 64),
                     (q0, q1, pts, float("nan"), 8, 0)]:
            with pytest.raises(svm.SvmError) as e:
                svm.svm_check_motions(m.h, *args, res)
            assert e.value.status == svm.SVM_E_INVALID
        with pytest.raises(svm.SvmError) as e:
            svm.svm_load_weights(m.h, b"XXXX" + b"\0" * 40)
        assert e.value.status == svm.SVM_E_WEIGHTS
    finally:
        m.close()


@pytest.mark.parametrize("seg", [2, 3])
def test_paths_of_segments(svm, robot, seg):
    """Three-segment paths q_start -> q_inVia -> q_outVia -> q_end
    and the two-segment grasp motions of Sec. V-C: one verdict per path (OR
    over its segments)."""
    paths = S.bin_paths(robot, 8, seed=1)[:, :seg + 1]
    q0 = paths[:, :seg].reshape(-1, 6)
    q1 = paths[:, 1:].reshape(-1, 6)
    flag = svm.SVM_PATHS3 if seg == 3 else svm.SVM_PATHS2
    pts = S.bin_cloud(3000, seed=0)
    m = Model(svm, robot, _layers())
    eps, N = 0.03, 32
    try:
        r = _check(svm, m, q0, q1, pts, eps, N, flag)
        dmin, coll = oracle.gcc_motion(robot, q0, q1, N, pts, eps)
        want = coll.reshape(-1, seg).max(axis=1)
        np.testing.assert_array_equal(r["collision"], want)
        r2 = _check(svm, m, q0, q1, pts, eps, N, flag | svm.SVM_NO_EARLY_EXIT)
        np.testing.assert_array_equal(r2["collision"], want)
        assert np.abs(r2["d_min"] - dmin.reshape(-1, seg).min(axis=1)).max() <= DIST_TOL
    finally:
        m.close()


def test_batch_over_scenes(svm, robot):
    """Two scenes of different sizes in one call (CSR offsets)."""
    a = S.cube_cloud(500, seed=1)
    b = S.bin_cloud(1300, seed=2)
    pts = np.concatenate([a, b])
    off = np.array([0, 500, 1800], dtype=np.int64)
    q0, q1 = S.uniform_motions(robot, 6, seed=6, max_step_deg=20)
    scene = np.array([0, 1, 1, 0, 1, 0], dtype=np.int32)
    m = Model(svm, robot, _layers())
    try:
        res = svm.new_results(6)
        svm.svm_check_batch(m.h, q0, q1, scene, _dev(pts), off, 0.05, 16, svm.SVM_NO_EARLY_EXIT, res)
        torch.cuda.synchronize()
        r = svm.results_to_numpy(res)[:6]
        for i in range(6):
            cloud = a if scene[i] == 0 else b
            dmin, coll = oracle.gcc_motion(robot, q0[i:i + 1], q1[i:i + 1], 16, cloud, 0.05)
            assert r["collision"][i] == coll[0]
            assert abs(r["d_min"][i] - dmin[0]) <= DIST_TOL
            assert r["n_flagged"][i] == len(cloud)
            # witness indices are absolute positions in the concatenated cloud
            if coll[0]:
                assert off[scene[i]] <= r["witness_point"][i] < off[scene[i] + 1] or r["witness_point"][i] == -1
    finally:
        m.close()


@pytest.mark.parametrize("prec,gated", [(0, False), (0, True), (1, True)])
def test_margin_ties_decided_in_fp64(svm, robot, prec, gated):
    """Pairs whose FP32 distance lies within 4e-6 m of the margin are counted
    and re-decided in FP64: with the margin set 1e-7 m above and below a point's
    exact distance (FP32 spacing there is ~7e-9 m), the verdicts follow the FP64
    distance (Eq. 5, free iff d > margin) and d_min is the FP64 value rounded to
    FP32.  Gated: every pair is flagged (tau = inf) and reaches the verifier
    through the network and compaction kernels."""
    q0, q1 = S.uniform_motions(robot, 4, seed=77, max_step_deg=30)
    pts = S.cube_cloud(4, seed=77)
    N = 16
    delta = oracle.swept_sdf_batch(robot, q0, q1, N, pts)          # (4, 4)
    m = Model(svm, robot, _layers(), prec=prec)
    flags = svm.SVM_NO_EARLY_EXIT | (0 if gated else svm.SVM_VERIFY_ALL)
    try:
        for k in range(4):
            one = pts[k:k + 1]
            d = delta[:, k]
            for off in (1e-7, -1e-7):
                eps = np.float32(np.abs(d).min() + off)             # near the closest motion's distance
                r = _check(svm, m, q0, q1, one, float(eps), N, flags)
                want = (d <= float(eps)).astype(np.uint8)
                np.testing.assert_array_equal(r["collision"], want)
                j = int(np.argmin(np.abs(d)))
                assert r["n_ambiguous"][j] == 1
                assert r["d_min"][j] == np.float32(d[j])
                if want[j]:
                    assert r["witness_point"][j] == 0 and 0 <= r["witness_step"][j] <= N
    finally:
        m.close()


def test_tie_list_overflow_is_reported(svm, robot):
    """Pairs at the margin beyond the tie list's capacity keep their FP32
    decision, and the record says so: with the list cut to 4 entries by the
    test hook, a motion with many points whose exact distance lies a few
    1e-7 m above the margin (all within the 4e-6 m band, FP64: free) carries
    status 2, and the motion without such points status 0; with the full list
    every such pair is decided in FP64, the verdicts equal the oracle's (Eq. 5)
    and every status is 0."""
    q0, _ = S.uniform_motions(robot, 2, seed=31)
    N = 4
    A, B = oracle.capsules(robot, q0[0])
    j = 1                                              # the upper arm, 0.47 m long
    a, e, r = A[j], B[j] - A[j], robot.radius[j]
    u = e / np.linalg.norm(e)
    n1 = np.cross(u, [0.0, 0.0, 1.0] if abs(u[2]) < 0.9 else [1.0, 0.0, 0.0])
    n1 /= np.linalg.norm(n1)
    n2 = np.cross(u, n1)
    g = S.Rng(5, 1)
    t, th = g.uniform(4000, 0.2, 0.8), g.uniform(4000, 0.0, 2 * np.pi)
    D = 0.05
    cand = a + t[:, None] * e + (r + D) * (np.cos(th)[:, None] * n1 + np.sin(th)[:, None] * n2)
    pts = np.zeros((len(cand), 4), np.float32)
    pts[:, :3] = cand
    d0 = oracle.swept_sdf_batch(robot, q0[:1], q0[:1], N, pts)[0]
    keep = np.abs(d0 - D) < 1e-6                        # capsule j is the nearest part of the robot
    pts = np.ascontiguousarray(pts[keep][:300])
    assert len(pts) >= 50
    q0s, q1s = q0.copy(), q0.copy()                   # two static motions; the second poses elsewhere
    delta = oracle.swept_sdf_batch(robot, q0s, q1s, N, pts)
    eps = float(np.float32(delta[0].min() - 2e-7))
    assert np.all(delta[0] - eps < 3e-6)                 # every point of motion 0 is at the margin
    want = (delta.min(axis=1) <= eps).astype(np.uint8)
    m = Model(svm, robot, _layers(), prec=0)
    flags = svm.SVM_VERIFY_ALL | svm.SVM_NO_EARLY_EXIT
    try:
        r = _check(svm, m, q0s, q1s, pts, eps, N, flags)
        np.testing.assert_array_equal(r["collision"], want)
        assert want[0] == 0 and r["n_ambiguous"][0] == len(pts)
        np.testing.assert_array_equal(r["status"], [0, 0])
        svm.svm_test_set_tie_cap(m.h, 4)
        r = _check(svm, m, q0s, q1s, pts, eps, N, flags)
        assert r["n_ambiguous"][0] == len(pts) and r["status"][0] == 2
        assert r["status"][1] == 0 and r["n_ambiguous"][1] == 0 and r["collision"][1] == want[1]
        svm.svm_test_set_tie_cap(m.h, 0)
        r = _check(svm, m, q0s, q1s, pts, eps, N, flags)
        np.testing.assert_array_equal(r["status"], [0, 0])
        np.testing.assert_array_equal(r["collision"], want)
    finally:
        m.close()
