"""Algorithm 1 (Sec. IV-B) on the GPU: svm_search_free_motion against the
oracle's sequential algorithm on box-world scenes (Sec. V-B), and the
prediction-only check (Eq. 6).

The oracle takes d_hat from its own network evaluation (FP64 for the FP32
model; hidden-layer inputs rounded to bfloat16 for the BF16 model) and the
exact distance from its geometric check (Eq. 5).  The returned motion, the
loop and the exact-check count are compared exactly when the oracle's answer
is stable under moving every prediction by up to the precision's tolerance;
otherwise (a prediction at the margin, or a near tie in the second loop's
order) several answers are correct and the test checks that the returned
motion is free."""
import time

import numpy as np
import pytest

import oracle
from paper_2402_15281_gb300 import synth as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

EPS, N = 0.005, 200
TOL = {0: 2e-4, 1: 4e-3}          # |d_hat GPU - oracle| bound per precision (m)


@pytest.fixture(scope="module")
def setup():
    import paper_2402_15281_gb300 as svm
    from paper_2402_15281_gb300 import training
    svm.build()
    robot = S.make_robot(1)
    # box-world-like motions (start and goal uniform in the joint limits), uniform
    # training points over the box-world volume
    # (many motions with few points each train better than the reverse)
    tq0, tq1 = S.uniform_motions(robot, 32768, seed=51)
    blob, hist = training.train_model(svm, robot, tq0, tq1, samples_per_motion=1024, steps=N, batch=65536,
                                      epochs=30, patience=8, box=(S.BOX_LO, S.BOX_HI))
    return svm, robot, blob, hist


def _model(svm, robot, blob, prec):
    h = svm.svm_create_model(robot, 256, 4, 0, prec, 0)
    svm.svm_load_weights(h, blob)
    return h


def _stable(dhat, delta, want, tol, seed):
    """The oracle's answer does not change when every prediction moves by up
    to tol (20 random draws plus the two uniform shifts)."""
    rng = np.random.default_rng(seed)
    shifts = [np.full_like(dhat, tol), np.full_like(dhat, -tol)] + \
             [rng.uniform(-tol, tol, dhat.shape) for _ in range(20)]
    return all(oracle.search_first_free(dhat + d, delta, EPS) == want for d in shifts)


@pytest.mark.parametrize("prec", [0, 1])
def test_predict_only_is_eq6(setup, prec):
    svm, robot, blob, _ = setup
    pts, *_ = S.box_world(11)
    q0, q1 = S.box_world_motions(robot, 100, seed=11)
    h = _model(svm, robot, blob, prec)
    try:
        res = svm.new_results(100)
        svm.svm_check_motions(h, q0, q1, torch.from_numpy(pts).cuda(), EPS, N, svm.SVM_PREDICT_ONLY, res)
        torch.cuda.synchronize()
        r = svm.results_to_numpy(res)[:100]
        Pq = oracle.quantized_params(svm.parse_blob(blob), prec)
        want = oracle.motion_dhat(Pq, 256, 4, 0, q0, q1, pts, fmt=prec)
        assert np.all(r["status"] == 0) and np.all(r["collision"] == 0) and np.all(r["n_verified"] == 0)
        assert np.abs(r["dhat_min"] - want).max() <= TOL[prec]
    finally:
        svm.svm_destroy_model(h)


@pytest.mark.parametrize("prec", [0, 1])
def test_search_matches_algorithm1(setup, prec):
    svm, robot, blob, _ = setup
    h = _model(svm, robot, blob, prec)
    Pq = oracle.quantized_params(svm.parse_blob(blob), prec)
    checked = unique = 0
    try:
        for scene in range(6):
            pts, *_ = S.box_world(100 + scene)
            q0, q1 = S.box_world_motions(robot, 100, seed=100 + scene)
            pts_d = torch.from_numpy(pts).cuda()
            dhat = oracle.motion_dhat(Pq, 256, 4, 0, q0, q1, pts, fmt=prec)
            delta, _ = oracle.gcc_motion(robot, q0, q1, N, pts, EPS)
            want = oracle.search_first_free(dhat, delta, EPS)
            g0 = oracle.search_gcc0(delta, EPS)
            got = [svm.svm_search_free_motion(h, q0, q1, pts_d, EPS, N, wave=w) for w in (1, 4)]
            gcc = svm.svm_search_free_motion(h, q0, q1, pts_d, EPS, N, flags=svm.SVM_SEARCH_GCC0)
            assert (gcc["motion"], gcc["n_exact"]) == (g0["motion"], g0["n_exact"])
            for a in got[1:]:
                assert {k: a[k] for k in ("motion", "loop", "n_exact")} == \
                       {k: got[0][k] for k in ("motion", "loop", "n_exact")}
                assert a["n_exact_run"] >= a["n_exact"]
            r = got[0]
            assert r["n_nn"] == 100 and r["n_exact_run"] == r["n_exact"]
            checked += 1
            if _stable(dhat, delta, want, TOL[prec], scene):
                unique += 1
                assert {k: r[k] for k in want} == want
            else:                                          # several answers are correct: check validity
                if r["motion"] >= 0:
                    assert delta[r["motion"]] > EPS
                assert (r["motion"] >= 0) == (want["motion"] >= 0)
            if r["motion"] >= 0:
                assert abs(r["delta"] - delta[r["motion"]]) <= 1e-5
                assert abs(r["delta_hat"] - dhat[r["motion"]]) <= TOL[prec]
        print(f"prec {prec}: {checked} scenes, {unique} with a unique answer compared exactly")
        assert unique >= 1
    finally:
        svm.svm_destroy_model(h)


def test_box_world_experiment(setup):
    """The box-world experiment of Sec. V-B (the quantities of its results
    table): 100 scenes x 100 motions from one start, 5 mm margin, 200 steps,
    BF16; for each scene and several orders of its motions, the time to the
    first free motion of GCC_0 and of Algorithm 1 and their exact-check
    counts, run sequentially (wave 1, the paper's algorithm) and with 8 or all
    candidates checked per launch (same answers, more exact checks run)."""
    svm, robot, blob, hist = setup
    h = _model(svm, robot, blob, 1)
    n_scenes, n_perm = 100, 5
    rng = np.random.default_rng(0)
    rows = {"gcc0": [], "nn": [], "gcc0_w8": [], "nn_w8": [], "gcc0_w128": [], "nn_w128": []}
    free_frac, cls = [], []
    try:
        for scene in range(n_scenes):
            pts, *_ = S.box_world(1000 + scene)
            q0, q1 = S.box_world_motions(robot, 100, seed=1000 + scene)
            pts_d = torch.from_numpy(pts).cuda()
            for k in range(n_perm):
                perm = rng.permutation(100)
                for name, flags, wave in (("gcc0", svm.SVM_SEARCH_GCC0, 1), ("nn", 0, 1),
                                          ("gcc0_w8", svm.SVM_SEARCH_GCC0, 8), ("nn_w8", 0, 8),
                                          ("gcc0_w128", svm.SVM_SEARCH_GCC0, 128), ("nn_w128", 0, 128)):
                    torch.cuda.synchronize()
                    t = time.perf_counter()
                    r = svm.svm_search_free_motion(h, q0[perm], q1[perm], pts_d, EPS, N, wave=wave, flags=flags)
                    rows[name].append((1e3 * (time.perf_counter() - t), r["n_exact"], r["n_nn_seq"],
                                       r["motion"] >= 0, r["n_exact_run"]))
            if scene < 10:
                delta, coll = oracle.gcc_motion(robot, q0, q1, N, pts, EPS)
                free_frac.append(1 - coll.mean())
                res = svm.new_results(100)
                svm.svm_check_motions(h, q0, q1, pts_d, EPS, N, svm.SVM_PREDICT_ONLY, res)
                torch.cuda.synchronize()
                pred_coll = svm.results_to_numpy(res)[:100]["dhat_min"] <= EPS
                cls.append((np.mean(pred_coll == (coll == 1)), np.mean(pred_coll & (coll == 0)),
                            np.mean(~pred_coll & (coll == 1))))
        g, n = np.array(rows["gcc0"]), np.array(rows["nn"])
        assert np.array_equal(g[:, 3], n[:, 3])             # both find a free motion in the same scenes
        for w1, wk in (("gcc0", "gcc0_w8"), ("nn", "nn_w8"), ("gcc0", "gcc0_w128"), ("nn", "nn_w128")):
            assert np.array_equal(np.array(rows[w1])[:, 1], np.array(rows[wk])[:, 1])   # same answer, other work
        print(f"box world, {n_scenes} scenes x {n_perm} orders (BF16 256x4, val MAE {hist['best_val_mae']:.4f} m); "
              f"free motions in the first 10 scenes: {np.mean(free_frac):.1%}; "
              f"scenes with a free motion: {g[:, 3].mean():.1%}")
        acc, fp, fn = np.mean(cls, axis=0)
        print(f"  motion classification at the margin (first 10 scenes): accuracy {acc:.1%}, "
              f"false positives (predicted collision, free) {fp:.1%}, false negatives {fn:.1%}")
        has_free = g[:, 3] > 0
        for subset, sel in (("all scenes", np.ones_like(has_free)), ("scenes with a free motion", has_free)):
            print(f"  {subset}:")
            for name, key in (("GCC_0", "gcc0"), ("GCC-NN", "nn"), ("GCC_0 w8", "gcc0_w8"), ("GCC-NN w8", "nn_w8"),
                              ("GCC_0 w128", "gcc0_w128"), ("GCC-NN w128", "nn_w128")):
                a = np.array(rows[key])[sel]
                print(f"    {name:11s} time {a[:, 0].mean():.3f} +- {a[:, 0].std():.3f} ms, exact checks "
                      f"{a[:, 1].mean():.2f} +- {a[:, 1].std():.2f} (run {a[:, 4].mean():.2f})" +
                      (f", NN checks (sequential) {a[:, 2].mean():.2f} +- {a[:, 2].std():.2f}" if "NN" in name else ""))
        assert n[:, 1].mean() <= g[:, 1].mean()
    finally:
        svm.svm_destroy_model(h)


def test_search_edge_cases(setup):
    svm, robot, blob, _ = setup
    h = _model(svm, robot, blob, 1)
    try:
        pts, *_ = S.box_world(5)
        pts_d = torch.from_numpy(pts).cuda()
        q0, q1 = S.box_world_motions(robot, 10, seed=5)
        empty = np.zeros((0, 6))
        r = svm.svm_search_free_motion(h, empty, empty, pts_d, EPS, N)
        assert (r["motion"], r["loop"], r["n_exact"], r["n_nn"]) == (-1, 0, 0, 0)
        # no points: every motion is free (d = d_hat = +inf); the first one is returned by the first loop
        none = torch.zeros((0, 4), dtype=torch.float32, device="cuda")
        r = svm.svm_search_free_motion(h, q0, q1, none, EPS, N)
        assert (r["motion"], r["loop"], r["n_exact"]) == (0, 1, 1) and r["delta"] == np.inf
        # a wave larger than the candidate list changes the work, not the answer
        a = svm.svm_search_free_motion(h, q0, q1, pts_d, EPS, N, wave=1)
        b = svm.svm_search_free_motion(h, q0, q1, pts_d, EPS, N, wave=1000)
        assert (a["motion"], a["loop"], a["n_exact"]) == (b["motion"], b["loop"], b["n_exact"])
        for kw in ({"wave": 0}, {"flags": 16}, {"flags": svm.SVM_SEARCH_PATHS2 | svm.SVM_SEARCH_PATHS3},
                   {"flags": svm.SVM_SEARCH_PATHS3}):         # 10 motions are not whole 3-segment paths
            with pytest.raises(svm.SvmError):
                svm.svm_search_free_motion(h, q0, q1, pts_d, EPS, N, **kw)
        res = svm.new_results(10)
        with pytest.raises(svm.SvmError):
            svm.svm_check_motions(h, q0, q1, pts_d, EPS, N, svm.SVM_PREDICT_ONLY | svm.SVM_VERIFY_ALL, res)
    finally:
        svm.svm_destroy_model(h)
