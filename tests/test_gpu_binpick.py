"""The bin-picking use of Algorithm 1 (Sec. V-C): grasp candidates reached by
two-segment motions (into the bin: preStart -> preVia -> grasp; out of it:
grasp -> postVia -> postEnd), the network predicts every candidate's
distance and only the second loop runs -- candidates checked exactly by
decreasing prediction until one is free.  The search is compared with the
oracle's second loop on the same paths (a path's prediction and exact
distance are the minimum over its segments), and the experiment's
quantities are measured against GCC_0 (exact checks in a random order)."""
import time

import numpy as np
import pytest

import oracle
from paper_2402_15281_gb300 import synth as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

EPS, N, P = 0.03, 128, 3000
TOL = {0: 2e-4, 1: 4e-3}


@pytest.fixture(scope="module")
def setup():
    import paper_2402_15281_gb300 as svm
    from paper_2402_15281_gb300 import training
    svm.build()
    robot = S.make_robot(1)
    tq0, tq1 = training.grasp_training_motions(robot, 4096, seed=45)
    blob, hist = training.train_model(svm, robot, tq0, tq1, samples_per_motion=2048, steps=N, batch=65536,
                                      epochs=30, patience=8)
    return svm, robot, blob, hist


def _segments(wp):
    return np.ascontiguousarray(wp[:, :2].reshape(-1, 6)), np.ascontiguousarray(wp[:, 1:].reshape(-1, 6))


def _stable(dhat, delta, want, tol, seed):
    rng = np.random.default_rng(seed)
    shifts = [np.full_like(dhat, tol), np.full_like(dhat, -tol)] + \
             [rng.uniform(-tol, tol, dhat.shape) for _ in range(20)]
    return all(oracle.search_sorted(dhat + d, delta, EPS) == want for d in shifts)


@pytest.mark.parametrize("prec", [0, 1])
def test_sorted_path_search_matches_oracle(setup, prec):
    svm, robot, blob, _ = setup
    h = svm.svm_create_model(robot, 256, 4, 0, prec, 0)
    svm.svm_load_weights(h, blob)
    Pq = oracle.quantized_params(svm.parse_blob(blob), prec)
    flags = svm.SVM_SEARCH_SORTED | svm.SVM_SEARCH_PATHS2
    compared = 0
    try:
        for scene in range(4):
            pts = S.bin_cloud(P, seed=500 + scene)
            pts_d = torch.from_numpy(pts).cuda()
            for wp in S.bin_grasp_paths(robot, 35, seed=500 + scene):
                q0, q1 = _segments(wp)
                dhat = oracle.motion_dhat(Pq, 256, 4, 0, q0, q1, pts, fmt=prec).reshape(-1, 2).min(axis=1)
                dseg, _ = oracle.gcc_motion(robot, q0, q1, N, pts, EPS)
                delta = dseg.reshape(-1, 2).min(axis=1)
                want = oracle.search_sorted(dhat, delta, EPS)
                got = svm.svm_search_free_motion(h, q0, q1, pts_d, EPS, N, flags=flags)
                assert got["n_nn"] == 70 and got["loop"] in (0, 2)
                if _stable(dhat, delta, want, TOL[prec], scene):
                    compared += 1
                    assert (got["motion"], got["n_exact"]) == (want["motion"], want["n_exact"])
                elif got["motion"] >= 0:
                    assert delta[got["motion"]] > EPS
                if got["motion"] >= 0:
                    assert abs(got["delta"] - delta[got["motion"]]) <= 1e-5
                g0 = svm.svm_search_free_motion(h, q0, q1, pts_d, EPS, N, flags=svm.SVM_SEARCH_GCC0 |
                                                svm.SVM_SEARCH_PATHS2)
                assert (g0["motion"], g0["n_exact"]) == tuple(oracle.search_gcc0(delta, EPS).values())
        print(f"prec {prec}: {compared} of 8 candidate sets compared exactly")
        assert compared >= 1
    finally:
        svm.svm_destroy_model(h)


def test_bin_picking_experiment(setup):
    """22 scenes x 35 grasp candidates, 3 000-point clouds, BF16; per scene and
    direction 20 orders of the candidates: GCC_0 checks them in that order,
    the network-sorted search in decreasing prediction (order-independent up
    to ties).  Exact checks, network segment evaluations and time to the
    first free path."""
    svm, robot, blob, hist = setup
    h = svm.svm_create_model(robot, 256, 4, 0, 1, 0)
    svm.svm_load_weights(h, blob)
    rng = np.random.default_rng(1)
    rows = {(d, a): [] for d in ("into", "out") for a in ("gcc0", "nn", "nn_all")}
    coll = {"into": [], "out": []}
    try:
        for scene in range(22):
            pts_d = torch.from_numpy(S.bin_cloud(P, seed=700 + scene)).cuda()
            for d, wp in zip(("into", "out"), S.bin_grasp_paths(robot, 35, seed=700 + scene)):
                q0, q1 = _segments(wp)
                full = svm.svm_search_free_motion(h, q0, q1, pts_d, EPS, N, wave=64,
                                                  flags=svm.SVM_SEARCH_GCC0 | svm.SVM_SEARCH_PATHS2)
                for k in range(20):
                    perm = rng.permutation(35)
                    seg = np.stack([2 * perm, 2 * perm + 1], axis=1).ravel()
                    for a, flags, wave in (("gcc0", svm.SVM_SEARCH_GCC0, 1), ("nn", svm.SVM_SEARCH_SORTED, 1),
                                           ("nn_all", svm.SVM_SEARCH_SORTED, 64)):
                        torch.cuda.synchronize()
                        t = time.perf_counter()
                        r = svm.svm_search_free_motion(h, q0[seg], q1[seg], pts_d, EPS, N, wave=wave,
                                                       flags=flags | svm.SVM_SEARCH_PATHS2)
                        rows[(d, a)].append((1e3 * (time.perf_counter() - t), r["n_exact"], r["n_nn"],
                                             r["motion"] >= 0))
                # share of colliding candidates in this scene (one exact check of all of them)
                res = svm.new_results(35)
                svm.svm_check_motions(h, q0, q1, pts_d, EPS, N, svm.SVM_VERIFY_ALL | svm.SVM_PATHS2, res)
                torch.cuda.synchronize()
                coll[d].append(svm.results_to_numpy(res)[:35]["collision"].mean())
        print(f"bin picking, 22 scenes x 35 candidates x 20 orders, {P} points (BF16 256x4, val MAE "
              f"{hist['best_val_mae']:.4f} m)")
        for d in ("into", "out"):
            print(f"  {d}: colliding candidates {np.mean(coll[d]):.1%}")
            for a, name in (("gcc0", "GCC_0"), ("nn", "GCC-NN (sorted)"), ("nn_all", "sorted, one launch")):
                x = np.array(rows[(d, a)])
                print(f"    {name:18s} time {x[:, 0].mean():.3f} +- {x[:, 0].std():.3f} ms, exact checks "
                      f"{x[:, 1].mean():.2f} +- {x[:, 1].std():.2f}" + (f", NN checks {x[:, 2].mean():.1f}"
                                                                        if a != "gcc0" else ""))
            g, n = np.array(rows[(d, "gcc0")]), np.array(rows[(d, "nn")])
            assert np.array_equal(g[:, 3], n[:, 3])
    finally:
        svm.svm_destroy_model(h)
