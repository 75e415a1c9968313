"""A batch of 32 uneven bin scenes in one launch sequence.

32 bin scenes with log-uniform cloud sizes in [10k, 500k] points (5.4 M
points for this seed), 16 motions per scene (512 motions, 86 M pairs), checked with
the plain FP32 path, BF16 and FP8 (trained network, calibrated gates), and
as a prepared plan replayed through a CUDA graph with an autotuned verifier.

Parity: every verdict of every precision, and of the exact check of every
pair (SVM_VERIFY_ALL), equals the FP64 oracle's (Eq. 5, all 512 motions,
stored by tests/golden/oracle_verdicts.py for these inputs), and the exact
check's d(X, m) of every motion is within 1e-5 m of the oracle's; plan, graph
replay and autotuned launches give the same records as svm_check_batch.
"""
import json
import time

import numpy as np
import pytest

import oracle_verdicts
from paper_2402_15281_gb300 import synth as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

EPS, N, SCENES, PER = 0.03, 128, 32, 16


@pytest.fixture(scope="module")
def setup():
    import paper_2402_15281_gb300 as svm
    from paper_2402_15281_gb300 import training
    svm.build()
    robot, sizes, clouds, q0, q1, scene = S.uneven_batch_workload(SCENES, PER)
    pts = np.concatenate(clouds)
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    tq0, tq1 = training.bin_training_motions(robot, 1024, seed=41)
    blob, _ = training.train_model(svm, robot, tq0, tq1, samples_per_motion=4096, steps=N, batch=65536,
                                   epochs=30, patience=10)
    return svm, training, robot, sizes, clouds, torch.from_numpy(pts).cuda(), off, q0, q1, scene, blob


DETERMINISTIC = ("status", "collision", "d_min", "dhat_min", "n_flagged", "n_verified", "n_ambiguous")


def _same(a, b):
    """Records agree on every field that does not depend on thread order
    (the witness is whichever collision was found first)."""
    for k in DETERMINISTIC:
        np.testing.assert_array_equal(a[k], b[k], err_msg=k)


def _batch(svm, h, s, flags):
    svm_, training, robot, sizes, clouds, pts_d, off, q0, q1, scene, blob = s
    res = svm.new_results(len(q0))
    torch.cuda.synchronize()
    t = time.perf_counter()
    svm.svm_check_batch(h, q0, q1, scene, pts_d, off, EPS, N, flags, res)
    torch.cuda.synchronize()
    return svm.results_to_numpy(res)[:len(q0)].copy(), 1e3 * (time.perf_counter() - t)


def test_uneven_batch_all_precisions(setup):
    svm, training, robot, sizes, clouds, pts_d, off, q0, q1, scene, blob = setup
    M = len(q0)
    coll, dmin, src = oracle_verdicts.load("uneven_batch", S.inputs_digest(pts_d.cpu().numpy(), q0, q1, scene))
    print(f"oracle verdicts: {src}; {coll.sum()} of {M} motions collide")
    cq0, cq1 = S.bin_motions(robot, 16, seed=1000)
    cal_pts = pts_d[off[0]:off[1]]
    ref = None
    for prec in (0, 1, 2):
        h = svm.svm_create_model(robot, 256, 4, 0, prec, 0)
        try:
            svm.svm_load_weights(h, blob)
            if prec == 2:
                svm.svm_calibrate_act_scales(h, cq0, cq1, cal_pts, 2.0)
            svm.svm_set_gate(h, training.calibrate_tau(svm, h, robot, cal_pts, EPS, N, cq0, cq1))
            if ref is None:
                ref, _ = _batch(svm, h, setup, svm.SVM_VERIFY_ALL | svm.SVM_NO_EARLY_EXIT)
                assert np.all(ref["status"] == 0)
                np.testing.assert_array_equal(ref["collision"], coll)
                assert np.abs(ref["d_min"] - dmin).max() <= 1e-5
            _batch(svm, h, setup, 0)                                   # warm-up
            r, ms = _batch(svm, h, setup, 0)
            assert np.all(r["status"] == 0)
            np.testing.assert_array_equal(r["collision"], coll)          # every verdict vs the FP64 oracle
            print(f"prec {prec}: {M} motions, {int(sizes.sum()) * PER / 1e6:.1f} M pairs in {ms:.1f} ms "
                  f"(wall), flagged {r['n_flagged'].sum() / (sizes.sum() * PER):.2%}")
        finally:
            svm.svm_destroy_model(h)
    assert 0 < ref["collision"].sum() < M


def _events_ms(stream, fn, reps=5):
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    fn()                                                           # warm-up
    ev0.record(stream)
    for _ in range(reps):
        fn()
    ev1.record(stream)
    stream.synchronize()
    return ev0.elapsed_time(ev1) / reps


def test_plan_graph_and_autotune(setup):
    """A prepared plan: its launch, and its CUDA-graph replay, give the same
    records as svm_check_batch (every deterministic field without early exit);
    the autotuner times the network kernel's grid and the verifier's shapes.
    With early exit (the default mode), direct call, plan launch and graph
    replay are timed on one stream with CUDA events over the same work: the
    replay must not be slower than the direct call, and its verdicts equal
    the FP64 oracle's."""
    svm, training, robot, sizes, clouds, pts_d, off, q0, q1, scene, blob = setup
    M = len(q0)
    coll, _, _ = oracle_verdicts.load("uneven_batch", S.inputs_digest(pts_d.cpu().numpy(), q0, q1, scene))
    h = svm.svm_create_model(robot, 256, 4, 0, svm.SVM_BF16, 0)
    plans = []
    try:
        svm.svm_load_weights(h, blob)
        cq0, cq1 = S.bin_motions(robot, 16, seed=1000)
        training.calibrate_tau(svm, h, robot, pts_d[off[0]:off[1]], EPS, N, cq0, cq1)
        flags = svm.SVM_NO_EARLY_EXIT
        want, _ = _batch(svm, h, setup, flags)
        plan = svm.Plan(h, q0, q1, scene, off, EPS, N, flags)
        plans.append(plan)
        stream = torch.cuda.Stream()
        res = svm.new_results(M)
        with torch.cuda.stream(stream):
            plan.launch(pts_d, res, stream)
            stream.synchronize()
            _same(svm.results_to_numpy(res)[:M], want)
            report = json.loads(plan.autotune(pts_d, res, stream))
            assert len(report["candidates"]) == 9 and report["best"]["ms"] > 0
            assert len(report["network_candidates"]) == 5
            for _ in range(3):                 # capture, then two replays
                res.zero_()
                plan.graph_launch(pts_d, res, stream)
                stream.synchronize()
                _same(svm.results_to_numpy(res)[:M], want)
            # the default mode, timed three ways on one stream
            fast = svm.Plan(h, q0, q1, scene, off, EPS, N, 0)
            plans.append(fast)
            direct_ms = _events_ms(stream, lambda: svm.svm_check_batch(h, q0, q1, scene, pts_d, off, EPS, N, 0, res,
                                                                       stream))
            direct = svm.results_to_numpy(res)[:M].copy()
            plan_ms = _events_ms(stream, lambda: fast.launch(pts_d, res, stream))
            fast.graph_launch(pts_d, res, stream)          # capture
            graph_ms = _events_ms(stream, lambda: fast.graph_launch(pts_d, res, stream))
            replay = svm.results_to_numpy(res)[:M].copy()
        for r in (direct, replay):
            assert np.all(r["status"] == 0)
            np.testing.assert_array_equal(r["collision"], coll)
        print(f"autotune best {report['best']} (network grids {report['network_candidates']}); early exit: "
              f"direct {direct_ms:.2f} ms, plan launch {plan_ms:.2f} ms, graph replay {graph_ms:.2f} ms per batch")
        assert graph_ms <= 1.05 * direct_ms
    finally:
        for pl in plans:
            pl.close()
        svm.svm_destroy_model(h)
