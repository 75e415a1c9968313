"""What the trained network gains over the method without it.

On a bin-picking scene the same motions are checked three ways: gated by a
network trained on the GPU (svm_train_*), gated by the untrained (Glorot)
network, and with the geometric check alone (every pair checked exactly, the
GCC_0 baseline of Sec. V-B).  Each gate is calibrated on separate motions.
All three must give the oracle's exact verdicts (Eq. 5, free iff d > eps);
the gain is the share of pairs that need the exact check, which the trained
network must cut well below the untrained one.  Timings are printed.
"""
import time

import numpy as np
import pytest

import oracle
from paper_2402_15281_gb300 import synth as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

EPS, N = 0.03, 128


@pytest.fixture(scope="module")
def svm():
    import paper_2402_15281_gb300 as svm
    svm.build()
    return svm


def _run(svm, h, q0, q1, pts_d, flags):
    res = svm.new_results(len(q0))
    svm.svm_check_motions(h, q0, q1, pts_d, EPS, N, flags, res)        # warm-up
    torch.cuda.synchronize()
    t = time.perf_counter()
    svm.svm_check_motions(h, q0, q1, pts_d, EPS, N, flags, res)
    torch.cuda.synchronize()
    return svm.results_to_numpy(res)[:len(q0)], 1e3 * (time.perf_counter() - t)


def test_trained_network_cuts_exact_checks(svm):
    from paper_2402_15281_gb300 import training
    robot = S.make_robot(1)
    tq0, tq1 = training.bin_training_motions(robot, 256, seed=41)
    blob, hist = training.train_model(svm, robot, tq0, tq1, samples_per_motion=2048, steps=N, batch=8192,
                                      epochs=12, patience=4)
    print(f"trained: best validation MAE {hist['best_val_mae']:.4f} m in {hist['seconds']:.1f} s")
    pts = S.bin_cloud(20000, seed=3)
    pts_d = torch.from_numpy(pts).cuda()
    cq0, cq1 = S.bin_motions(robot, 16, seed=1000)
    q0, q1 = S.bin_motions(robot, 16, seed=5)
    dmin, coll = oracle.gcc_motion(robot, q0, q1, N, pts, EPS)
    assert 0 < coll.sum() < 16
    out = {}
    for name, b in (("trained", blob), ("untrained", svm.make_blob(S.xavier_weights(256, 4, seed=2)))):
        h = svm.svm_create_model(robot, 256, 4, 0, svm.SVM_BF16, 0)
        try:
            svm.svm_load_weights(h, b)
            tau = training.calibrate_tau(svm, h, robot, pts_d, EPS, N, cq0, cq1)
            svm.svm_set_gate(h, tau)
            r, ms = _run(svm, h, q0, q1, pts_d, svm.SVM_NO_EARLY_EXIT)
            rs, _ = _run(svm, h, q0, q1, pts_d, svm.SVM_STRICT)
            out[name] = (r, ms, tau)
            np.testing.assert_array_equal(r["collision"], coll)
            np.testing.assert_array_equal(rs["collision"], coll)
            if name == "trained":
                g, gms = _run(svm, h, q0, q1, pts_d, svm.SVM_NO_EARLY_EXIT | svm.SVM_VERIFY_ALL)
                np.testing.assert_array_equal(g["collision"], coll)
                assert np.abs(g["d_min"] - dmin).max() <= 1e-5
                out["gcc0"] = (g, gms, None)
        finally:
            svm.svm_destroy_model(h)
    total = 16 * len(pts)
    for name, (r, ms, tau) in out.items():
        print(f"{name:10s} exact checks {r['n_verified'].sum() / total:7.2%} of pairs, {ms:7.2f} ms"
              + (f", tau {tau:.4f} m" if tau is not None else ""))
    assert out["trained"][0]["n_verified"].sum() < 0.5 * out["untrained"][0]["n_verified"].sum()
