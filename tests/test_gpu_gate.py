"""Gate calibration through the C ABI (svm_calibrate_gate).

tau = safety * max(f - delta) over calibration pairs with delta <= margin +
band: the margin widened by the measured error of the network.  The library
forms it in its own kernels (network outputs in chunks of motions, exact
distances recomputed in the reduction, never stored).  The test forms the
same maximum from the stored outputs of svm_eval_pairs and svm_label_pairs
with torch and requires the identical float, in every precision, on a
calibration set that spans two chunks, and with no pair near enough.
"""
import numpy as np
import pytest

from paper_2402_15281_gb300 import synth as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

EPS, N = 0.03, 128


@pytest.fixture(scope="module")
def svm():
    import paper_2402_15281_gb300 as svm
    svm.build()
    return svm


def _reference(svm, h, q0, q1, pts_d, margin, band, safety, chunk=64):
    over, n_near = -np.inf, 0
    for c in range(0, len(q0), chunk):
        a, b = q0[c:c + chunk], q1[c:c + chunk]
        f = torch.empty((len(a), pts_d.shape[0]), device="cuda")
        d = torch.empty_like(f)
        svm.svm_eval_pairs(h, a, b, pts_d, f)
        svm.svm_label_pairs(h, a, b, pts_d, N, d)
        near = d <= margin + band
        n_near += int(near.sum().item())
        if bool(near.any()):
            over = max(over, torch.where(near, f - d, torch.full_like(f, -float("inf"))).max().item())
    tau = max(0.0, safety * over) if n_near else 0.0
    return float(np.float32(tau)), float(np.float32(over)), n_near


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_calibrate_gate_equals_stored_outputs(svm, prec):
    robot = S.make_robot(1)
    pts = torch.from_numpy(S.bin_cloud(60_000, seed=5)).cuda()
    q0, q1 = S.bin_motions(robot, 24, seed=1000)
    h = svm.svm_create_model(robot, 256, 4, 0, prec, 0)
    try:
        svm.svm_load_weights(h, svm.make_blob(S.xavier_weights(256, 4, seed=2)))
        if prec == 2:
            svm.svm_calibrate_act_scales(h, q0, q1, pts, 2.0)
        tau, over, n_near = svm.svm_calibrate_gate(h, q0, q1, pts, EPS, N, 0.05, 1.25)
        want = _reference(svm, h, q0, q1, pts, EPS, 0.05, 1.25)
        assert (tau, over, n_near) == want
        assert n_near > 0 and tau > 0
        # no pair within margin + band: tau = 0, over = -inf
        far = torch.from_numpy(S.cube_cloud(2000, seed=1, lo=(5.0, 5.0, 5.0), hi=(6.0, 6.0, 6.0))).cuda()
        assert svm.svm_calibrate_gate(h, q0, q1, far, EPS, N, 0.05, 1.25) == (0.0, -np.inf, 0)
    finally:
        svm.svm_destroy_model(h)


def test_calibrate_gate_spans_chunks(svm):
    """420 motions x 170 000 points: more pairs than one chunk of 2^26 outputs."""
    robot = S.make_robot(1)
    pts = torch.from_numpy(S.bin_cloud(170_000, seed=6)).cuda()
    q0, q1 = S.bin_motions(robot, 420, seed=1001)
    assert 420 * 170_000 > 1 << 26
    h = svm.svm_create_model(robot, 256, 4, 0, 1, 0)
    try:
        svm.svm_load_weights(h, svm.make_blob(S.xavier_weights(256, 4, seed=2)))
        got = svm.svm_calibrate_gate(h, q0, q1, pts, EPS, N, 0.05, 1.25)
        assert got == _reference(svm, h, q0, q1, pts, EPS, 0.05, 1.25)
    finally:
        svm.svm_destroy_model(h)
