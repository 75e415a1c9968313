"""The block architecture of Sec. IV-A on the FP32 path: the library's network
(BatchNorm folded, jump input split into a per-motion bias and an x-term)
against the oracle's unfolded FP64 definition, a gated check against the
oracle's flags and exact distances, and the inference times at the shapes
of the paper's inference-time table (one motion x 1 000 / 3 000 / 20 000
points; 5x512, 11x512 and 11x1024).  At width 1024 the FP32 kernel runs each
64-pair tile in two passes of 32 pairs, so the parity cases include it."""
import numpy as np
import pytest

import oracle
from paper_2402_15281_gb300 import synth as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def svm():
    import paper_2402_15281_gb300 as svm
    svm.build()
    return svm


def _model(svm, robot, P, tau=float("inf")):
    width, nb = P["init"][0].shape[0], len(P["blocks"])
    h = svm.svm_create_model(robot, width, nb, 0, svm.SVM_FP32, 0, arch=svm.SVM_ARCH_BLOCKS)
    svm.svm_load_weights(h, svm.make_block_blob(P, tau=tau))
    return h


@pytest.mark.parametrize("width,nb", [(64, 1), (256, 2), (512, 5), (512, 11), (1024, 2), (1024, 11)])
def test_block_network_matches_oracle(svm, width, nb):
    robot = S.make_robot(1)
    P = S.block_weights(width, nb, seed=width + nb)
    q0, q1 = S.uniform_motions(robot, 3, seed=nb)
    pts = S.cube_cloud(300, seed=width)       # 300 points: several tiles and a ragged tail
    h = _model(svm, robot, P)
    try:
        f = torch.empty((3, 300), device="cuda")
        svm.svm_eval_pairs(h, q0, q1, torch.from_numpy(pts).cuda(), f)
        torch.cuda.synchronize()
        got = f.cpu().numpy().astype(np.float64)
    finally:
        svm.svm_destroy_model(h)
    want = oracle.block_pairs(P, q0, q1, pts)
    scale = max(1.0, np.abs(want).max())
    err = np.abs(got - want).max()
    print(f"{nb}x{width}: |f| up to {np.abs(want).max():.2f}, max |f - f64| {err:.2e}")
    assert err <= 2e-5 * scale * np.sqrt(nb)


@pytest.mark.parametrize("width,nb", [(256, 3), (1024, 2)])
def test_block_network_gated_check(svm, width, nb):
    """Flags and verdicts of a gated check equal the oracle's: flagged iff
    f <= margin + tau (no f within 1e-3 of the gate), collision iff a flagged
    point's exact distance is <= margin."""
    robot = S.make_robot(1)
    P = S.block_weights(width, nb, seed=9)
    q0, q1 = S.uniform_motions(robot, 6, seed=9, max_step_deg=25)
    pts = S.cube_cloud(2000, seed=9)
    f = oracle.block_pairs(P, q0, q1, pts)
    eps, N = 0.05, 32
    # a gate above the margin (tau >= 0) in a gap of the predictions, from their 30th percentile up
    fs = np.sort(f.ravel())
    k = max(int(0.3 * len(fs)), int(np.searchsorted(fs, eps + 0.01)))
    while fs[k + 1] - fs[k] < 2e-3:
        k += 1
    gate = 0.5 * (fs[k] + fs[k + 1])
    assert gate - eps >= 0
    h = _model(svm, robot, P, tau=gate - eps)
    try:
        res = svm.new_results(6)
        svm.svm_check_motions(h, q0, q1, torch.from_numpy(pts).cuda(), eps, N, svm.SVM_NO_EARLY_EXIT, res)
        torch.cuda.synchronize()
        r = svm.results_to_numpy(res)[:6]
    finally:
        svm.svm_destroy_model(h)
    flagged = f <= gate
    delta = oracle.swept_sdf_batch(robot, q0, q1, N, pts)
    np.testing.assert_array_equal(r["n_flagged"], flagged.sum(axis=1))
    np.testing.assert_array_equal(r["collision"], np.any(flagged & (delta <= eps), axis=1).astype(np.uint8))
    np.testing.assert_allclose(r["dhat_min"], f.min(axis=1), atol=1e-4)


def test_inference_times_at_the_paper_shapes(svm):
    """Network time of one motion x n points (prediction only: the network and
    the per-motion minimum), CUDA events, median of 50 calls after warm-up."""
    robot = S.make_robot(1)
    q0, q1 = S.uniform_motions(robot, 1, seed=0)
    rows = []
    for nb, width in ((5, 512), (11, 512), (11, 1024)):
        P = S.block_weights(width, nb, seed=1)
        h = _model(svm, robot, P)
        try:
            for n in (1000, 3000, 20000):
                pts = torch.from_numpy(S.cube_cloud(n, seed=n)).cuda()
                res = svm.new_results(1)
                ts = []
                for k in range(60):
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record()
                    svm.svm_check_motions(h, q0, q1, pts, 0.01, 64, svm.SVM_PREDICT_ONLY, res)
                    e1.record()
                    torch.cuda.synchronize()
                    if k >= 10:
                        ts.append(e0.elapsed_time(e1))
                rows.append((f"{nb}x{width}", n, float(np.median(ts))))
        finally:
            svm.svm_destroy_model(h)
    for name, n, ms in rows:
        print(f"block network {name} FP32, 1 motion x {n} points: {ms:.3f} ms")
    assert all(ms > 0 for _, _, ms in rows)


def test_block_model_arguments(svm):
    import struct
    robot = S.make_robot(1)
    P = S.block_weights(64, 2, seed=3)
    blob = svm.make_block_blob(P)
    # the block architecture runs on the FP32 path with ReLU only
    for prec, act in ((svm.SVM_BF16, 0), (svm.SVM_FP32, 1)):
        with pytest.raises(svm.SvmError):
            svm.svm_create_model(robot, 64, 2, act, prec, 0, arch=svm.SVM_ARCH_BLOCKS)
    h = svm.svm_create_model(robot, 64, 2, 0, svm.SVM_FP32, 0, arch=svm.SVM_ARCH_BLOCKS)
    try:
        bad = [svm.make_blob(S.xavier_weights(64, 2)),                      # version 1
               blob[:-4],                                                   # truncated
               blob + b"\0\0\0\0",                                          # trailing bytes
               svm.make_block_blob(S.block_weights(64, 3, seed=3)),         # 3 blocks for a 2-block model
               blob[:28] + struct.pack("<f", float("nan")) + blob[32:]]     # bad BatchNorm epsilon
        for b in bad:
            with pytest.raises(svm.SvmError):
                svm.svm_load_weights(h, b)
        svm.svm_load_weights(h, blob)
        used = svm.svm_export_weights(h)
        assert used.size == (len(blob) - 32) // 4 - 2 * (2 + 2)          # every float, no shape words
    finally:
        svm.svm_destroy_model(h)
