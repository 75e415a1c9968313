"""The block architecture of Sec. IV-A (Fig. 2) on the tensor cores: BF16
operands, FP32 accumulation in TMEM, width 512 (the paper's 5x512 and 11x512
networks; its "16 bit" variant of the inference-time table).

* weight rounding: the library's rounded weights equal the oracle's
  quantiser bit for bit;
* kernel arithmetic: against the oracle that keeps the activations in
  bfloat16 between blocks as the kernel does (block_forward_rounded, same
  rounded weights): median within 2e-5 of the output scale; the remaining
  pairs are rounding decisions that flip where the FP32 and FP64 values
  straddle a bfloat16 boundary, bounded at the 99th percentile;
* accuracy against the plain FP64 network on the same weights: printed;
* a gated check: flagged counts, verdicts and d_min equal the oracle's
  combined check run on the kernel's own predictions (svm_eval_pairs runs
  the same kernel with the output stored);
* times at the paper's inference shapes (one motion x 1 000 / 3 000 /
  20 000 points), beside the FP32 path.
"""
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


def _model(svm, robot, P, prec, tau=float("inf")):
    width, nb = P["init"][0].shape[0], len(P["blocks"])
    h = svm.svm_create_model(robot, width, nb, 0, prec, 0, arch=svm.SVM_ARCH_BLOCKS)
    svm.svm_load_weights(h, svm.make_block_blob(P, tau=tau))
    return h


def _flatten(Q):
    out = [np.asarray(Q["init"][0]).ravel(), np.asarray(Q["init"][1]).ravel()]
    for blk in Q["blocks"]:
        out += [np.asarray(a).ravel() for a in blk]
    out += [np.asarray(Q["final"][0]).ravel(), np.asarray(Q["final"][1]).ravel()]
    return np.concatenate(out).astype(np.float32)


def _eval(svm, h, q0, q1, pts):
    f = torch.empty((len(q0), len(pts)), device="cuda")
    svm.svm_eval_pairs(h, q0, q1, torch.from_numpy(pts).cuda(), f)
    torch.cuda.synchronize()
    return f.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("nb,n_motions,n_points", [(1, 3, 300), (2, 4, 5000), (5, 3, 300), (11, 2, 700)])
def test_block_tc_matches_oracle(svm, nb, n_motions, n_points):
    """Several 128-pair tiles per motion with a ragged tail; 4 x 5 000 points
    is 160 tiles, so some CTAs run a second tile on the same TMEM."""
    robot = S.make_robot(1)
    P = S.block_weights(512, nb, seed=500 + nb)
    Q = oracle.quantized_block_params(P, 1)
    q0, q1 = S.uniform_motions(robot, n_motions, seed=nb)
    pts = S.cube_cloud(n_points, seed=nb)
    h = _model(svm, robot, P, svm.SVM_BF16)
    try:
        np.testing.assert_array_equal(svm.svm_export_weights(h), _flatten(Q))
        got = _eval(svm, h, q0, q1, pts)
    finally:
        svm.svm_destroy_model(h)
    emu = oracle.block_pairs_rounded(Q, q0, q1, pts)
    ref = oracle.block_pairs(Q, q0, q1, pts)
    scale = max(1.0, np.abs(ref).max())
    e_emu, e_ref = np.abs(got - emu), np.abs(got - ref)
    print(f"BF16 blocks {nb}x512, {n_motions}x{n_points}: |f| up to {np.abs(ref).max():.2f}; vs emulation median "
          f"{np.median(e_emu):.1e} p99 {np.quantile(e_emu, 0.99):.1e} max {e_emu.max():.1e}; vs FP64 (same "
          f"weights) median {np.median(e_ref):.1e} p99 {np.quantile(e_ref, 0.99):.1e} max {e_ref.max():.1e}")
    assert np.isfinite(got).all()
    assert np.median(e_emu) <= 2e-5 * scale
    assert np.quantile(e_emu, 0.99) <= 5e-3 * scale


def test_block_tc_gated_check(svm):
    """Flags, verdicts and distances of a gated check equal the oracle's
    combined check on the kernel's own predictions and the FP32 gate."""
    robot = S.make_robot(1)
    P = S.block_weights(512, 3, seed=9)
    q0, q1 = S.uniform_motions(robot, 6, seed=9, max_step_deg=25)
    pts = S.cube_cloud(2000, seed=9)
    eps, N = 0.05, 32
    h = _model(svm, robot, P, svm.SVM_BF16)
    try:
        fk = _eval(svm, h, q0, q1, pts)
        # a gate above the margin in a gap of the predictions, from their 30th percentile up
        fs = np.sort(fk.ravel())
        k = max(int(0.3 * len(fs)), int(np.searchsorted(fs, eps + 0.01)))
        while fs[k + 1] - fs[k] < 1e-4:
            k += 1
        gate = float(np.float32(0.5 * (fs[k] + fs[k + 1])))
        svm.svm_set_gate(h, gate - eps)
        gate32 = float(np.float32(np.float32(eps) + np.float32(gate - eps)))
        res = svm.new_results(6)
        svm.svm_check_motions(h, q0, q1, torch.from_numpy(pts).cuda(), eps, N, svm.SVM_NO_EARLY_EXIT, res)
        torch.cuda.synchronize()
        r = svm.results_to_numpy(res)[:6]
    finally:
        svm.svm_destroy_model(h)
    ref = oracle.check_motions(None, 512, 3, 0, robot, q0, q1, N, pts, eps, gate32, f=fk)
    assert np.all(r["status"] == 0)
    np.testing.assert_array_equal(r["n_flagged"].astype(np.int64), ref["n_flagged"])
    np.testing.assert_array_equal(r["collision"], ref["collision"])
    np.testing.assert_array_equal(r["dhat_min"].astype(np.float64), ref["dhat_min"])
    fin = np.isfinite(ref["d_min"])
    assert np.all(np.abs(r["d_min"][fin] - ref["d_min"][fin]) <= 1e-5)
    assert 0 < ref["collision"].sum() < 6


def test_block_tc_times_at_the_paper_shapes(svm):
    """Network time of one motion x n points (prediction only: the network and
    the per-motion minimum), CUDA events, median of 50 calls after warm-up, for
    the BF16 tensor-core kernel and the FP32 path on the same weights."""
    robot = S.make_robot(1)
    q0, q1 = S.uniform_motions(robot, 1, seed=0)
    rows = []
    for nb in (5, 11):
        P = S.block_weights(512, nb, seed=1)
        for prec, name in ((svm.SVM_BF16, "BF16"), (svm.SVM_FP32, "FP32")):
            h = _model(svm, robot, P, prec)
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
                    rows.append((f"{nb}x512 {name}", n, float(np.median(ts))))
            finally:
                svm.svm_destroy_model(h)
    for name, n, ms in rows:
        print(f"block network {name}, 1 motion x {n} points: {ms:.3f} ms")
    assert all(ms > 0 for _, _, ms in rows)


def test_block_tc_throughput_roofline(svm):
    """The tensor-core block kernel on a large workload: 16 motions x a
    200 000-point bin cloud (3.2 M pairs, 25 008 tiles), prediction only.  The
    network phase (CUDA events inside the library) against the algorithmic
    FLOP per pair, 2 (3 W + L W^2 + (L - 1) 3 W + W + 3) (x-parts, h-parts and
    the final layer; the q-parts are per-motion constants), as a fraction of the
    measured burst BF16 peak."""
    import json
    import os
    robot = S.make_robot(1)
    pts = torch.from_numpy(S.bin_cloud(200_000, seed=0)).cuda()
    q0, q1 = S.bin_motions(robot, 16, seed=0)
    path = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "MEASURED_PEAKS.json")
    peak = json.load(open(path)).get("bf16_tflops", 1900.0) if os.path.exists(path) else 1900.0
    W = 512
    for nb in (5, 11):
        P = S.block_weights(W, nb, seed=1)
        h = _model(svm, robot, P, svm.SVM_BF16)
        try:
            svm.svm_profile_enable(h, True)
            res = svm.new_results(16)
            ms = []
            for k in range(8):
                svm.svm_check_motions(h, q0, q1, pts, 0.03, 64, svm.SVM_PREDICT_ONLY, res)
                if k >= 3:
                    ms.append(float(svm.svm_profile_read(h)[1]))
            torch.cuda.synchronize()
        finally:
            svm.svm_destroy_model(h)
        flop = 16 * 200_000 * 2 * (3 * W + nb * W * W + (nb - 1) * 3 * W + W + 3)
        t = float(np.median(ms))
        tf = flop / (t * 1e-3) / 1e12
        print(f"BF16 blocks {nb}x512, 16 motions x 200 000 points: network {t:.3f} ms = {tf:.0f} TFLOP/s = "
              f"{tf / peak:.2f} of the measured burst BF16 peak")
        assert tf > 0


def test_block_tc_bounded_wait_expiry_is_reported_and_recoverable(svm):
    """The block kernel's failure path, without a GPU fault: the test hook
    withholds CTA 0's first hand-over (its TMEM and input tile free for the
    first tile's layer 0), the MMA warp's wait expires after 2 s, every role
    leaves its loop, every record of that call carries status 1, and the next
    call on the same model and context gives the normal records."""
    import time
    robot = S.make_robot(1)
    P = S.block_weights(512, 3, seed=11)
    q0, q1 = S.uniform_motions(robot, 4, seed=11)
    pts = torch.from_numpy(S.cube_cloud(20000, seed=11)).cuda()
    h = _model(svm, robot, P, svm.SVM_BF16)
    try:
        res = svm.new_results(4)
        svm.svm_check_motions(h, q0, q1, pts, 0.05, 32, svm.SVM_NO_EARLY_EXIT, res)
        torch.cuda.synchronize()
        want = svm.results_to_numpy(res)[:4].copy()
        assert np.all(want["status"] == 0)
        svm.svm_test_expire_wait(h, 1)
        t = time.perf_counter()
        svm.svm_check_motions(h, q0, q1, pts, 0.05, 32, svm.SVM_NO_EARLY_EXIT, res)
        torch.cuda.synchronize()
        waited = time.perf_counter() - t
        bad = svm.results_to_numpy(res)[:4].copy()
        assert np.all(bad["status"] == 1) and 1.5 < waited < 30
        svm.svm_check_motions(h, q0, q1, pts, 0.05, 32, svm.SVM_NO_EARLY_EXIT, res)
        torch.cuda.synchronize()
        again = svm.results_to_numpy(res)[:4]
        assert np.all(again["status"] == 0)
        for k in ("collision", "d_min", "dhat_min", "n_flagged", "n_verified"):
            np.testing.assert_array_equal(again[k], want[k], err_msg=k)
    finally:
        svm.svm_destroy_model(h)
