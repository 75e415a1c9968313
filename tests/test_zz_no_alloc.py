"""The allocation-free check entry point against svm_check_motions.

svm_check_motions_noalloc is for callers that cannot allocate device memory
while they check motions: a real-time loop whose memory is fixed at start-up,
or a process whose device memory belongs to another framework's allocator.
It runs the same kernels with its scratch in one fixed device array, so its
results must equal svm_check_motions' on the same inputs: verdicts and flag
counts exactly, distances within the 1e-5 m used by the other tests.  It is
called twice in a row, so the second call runs on scratch that still holds
the first call's contents; its exact check of every pair is also compared
with the FP64 oracle (Eq. 5).  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2402_15281_gb300 import synth as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DIST_TOL = 1e-5


@pytest.fixture(scope="module")
def svm():
    import paper_2402_15281_gb300 as svm
    svm.build()
    return svm


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("flags", [2, 0, 3])
def test_noalloc_matches_check_motions(svm, prec, flags):
    robot = S.make_robot(1)
    q0, q1 = S.bin_motions(robot, 24, seed=5)
    pts = torch.from_numpy(S.bin_cloud(30000, seed=5)).cuda()
    layers = S.xavier_weights(256, 4, seed=2)
    layers[-1] = (layers[-1][0], np.array([0.02], dtype=np.float32))
    h = svm.svm_create_model(robot, 256, 4, 0, prec, 0)
    try:
        svm.svm_load_weights(h, svm.make_blob(layers, tau=0.0))
        res = svm.new_results(24)
        svm.svm_check_motions(h, q0, q1, pts, 0.03, 128, flags, res)
        torch.cuda.synchronize()
        want = svm.results_to_numpy(res)[:24]
        q0d = torch.from_numpy(q0).cuda()
        q1d = torch.from_numpy(q1).cuda()
        for _ in range(2):
            got_t = svm.new_results(24)
            svm.svm_check_motions_noalloc(h, q0d, q1d, pts, 0.03, 128, flags, got_t)
            torch.cuda.synchronize()
            got = svm.results_to_numpy(got_t)[:24]
            assert np.all(got["status"] == 0)
            np.testing.assert_array_equal(got["collision"], want["collision"])
            np.testing.assert_array_equal(got["n_flagged"], want["n_flagged"])
            np.testing.assert_array_equal(got["dhat_min"], want["dhat_min"])
            if flags & svm.SVM_NO_EARLY_EXIT:
                np.testing.assert_array_equal(got["n_verified"], want["n_verified"])
                assert np.all(np.abs(got["d_min"] - want["d_min"]) <= DIST_TOL)
            else:   # early exit: the first collision found is not unique, the verdict is
                assert np.all(got["d_min"][got["collision"] == 1] <= 0.03 + DIST_TOL)
            assert 0 < want["collision"].sum() < 24
    finally:
        svm.svm_destroy_model(h)


def test_noalloc_rejects_calls_beyond_its_scratch(svm):
    robot = S.make_robot(1)
    h = svm.svm_create_model(robot, 256, 4, 0, 0, 0)
    try:
        svm.svm_load_weights(h, svm.make_blob(S.xavier_weights(256, 4, seed=2)))
        q = torch.zeros((64, 6), dtype=torch.float64, device="cuda")
        pts = torch.zeros((200000, 4), dtype=torch.float32, device="cuda")
        res = svm.new_results(64)
        with pytest.raises(svm.SvmError) as e:
            svm.svm_check_motions_noalloc(h, q, q, pts, 0.03, 128, 0, res)
        assert e.value.status == svm.SVM_E_INVALID and "32 MiB" in str(e.value)
    finally:
        svm.svm_destroy_model(h)


def test_noalloc_exact_check_equals_oracle(svm):
    """The geometric check of every pair through the allocation-free entry
    point, twice in a row: verdicts equal the FP64 oracle's (Eq. 5, free iff
    d > eps) and d(X, m) is within 1e-5 m of it."""
    robot = S.make_robot(1)
    q0, q1 = S.bin_motions(robot, 24, seed=6)
    cloud = S.bin_cloud(30000, seed=6)
    dmin, coll = oracle.gcc_motion(robot, q0, q1, 128, cloud, 0.03)
    assert 0 < coll.sum() < 24
    pts = torch.from_numpy(cloud).cuda()
    h = svm.svm_create_model(robot, 256, 4, 0, 1, 0)
    try:
        q0d = torch.from_numpy(q0).cuda()
        q1d = torch.from_numpy(q1).cuda()
        for _ in range(2):
            res = svm.new_results(24)
            svm.svm_check_motions_noalloc(h, q0d, q1d, pts, 0.03, 128, svm.SVM_VERIFY_ALL | svm.SVM_NO_EARLY_EXIT,
                                          res)
            torch.cuda.synchronize()
            got = svm.results_to_numpy(res)[:24]
            assert np.all(got["status"] == 0)
            np.testing.assert_array_equal(got["collision"], coll)
            assert np.abs(got["d_min"] - dmin).max() <= DIST_TOL
    finally:
        svm.svm_destroy_model(h)


def test_noalloc_rejects_host_and_misaligned_joint_arrays(svm):
    """q0/q1 are read on the device: a host array or one that is not 8-byte
    aligned is refused with SVM_E_INVALID before anything is launched."""
    robot = S.make_robot(1)
    h = svm.svm_create_model(robot, 256, 4, 0, 0, 0)
    try:
        svm.svm_load_weights(h, svm.make_blob(S.xavier_weights(256, 4, seed=2)))
        pts = torch.zeros((1000, 4), dtype=torch.float32, device="cuda")
        res = svm.new_results(4)
        qd = torch.zeros((4, 6), dtype=torch.float64, device="cuda")
        qh = np.zeros((4, 6))
        raw = torch.zeros(4 * 6 * 8 + 16, dtype=torch.uint8, device="cuda")
        L = svm.lib()
        vp = ctypes.c_void_p
        for a, b in ((qh.ctypes.data, qd.data_ptr()), (qd.data_ptr(), qh.ctypes.data),
                     (raw.data_ptr() + 4, qd.data_ptr())):
            st = L.svm_check_motions_noalloc(h, vp(a), vp(b), 4, vp(pts.data_ptr()), 1000, ctypes.c_float(0.03),
                                             16, 0, vp(res.data_ptr()), None)
            assert st == svm.SVM_E_INVALID
            assert "q0/q1" in L.svm_last_error(h).decode()
        torch.cuda.synchronize()
    finally:
        svm.svm_destroy_model(h)
