"""CPU checks of the C ABI: the library builds for sm_103a, loads, and exports
every entry point that include/svm.h declares.  No kernel is launched."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_entry_points():
    text = open(os.path.join(ROOT, "include", "svm.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(svm_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def libsvm():
    from paper_2402_15281_gb300 import buildlib as b
    path = b.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_entry_points()
    for must in ("svm_create_model", "svm_load_weights", "svm_check_motions", "svm_destroy_model"):
        assert must in names


def test_library_exports_every_declared_symbol(libsvm):
    missing = [n for n in declared_entry_points() if not hasattr(libsvm, n)]
    assert not missing, missing


def test_status_strings(libsvm):
    libsvm.svm_status_string.restype = ctypes.c_char_p
    assert libsvm.svm_status_string(0) == b"ok"
    assert libsvm.svm_status_string(4) == b"device wait timed out"
    assert libsvm.svm_status_string(99) == b"unknown status"


def test_binding_raises_without_library(monkeypatch, tmp_path):
    import paper_2402_15281_gb300 as svm
    monkeypatch.setattr(svm, "_lib", None)
    monkeypatch.setattr(svm, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError):
        svm.lib()


def test_blob_layout():
    import numpy as np
    import struct
    import paper_2402_15281_gb300 as svm
    from paper_2402_15281_gb300 import synth as S
    layers = S.xavier_weights(16, 2, seed=1)
    blob = svm.make_blob(layers, tau=0.25)
    assert blob[:4] == b"SVMW"
    ver, nl, ind, w, act, tau = struct.unpack("<IIIIIf", blob[4:28])
    assert (ver, nl, ind, w, act, tau) == (1, 4, 15, 16, 0, 0.25)
    n = sum(W.size + b.size for W, b in layers)
    assert len(blob) == 28 + 8 * 4 + 4 * n
    o, i = struct.unpack("<II", blob[28:36])
    assert (o, i) == (16, 15)
    np.testing.assert_array_equal(np.frombuffer(blob[36:36 + 4 * 240], "<f4").reshape(16, 15), layers[0][0])


def test_binding_checks_buffers_before_the_call():
    """The binding refuses, before any library call, point buffers that are
    not (P, 4) float32 and output buffers shorter than what the call writes
    (one 32-byte record per motion or per path; M x P floats of f)."""
    import torch
    import paper_2402_15281_gb300 as svm
    with pytest.raises(ValueError, match="float32"):
        svm._points(torch.zeros((10, 4), dtype=torch.float64))
    with pytest.raises(ValueError, match="float32"):
        svm._points(torch.zeros((10, 3), dtype=torch.float32))
    with pytest.raises(ValueError, match="CUDA"):               # right shape, but host memory
        svm._points(torch.zeros((10, 4), dtype=torch.float32))
    with pytest.raises(ValueError, match="writes 256"):
        svm._out(torch.zeros((7, 32), dtype=torch.uint8), 32 * 8, "results")
    assert svm._n_records(9, svm.SVM_PATHS3) == 3 and svm._n_records(8, svm.SVM_PATHS2) == 4
    assert svm._n_records(5, svm.SVM_STRICT | svm.SVM_NO_EARLY_EXIT) == 5
