"""Host driver of the GPU trainer (svm_train_* in include/svm.h).

Only orchestration lives here: the epoch loop, the learning-rate schedule of
Sec. V (Adam at lr 1e-3, reduced by 10x after `patience` epochs without a
better validation error, best-validation weights kept) and the split of the
motions into training, validation and (optionally) test sets (60/25/15 by
motion in the paper).  Data generation, labels, forward, backward and
Adam run in the library's kernels.
"""
from __future__ import annotations

import time

import numpy as np

from . import synth as S


def bin_training_motions(robot, n, seed):
    """Motions like the bin-picking workload: 3/4 grasp motions into the bin
    (synth.bin_motions), 1/4 short uniform motions, in a seeded random order."""
    qa0, qa1 = S.bin_motions(robot, n - n // 4, seed=seed)
    qb0, qb1 = S.uniform_motions(robot, n // 4, seed=seed, max_step_deg=30)
    q0, q1 = np.concatenate([qa0, qb0]), np.concatenate([qa1, qb1])
    order = np.argsort(S.Rng(seed, 99).uniform(n))
    return q0[order], q1[order]


def path_training_motions(robot, n, seed):
    """Motions like the three-segment paths of Sec. V-C: the segments of
    n // 6 paths (synth.bin_paths: into the bin, between the vias, out of the
    bin) plus bin_training_motions for the rest, in a seeded random order."""
    n_paths = n // 6
    paths = S.bin_paths(robot, n_paths, seed=seed)
    pa0, pa1 = paths[:, :3].reshape(-1, 6), paths[:, 1:].reshape(-1, 6)
    qb0, qb1 = bin_training_motions(robot, n - len(pa0), seed)
    q0, q1 = np.concatenate([pa0, qb0]), np.concatenate([pa1, qb1])
    order = np.argsort(S.Rng(seed, 98).uniform(n))
    return q0[order], q1[order]


def grasp_training_motions(robot, n, seed):
    """Segments of the two-segment grasp motions of Sec. V-C (into and out of
    the bin, synth.bin_grasp_paths) for half of the n motions,
    bin_training_motions for the rest, in a seeded random order."""
    k = n // 8                         # k candidates give 4k segments
    into, out = S.bin_grasp_paths(robot, k, seed=seed)
    seg0 = np.concatenate([into[:, :2], out[:, :2]]).reshape(-1, 6)
    seg1 = np.concatenate([into[:, 1:], out[:, 1:]]).reshape(-1, 6)
    qb0, qb1 = bin_training_motions(robot, n - len(seg0), seed)
    q0, q1 = np.concatenate([seg0, qb0]), np.concatenate([seg1, qb1])
    order = np.argsort(S.Rng(seed, 97).uniform(n))
    return q0[order], q1[order]


def train_model(svm, robot, q0, q1, width=256, n_hidden=4, act=0, samples_per_motion=4096, steps=128,
                batch=65536, epochs=30, lr=1e-3, val_fraction=0.2, patience=10, data_seed=7, init_seed=2,
                device=0, log=None, box=None, test_fraction=0.0):
    """Train f on GPU-generated data for the motions (q0, q1); box = (lo, hi)
    sets the box of the uniformly drawn points.  The motions split in order
    into training, validation (val_fraction) and test (test_fraction) sets;
    data is generated for all of them.  Returns (blob of the best-validation
    weights, history dict); with a test set the history holds its mean
    absolute error under the best weights ("test_mae") and its sample range."""
    t0 = time.perf_counter()
    n = len(q0)
    n_te = int(round(n * test_fraction))
    n_val = max(1, int(round(n * val_fraction)))
    n_tr = n - n_val - n_te
    t = svm.svm_train_create(robot, width, n_hidden, act, batch, device)
    hist = {"epoch_loss": [], "val_mae": [], "lr": []}
    try:
        svm.svm_train_set_weights(t, svm.make_blob(S.xavier_weights(width, n_hidden, seed=init_seed), act=act))
        if box is not None:
            svm.svm_train_set_box(t, box[0], box[1])
        svm.svm_train_make_data(t, q0, q1, samples_per_motion, steps, data_seed)
        tr_end = n_tr * samples_per_motion
        va_end = (n_tr + n_val) * samples_per_motion
        best, best_blob, stale = np.inf, None, 0
        t_train = 0.0
        for e in range(epochs):
            te = time.perf_counter()
            loss = svm.svm_train_epoch(t, 0, tr_end, lr, 1000 + e)
            t_train += time.perf_counter() - te
            mae = svm.svm_train_evaluate(t, tr_end, va_end)
            hist["epoch_loss"].append(loss)
            hist["val_mae"].append(mae)
            hist["lr"].append(lr)
            if log:
                log(f"epoch {e}: train L1 {loss:.4f} m, val MAE {mae:.4f} m, lr {lr:g}")
            if mae < best:
                best, best_blob, stale = mae, svm.svm_train_get_weights(t), 0
            else:
                stale += 1
                if stale >= patience:
                    lr *= 0.1
                    stale = 0
        hist["best_val_mae"] = float(best)
        hist["train_samples"] = int(tr_end)
        hist["total_samples"] = int(n * samples_per_motion)
        if n_te > 0:
            svm.svm_train_set_weights(t, best_blob)
            hist["test_mae"] = float(svm.svm_train_evaluate(t, va_end, n * samples_per_motion))
            hist["test_motions"] = (n_tr + n_val, n)
        hist["samples_per_s"] = float(epochs * (tr_end // batch) * batch / max(t_train, 1e-9))
        hist["seconds"] = time.perf_counter() - t0
        return best_blob, hist
    finally:
        svm.svm_train_destroy(t)


def calibrate_tau(svm, model, robot, pts_d, margin, steps, q0, q1, band=0.05, safety=1.25):
    """Set the model's gate from calibration motions and return its offset:
    tau = safety * max(f - delta) over the calibration pairs whose exact
    distance is within margin + band (pairs that can collide), never below 0.
    The whole computation (network in the model's precision, exact labels,
    the maximum) runs in the library's svm_calibrate_gate."""
    tau, _, _ = svm.svm_calibrate_gate(model, q0, q1, pts_d, margin, steps, band, safety)
    return tau
