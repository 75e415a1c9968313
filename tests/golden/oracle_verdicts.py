"""The FP64 oracle's exact verdicts for every motion of the full-size
workloads, stored so that the GPU tests and the benchmark can compare every
verdict with the oracle without running it.

For each workload and each motion (or path segment) the stored record is the
exact check of Eq. 5 (Sec. IV-B): d(X, m) = min over the whole cloud of the
sampled swept-volume distance (Eqs. 1, 3, 4 sampled at N + 1 poses), and
"collision iff d(X, m) <= eps" (free iff d > eps_S).  It depends on the robot,
the motions and the cloud only, not on the network: a combined check whose
gate is wide enough must return exactly these verdicts.

Workloads (drawn by paper_2402_15281_gb300.synth, seeds fixed there):
  bin_picking   64 grasp motions x a 200 000-point bin cloud, eps 0.03 m,
                128 steps (the benchmark's workload);
  uneven_batch  32 bin scenes, log-uniform 10k-500k points each, 16 motions
                per scene (512 motions), eps 0.03 m, 128 steps;
  paths3        128 three-segment paths (384 segments) x a 300 000-point bin
                cloud, eps 0.03 m, 128 steps; one record per segment.

Each record also stores a SHA-256 of the inputs it was computed from.  Where
another machine draws different inputs (the clouds use transcendental
functions whose last bit may differ between platforms), ``load`` sees the
digest differ and runs the oracle on that machine's inputs instead.

Run ``python tests/golden/oracle_verdicts.py`` to rewrite
``oracle_verdicts.json`` (about five minutes on 8 cores).  Only the oracle
computes the stored values.
"""
from __future__ import annotations

import json
import os
import sys
import time

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_ROOT = os.path.dirname(os.path.dirname(_HERE))
if _ROOT not in sys.path:
    sys.path.insert(0, _ROOT)

from paper_2402_15281_gb300 import synth as S  # noqa: E402

PATH = os.path.join(_HERE, "oracle_verdicts.json")
EPS = 0.03
STEPS = 128


def inputs(name):
    """(robot, list of (points, q0, q1) groups, digest) of a workload; the
    records of the groups follow one another in motion order."""
    if name == "bin_picking":
        robot, pts, q0, q1 = S.bin_picking_workload(0)
        return robot, [(pts, q0, q1)], S.inputs_digest(pts, q0, q1)
    if name == "uneven_batch":
        robot, sizes, clouds, q0, q1, scene = S.uneven_batch_workload()
        groups = []
        for s, c in enumerate(clouds):
            sel = scene == s
            groups.append((c, q0[sel], q1[sel]))
        return robot, groups, S.inputs_digest(np.concatenate(clouds), q0, q1, scene)
    if name == "paths3":
        robot, pts, q0, q1 = S.three_segment_path_workload()
        return robot, [(pts, q0, q1)], S.inputs_digest(pts, q0, q1)
    raise KeyError(name)


def compute(name, loaded=None):
    """Run the oracle (Eq. 5 per motion) on a workload.  Returns the record:
    dict(inputs_sha256, eps, steps, collision (list of 0/1), d_min (list))."""
    import oracle
    robot, groups, digest = loaded if loaded is not None else inputs(name)
    dmin, coll = [], []
    for pts, q0, q1 in groups:
        d, c = oracle.gcc_motion(robot, q0, q1, STEPS, pts, EPS)
        dmin.append(d)
        coll.append(c)
    return {"inputs_sha256": digest, "eps": EPS, "steps": STEPS,
            "collision": [int(v) for v in np.concatenate(coll)],
            "d_min": [float(v) for v in np.concatenate(dmin)]}


def stored(name):
    """The stored record of a workload, or None."""
    if not os.path.exists(PATH):
        return None
    return json.load(open(PATH)).get(name)


def load(name, digest, loaded=None):
    """(collision (M,) int, d_min (M,) float64, source) for a workload whose
    inputs have the given digest: the stored record if its digest matches,
    else the oracle run here on these inputs (source says which)."""
    rec = stored(name)
    if rec is None or rec["inputs_sha256"] != digest:
        rec = compute(name, loaded)
        src = "oracle run on this machine (stored inputs differ)"
    else:
        src = "stored oracle record"
    return np.array(rec["collision"], dtype=np.int64), np.array(rec["d_min"], dtype=np.float64), src


def main():
    out = {"what": "FP64 oracle, Eq. 5 per motion: collision iff min over the cloud of the sampled "
                   "swept-volume distance <= eps; written by tests/golden/oracle_verdicts.py"}
    for name in ("bin_picking", "uneven_batch", "paths3"):
        t = time.perf_counter()
        rec = compute(name)
        out[name] = rec
        print(f"{name}: {len(rec['collision'])} records, {sum(rec['collision'])} collisions, "
              f"{time.perf_counter() - t:.1f} s", flush=True)
    with open(PATH, "w") as f:
        json.dump(out, f)
        f.write("\n")


if __name__ == "__main__":
    main()
