"""Host logic of the training driver on the CPU, with the GPU trainer replaced
by a fake that records its calls: the split of the motions into training and
validation samples, the learning-rate schedule of Sec. V (reduce by 10x after
`patience` epochs without a better validation error) and the return of the
best-validation weights."""
import numpy as np

from paper_2402_15281_gb300 import synth as S
from paper_2402_15281_gb300 import training


class FakeTrainer:
    def __init__(self, val_maes):
        self.val_maes = list(val_maes)
        self.calls = []
        self.epoch = 0

    # the svm_train_* surface train_model uses
    def svm_train_create(self, robot, width, n_hidden, act, batch, device):
        self.calls.append(("create", width, n_hidden, act, batch))
        return "handle"

    def svm_train_set_weights(self, t, blob):
        self.calls.append(("set_weights", len(blob)))

    def svm_train_set_box(self, t, lo, hi):
        self.calls.append(("set_box", tuple(lo), tuple(hi)))

    def svm_train_make_data(self, t, q0, q1, spm, steps, seed):
        self.calls.append(("make_data", len(q0), spm, steps, seed))

    def svm_train_epoch(self, t, begin, end, lr, seed):
        self.calls.append(("epoch", begin, end, lr, seed))
        return 1.0 / (1 + self.epoch)

    def svm_train_evaluate(self, t, begin, end):
        self.calls.append(("evaluate", begin, end))
        mae = self.val_maes[self.epoch]
        self.epoch += 1
        return mae

    def svm_train_get_weights(self, t):
        return f"weights after epoch {self.epoch - 1}".encode()

    def svm_train_destroy(self, t):
        self.calls.append(("destroy",))

    def make_blob(self, layers, act=0, tau=float("inf")):
        return b"blob"


def test_split_schedule_and_best_weights():
    robot = S.make_robot(1)
    q0, q1 = S.uniform_motions(robot, 10, seed=1)
    # validation error: improves, stalls for 3 epochs (patience 3 -> lr / 10), improves, stalls 3 again
    maes = [0.5, 0.4, 0.41, 0.42, 0.43, 0.3, 0.31, 0.32, 0.33, 0.35]
    fake = FakeTrainer(maes)
    blob, hist = training.train_model(fake, robot, q0, q1, width=64, n_hidden=2, samples_per_motion=100,
                                      steps=8, batch=256, epochs=10, lr=1e-3, val_fraction=0.2, patience=3,
                                      box=((-1, -1, 0), (1, 1, 2)))
    epochs = [c for c in fake.calls if c[0] == "epoch"]
    evals = [c for c in fake.calls if c[0] == "evaluate"]
    # 10 motions, 2 for validation: training samples [0, 800), validation [800, 1000), split by motion
    assert all(c[1:3] == (0, 800) for c in epochs) and all(c[1:] == (800, 1000) for c in evals)
    lrs = [c[3] for c in epochs]
    np.testing.assert_allclose(lrs, [1e-3] * 5 + [1e-4] * 4 + [1e-5])
    assert hist["lr"] == lrs and hist["val_mae"] == maes
    assert hist["best_val_mae"] == 0.3 and blob == b"weights after epoch 5"
    assert [c[4] for c in epochs] == [1000 + e for e in range(10)]          # a new shuffle per epoch
    assert ("set_box", (-1, -1, 0), (1, 1, 2)) in fake.calls and fake.calls[-1] == ("destroy",)


def test_trainer_is_destroyed_when_a_call_fails():
    class Failing(FakeTrainer):
        def svm_train_epoch(self, *a):
            raise RuntimeError("device error")

    robot = S.make_robot(1)
    q0, q1 = S.uniform_motions(robot, 4, seed=2)
    fake = Failing([0.1])
    try:
        training.train_model(fake, robot, q0, q1, epochs=1)
    except RuntimeError:
        pass
    assert fake.calls[-1] == ("destroy",)


def test_calibrate_tau_calls_the_library():
    """The host driver holds no gate arithmetic: calibrate_tau passes the
    calibration set, margin, steps, band (0.05 m) and safety factor (1.25) to
    the library's svm_calibrate_gate and returns the tau it computed (the GPU
    test test_gpu_gate.py checks that value)."""
    calls = []

    class Fake:
        def svm_calibrate_gate(self, model, q0, q1, pts, margin, steps, band, safety):
            calls.append((model, q0, q1, pts, margin, steps, band, safety))
            return 0.0421, 0.0337, 17

    q = np.zeros((2, 6))
    assert training.calibrate_tau(Fake(), "h", None, "pts", 0.03, 8, q, q) == 0.0421
    assert calls == [("h", q, q, "pts", 0.03, 8, 0.05, 1.25)]
