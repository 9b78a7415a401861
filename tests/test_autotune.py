"""The autotuner's selection logic on the CPU with a stand-in for the device
batch: it starts from the smallest nprobe whose full scan reaches the recall
target, raises nprobe per (Delta_d, schedule) until the target is met, keeps
the fastest configuration that meets it, tries the test on the completed
distance and the kernel knobs (scan kernel, queries per work unit) at the
chosen configuration for the learned estimator only, and falls back to the
best recall when nothing meets the target."""
import numpy as np

from paper_2404_16322_gb300 import autotune


class FakeBench:
    """Recall grows with nprobe (0.9 at 8, +0.02 per doubling step of the
    grid); time grows with nprobe and depends on (Delta_d, schedule)."""

    def __init__(self, estimator="learned", recall_shift=0.0, knob_ms=None, knob_recall=None):
        self.estimator = estimator
        self.shift = recall_shift
        self.knob_ms = knob_ms or {}  # (scan kernel, queries per unit) -> time offset
        self.knob_recall = knob_recall or {}
        self.calls = []
        self._last = None
        self.K = 10

    def _recall(self, nprobe, mode):
        grid = [8, 16, 24, 32, 48, 64, 96, 128]
        return min(1.0, 0.9 + 0.02 * grid.index(nprobe) + self.shift - (0.001 if mode == "prune" else 0.0))

    def run(self, nprobe, delta_d, mode, first_wave=1, stats=False, growth=0, final_test=False, scan_kernel="auto",
            queries_per_unit=0):
        self.calls.append((nprobe, delta_d, mode, first_wave, growth, final_test, scan_kernel, queries_per_unit))
        self._last = self._recall(nprobe, mode) + self.knob_recall.get((scan_kernel, queries_per_unit), 0.0)

    def result(self):
        # ids whose recall@10 against gt = arange(10) per query is _last
        hit = int(round(self._last * 10))
        row = np.concatenate([np.arange(hit), 100 + np.arange(10 - hit)])
        return np.tile(row, (4, 1))

    def time(self, nprobe, delta_d, mode, steps, warmup, first_wave=1, growth=0, final_test=False,
             scan_kernel="auto", queries_per_unit=0, graph=False):
        self.calls.append((nprobe, delta_d, mode, first_wave, growth, final_test, scan_kernel, queries_per_unit))
        ms = nprobe * (1.0 if mode == "full" else 0.5 + 0.01 * delta_d) + (0.3 if growth == 1 else 0.0)
        ms += 0.05 if final_test else 0.0
        ms += self.knob_ms.get((scan_kernel, queries_per_unit), 0.1)
        ms -= 0.001 * first_wave
        return ms * steps, [ms] * max(steps, 1)


GT = np.tile(np.arange(10), (4, 1))
NPROBES = (8, 16, 24, 32, 48, 64, 96, 128)


def test_picks_the_fastest_configuration_that_meets_the_target():
    b = FakeBench()
    best, tried = autotune.autotune(b, GT, 0.95, 10, (8, 16, 32), nprobes=NPROBES, mode="prune")
    # the full scan first reaches 0.95 at nprobe 32 (0.9 + 0.02 * 3 = 0.96)
    assert best["recall"] >= 0.95
    ok = [t for t in tried if t["recall"] >= 0.95]
    assert best["ms"] == min(t["ms"] for t in ok)
    assert best["delta_d"] == 8 and best["growth"] == 30 and best["nprobe"] == 32
    # nothing below the full scan's first passing nprobe was timed
    assert min(t["nprobe"] for t in tried) >= 32
    # the completed-distance test was tried once, on the best configuration, and lost
    fin = [t for t in tried if t["final_test"]]
    assert len(fin) == 1 and not best["final_test"]
    assert best["scan_kernel"] == "auto" and best["queries_per_unit"] == 0
    # every kernel knob was timed once, at the chosen configuration
    kn = [t for t in tried if (t["scan_kernel"], t["queries_per_unit"]) != ("auto", 0)]
    assert len(kn) == len(autotune.KNOBS) - 2
    assert all((t["nprobe"], t["delta_d"], t["growth"]) == (32, 8, 30) for t in kn)


def test_a_faster_kernel_knob_is_kept_unless_it_loses_recall():
    b = FakeBench(knob_ms={("auto", 0): 0.1, ("tensor", 64): -0.2, ("cuda", 8): -0.3},
                  knob_recall={("cuda", 8): -0.2})
    best, tried = autotune.autotune(b, GT, 0.95, 10, (8,), nprobes=NPROBES, mode="prune")
    # cuda/8 is fastest but falls below the target; tensor/64 is next
    assert (best["scan_kernel"], best["queries_per_unit"]) == ("tensor", 64)
    assert best["recall"] >= 0.95


def test_the_completed_distance_test_is_not_tried_for_opq():
    b = FakeBench(estimator="pq")
    best, tried = autotune.autotune(b, GT, 0.95, 10, (16,), nprobes=NPROBES, mode="prune")
    assert not any(t["final_test"] for t in tried)
    assert not any(c[5] for c in b.calls)
    assert all(c[6] == "auto" and c[7] == 0 for c in b.calls)


def test_full_mode_tunes_only_the_schedule():
    b = FakeBench()
    best, tried = autotune.autotune(b, GT, 0.95, 10, (8, 16, 32), nprobes=NPROBES, mode="full")
    assert {t["delta_d"] for t in tried} == {0} and best["mode"] == "full"


def test_falls_back_to_the_best_recall_when_the_target_is_out_of_reach():
    b = FakeBench(recall_shift=-0.5)
    best, tried = autotune.autotune(b, GT, 0.95, 10, (16,), nprobes=NPROBES, mode="prune")
    assert best["recall"] == max(t["recall"] for t in tried) and best["recall"] < 0.95
