"""Host logic of the schedule autotuner (no GPU): the choice of the fastest
schedule, the parity gate before timing, the JSON table keyed by GPU, grid and
precision, and the committed table's consistency with the compiled schedules.
The GPU-facing parts (device name, timing, the parity run) are replaced by
fakes."""
import json

import pytest

from paper_2012_15133_gb300 import autotune as A


@pytest.fixture
def fake_gpu(monkeypatch, tmp_path):
    import paper_2012_15133_gb300.spfc as S
    cache = tmp_path / "tune.json"
    monkeypatch.setenv("SPFC_TUNE_CACHE", str(cache))
    monkeypatch.setattr(A, "_gpu_name", lambda: "Test GPU")
    monkeypatch.setattr(S, "num_schedules", lambda d, n: 4)
    # schedule s: resident 10 + |s - 2| us, flushed 20 - s us (sums 30, 28, 26, 26 -> first minimum 2)
    monkeypatch.setattr(A, "time_schedule", lambda n, p, s: (10.0 + abs(s - 2), 20.0 - s))
    monkeypatch.setattr(A, "check_schedule", lambda n, p, s: 0.0)
    return cache


def test_tune_picks_the_fastest_schedule_and_lookup_reads_it(fake_gpu):
    assert A.lookup(2, 256, "fp32") == 0          # no table yet
    best, results = A.tune(256, "fp32", verbose=False)
    assert best == 2 and sorted(results) == [0, 1, 2, 3]
    assert A.lookup(2, 256, "fp32") == 2
    assert A.lookup(2, 256, "fp64") == 0          # other precision: untuned
    assert A.lookup(2, 512, "fp32") == 0          # other grid: untuned
    table = json.loads(fake_gpu.read_text())
    assert list(table) == ["Test GPU|d2|n256|fp32"]
    assert table["Test GPU|d2|n256|fp32"]["timings"]["3"]["flushed_us"] == 17.0
    # a second grid is added, the first kept
    A.tune(128, "fp64", verbose=False)
    assert A.lookup(2, 256, "fp32") == 2 and A.lookup(2, 128, 0) == 2


def test_a_schedule_that_disagrees_is_refused_before_timing(fake_gpu, monkeypatch):
    monkeypatch.setattr(A, "check_schedule", lambda n, p, s: 1e-3 if s == 3 else 0.0)
    with pytest.raises(RuntimeError, match="schedule 3"):
        A.tune(256, "fp32", verbose=False)
    assert not fake_gpu.exists()
    # the gate follows the precision: 1e-12 on the float64 path, 1e-5 on float32
    monkeypatch.setattr(A, "check_schedule", lambda n, p, s: 1e-9)
    assert A.tune(256, "fp32", verbose=False)[0] == 2
    with pytest.raises(RuntimeError):
        A.tune(256, "fp64", verbose=False)


def test_a_damaged_table_reads_as_untuned_and_is_rewritten(fake_gpu):
    fake_gpu.write_text("{not json")
    assert A.lookup(2, 256, "fp32") == 0
    A.tune(256, "fp32", verbose=False)
    assert A.lookup(2, 256, "fp32") == 2


def test_the_committed_table_names_compiled_schedules():
    from paper_2012_15133_gb300.spfc import num_schedules
    with open(A.DEFAULT_CACHE) as f:
        table = json.load(f)
    assert table
    from paper_2012_15133_gb300.autotune import batch_schedules
    for key, entry in table.items():
        gpu, d, n, prec = key.split("|")
        assert d in ("d2", "batch") and prec in ("fp32", "fp64")
        if d == "batch":
            assert entry["schedule"] in batch_schedules(int(n[1:])), key
            times = {int(s): t["step_us"] for s, t in entry["timings"].items()}
            assert set(times) == set(batch_schedules(int(n[1:]))), key
            assert entry["schedule"] == min(times, key=times.get), key
            continue
        assert 0 <= entry["schedule"] < num_schedules(2, int(n[1:])), key
        sums = {int(s): t["resident_us"] + t["flushed_us"] for s, t in entry["timings"].items()}
        assert entry["schedule"] == min(sums, key=sums.get), key


def test_batch_tuner_picks_the_fastest_and_lookup_reads_it(tmp_path, monkeypatch):
    """The batch tuner times every compiled batch schedule of a grid size (the
    GPU parts faked), refuses one that disagrees, and Batch(schedule="auto")
    reads the table."""
    monkeypatch.setenv("SPFC_TUNE_CACHE", str(tmp_path / "t.json"))
    monkeypatch.setattr(A, "_gpu_name", lambda: "FakeGPU")
    monkeypatch.setattr(A, "batch_schedules", lambda n: [0, 2, 4, 5])
    monkeypatch.setattr(A, "check_batch", lambda n, p, s: 0.0)
    monkeypatch.setattr(A, "time_batch", lambda n, p, s: {0: 30.0, 2: 25.0, 4: 20.0, 5: 22.0}[s])
    assert A.lookup_batch(512, "fp32") == -1
    best, res = A.tune_batch(512, "fp32", verbose=False)
    assert best == 4 and A.lookup_batch(512, "fp32") == 4 and A.lookup_batch(256, "fp32") == -1
    monkeypatch.setattr(A, "check_batch", lambda n, p, s: 1e-3 if s == 5 else 0.0)
    with pytest.raises(RuntimeError, match="batch schedule 5"):
        A.tune_batch(256, "fp32", verbose=False)
