"""The autotuner's record table (host logic, no GPU)."""
import json

from paper_math_9809043_gb300 import tune as TU


def test_key_of_is_stable():
    assert TU.key_of({}) == "default"
    assert TU.key_of({"fuse_width": 64, "plain_sweeps": 0}) == "fuse_width=64,plain_sweeps=0"


def test_record_and_best_roundtrip(tmp_path):
    path = str(tmp_path / "t.json")
    assert TU.best("GPU X", "w", path) is None
    table = TU.record(TU.load_table(path), "GPU X", "w", {"fuse_width": 96}, {"default": 2.0, "fuse_width=96": 1.5})
    with open(path, "w") as f:
        json.dump(table, f)
    assert TU.best("GPU X", "w", path) == {"fuse_width": 96}
    assert TU.best("GPU Y", "w", path) is None
    assert TU.best("GPU X", "v", path) is None


def test_candidates_are_option_fields():
    from paper_math_9809043_gb300 import msrcg as M
    names = {f[0] for f in M.Opts._fields_}
    for cand in TU.CANDIDATES:
        assert set(cand) <= names, cand
    assert "inner_floor" in names and TU.FLOORS[0] == 1e-6  # the second stage's field; the first is the default
