"""Host logic of the autotuner: the fastest candidate wins, failing candidates are skipped, results are cached per
signature and reused unless forced.  The timing is replaced by a table, so no GPU is needed."""
import json

import pytest

from paper_2601_10819_gb300 import msda, tune


@pytest.fixture
def fake_timing(tmp_path, monkeypatch):
    monkeypatch.setenv("MSDA_TUNE_CACHE", str(tmp_path / "tune.json"))
    monkeypatch.setattr(tune, "SHIPPED", str(tmp_path / "none.json"))
    table = {}
    calls = []

    def run(cand):
        calls.append(cand["warps"])
        if table[cand["warps"]] is None:
            raise msda.MSDAError("msda_forward", 2, "unsupported mapping")
        return table[cand["warps"]]

    monkeypatch.setattr(tune, "_time", lambda fn, reps=5: fn())
    return table, calls, run, tmp_path / "tune.json"


CANDS = [dict(vec=2, warps=w) for w in (2, 4, 8)]


def test_fastest_wins_and_failures_are_skipped(fake_timing):
    table, calls, run, path = fake_timing
    table.update({2: 3.0, 4: None, 8: 1.5})
    assert tune._best("fwd", "sigA", CANDS, run, force=False) == dict(vec=2, warps=8)
    stored = json.loads(path.read_text())["sigA"]
    assert stored["best"] == dict(vec=2, warps=8) and stored["ms"] == 1.5
    assert sorted(e["warps"] for e in stored["all"]) == [2, 8]


def test_cached_until_forced(fake_timing):
    table, calls, run, _ = fake_timing
    table.update({2: 1.0, 4: 2.0, 8: 3.0})
    assert tune._best("bwd", "sigB", CANDS, run, force=False)["warps"] == 2
    n = len(calls)
    table.update({2: 5.0, 4: 0.5, 8: 3.0})
    assert tune._best("bwd", "sigB", CANDS, run, force=False)["warps"] == 2  # from the cache, nothing timed
    assert len(calls) == n
    assert tune._best("bwd", "sigB", CANDS, run, force=True)["warps"] == 4
    assert tune._best("bwd", "sigOther", CANDS, run, force=False)["warps"] == 4


def test_no_valid_mapping_raises(fake_timing):
    table, _, run, _ = fake_timing
    table.update({2: None, 4: None, 8: None})
    with pytest.raises(RuntimeError):
        tune._best("fwd", "sigC", CANDS, run, force=False)


def test_shipped_table_is_read_and_well_formed():
    with open(tune.SHIPPED) as f:
        d = json.load(f)
    assert d, "the package ships measured mappings"
    for sig, e in d.items():
        assert sig.split("|")[1] in ("fwd", "bwd", "bwd-det", "batched"), sig
        assert e["best"]["vec"] in (0, 1, 2, 4) and e["best"]["warps"] in (0, 1, 2, 4, 8, 16) and e["ms"] > 0
