"""Host logic of the autotuner (no GPU): the decisions it writes and the
merge of a partial run into an earlier table, with the kernel timings
replaced by a deterministic stand-in."""
import json

import paper_1412_1840_gb300 as cp
from paper_1412_1840_gb300 import tune as T


TENSOR_RATE = {8: 1.5, 12: 1.2, 16: 0.9, 32: 0.9, 48: 0.5}


def fake_timed(calls):
    """Pair rates that depend only on the form, the class and sigma_t: the
    direct form runs at 1.0 (cos form, sigma_t 0.3) or 0.8 (sin form,
    sigma_t 0.2); the tensor classes at TENSOR_RATE, so that 8 and 12 beat
    the cos form, 16 loses to it, 32 beats the sin form it is compared with
    and 48 loses to it."""
    def timed(t, y, e, off, grid, reps=2, sigma_t=0.3, **kw):
        calls.append((kw.get("form"), kw.get("n_max"), sigma_t))
        if kw.get("form") == cp.CP_FORM_TENSOR:
            rate = TENSOR_RATE[kw["n_max"]]
        else:
            rate = 1.0 if sigma_t >= 0.3 else 0.8
        return {"ms": 1.0, "pair_freq_per_s": rate}
    return timed


def test_decisions_and_sin_form_reference(monkeypatch):
    calls = []
    monkeypatch.setattr(T, "timed", fake_timed(calls))
    table = T.tune(n_freq=64, target_pair_freq=1e6, log=lambda *a: None)
    assert len(table["buckets"]) >= 3
    for b in table["buckets"]:
        assert b["direct_fc"] in (16, 8, 4, 2) and T.fc_fits(b["max_n"], b["direct_fc"])
        assert b["direct_sin_form"] == 0.8
        assert b["tensor"] == {"8": True, "12": True, "16": False, "32": True, "48": False}
    # the sin-form reference is timed at sigma_t 0.2, the fc sweep at 0.3
    assert any(f == cp.CP_FORM_DIRECT and s == 0.2 for f, _, s in calls)
    assert all(s == 0.3 for f, n, s in calls if f == cp.CP_FORM_TENSOR)
    t = cp.tuning_from(table)                                         # the binding accepts the table
    assert t.n_buckets == len(table["buckets"])


def test_merge_times_only_the_listed_classes(monkeypatch, tmp_path):
    calls = []
    monkeypatch.setattr(T, "timed", fake_timed(calls))
    base = T.tune(n_freq=64, target_pair_freq=1e6, classes=(8, 12, 16, 32), log=lambda *a: None)
    path = tmp_path / "base.json"
    path.write_text(json.dumps(base))
    calls.clear()
    merged = T.tune(n_freq=64, target_pair_freq=1e6, classes=(48,), base=json.loads(path.read_text()),
                    log=lambda *a: None)
    timed_classes = {n for f, n, _ in calls if f == cp.CP_FORM_TENSOR}
    assert timed_classes == {48}
    direct_cos = [c for c in calls if c[0] == cp.CP_FORM_DIRECT and c[2] == 0.3]
    assert direct_cos == []                                           # the fc sweep is kept, not redone
    for b0, b1 in zip(base["buckets"], merged["buckets"]):
        assert b1["direct_fc"] == b0["direct_fc"] and b1["direct"] == b0["direct"]
        for cls in ("8", "12", "16", "32"):
            assert b1["tensor"][cls] == b0["tensor"][cls]
        assert "48" in b1["tensor"] and "48" not in b0["tensor"]
