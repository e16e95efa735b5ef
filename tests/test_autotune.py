"""Host logic of the polarization autotuner: shape buckets, the choice under the error bound,
and the JSON cache (no GPU: the measurement is a stand-in)."""
import importlib.util
import json
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _autotune():
    spec = importlib.util.spec_from_file_location(
        "gw_autotune", os.path.join(ROOT, "paper_1003_0316_gb300", "autotune.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_buckets():
    at = _autotune()
    assert at.bucket(600, 409600, 16, "X") == "X|nb640|K524288|nw16"
    assert at.bucket(640, 300000, 16, "X") == at.bucket(601, 262144, 16, "X")
    assert at.bucket(641, 409600, 16, "X") != at.bucket(640, 409600, 16, "X")


def test_choice_respects_the_bound_and_the_cache(tmp_path):
    at = _autotune()
    calls = []

    def fake(c, nb, K, nw):
        calls.append(c)
        # BF16x3 is faster but (here) less accurate than the bound; b_stages 6 and larger
        # groups faster
        ms = (1.0 if c["precision"] == "bf16x3" else 2.0) - 0.1 * (c["b_stages"] == 6) \
            - 0.01 * c["group_items_per_sm"]
        err = 3e-6 if c["precision"] == "bf16x3" else 2e-7
        return ms, err

    path = str(tmp_path / "cache.json")
    e = at.tune(600, 409600, 16, cache_path=path, measure=fake, device_name="X", bound=1e-6)
    assert e["precision"] == "tf32x3" and e["b_stages"] == 6 and e["group_items_per_sm"] == 8
    assert not e["cached"] and len(calls) == len(at.candidates())
    assert at.options_of(e, accumulate=True) == {"b_stages": 6, "group_items_per_sm": 8,
                                                 "accumulate": True}
    # a looser bound admits BF16x3; a new key, so it is measured again
    e2 = at.tune(600, 409600, 16, cache_path=path, measure=fake, device_name="X", bound=1e-5)
    assert e2["precision"] == "bf16x3"
    # the same shape again comes from the file, without measuring
    n = len(calls)
    e3 = at.tune(620, 400000, 16, cache_path=path, measure=fake, device_name="X", bound=1e-6)
    assert e3["cached"] and len(calls) == n and e3["precision"] == "tf32x3"
    d = json.load(open(path))
    assert len(d) == 2 and all("tried" in v and len(v["tried"]) == len(at.candidates())
                               for v in d.values())


def test_no_precision_within_the_bound_raises(tmp_path):
    at = _autotune()
    import pytest
    with pytest.raises(RuntimeError):
        at.tune(300, 1000, 8, cache_path=str(tmp_path / "c.json"),
                measure=lambda c, nb, K, nw: (1.0, 1e-3), device_name="X")
    assert at.select([{"precision": "bf16x3", "b_stages": 4, "group_items_per_sm": 4,
                       "ms": 1.0, "err": None}], 1e-6) is None
