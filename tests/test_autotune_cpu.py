"""Host logic of the autotune cache (no GPU): keys, hits, misses, disabled cache."""
import json

import pytest

from paper_1310_1871_gb300 import amlbm, autotune


class _FakeLib:
    def amlbm_version(self):
        return b"amlbm test"


@pytest.fixture
def fake(monkeypatch, tmp_path):
    torch = pytest.importorskip("torch")
    calls = []

    def raw(specs, storage, steps=20, stream=None):
        calls.append((len(specs), storage))
        return "fused", (26, 16), [{"schedule": "fused", "tile": [26, 16], "ms_per_step": 0.05, "mlups": 1.0}]

    monkeypatch.setattr(amlbm, "load", lambda *a, **k: _FakeLib())
    monkeypatch.setattr(amlbm, "autotune_raw", raw)
    monkeypatch.setattr(torch.cuda, "get_device_name", lambda *a: "FakeGPU")
    path = tmp_path / "tune.json"
    monkeypatch.setenv("AMLBM_TUNE_CACHE", str(path))
    return calls, path


def specs(n=3):
    return [amlbm.InstanceSpec(40 + 8 * k, 20 + 4 * k) for k in range(n)]


def test_first_call_measures_and_second_hits_cache(fake):
    calls, path = fake
    a = autotune.tune(specs(), "bf16")
    assert not a["cached"] and a["schedule"] == "fused" and a["tile"] == [26, 16]
    b = autotune.tune(specs(), "bf16")
    assert b["cached"] and b["tile"] == [26, 16]
    assert len(calls) == 1
    assert len(json.load(open(path))) == 1


def test_key_depends_on_shapes_storage_and_device_not_on_tau():
    s = specs()
    k = autotune.signature(s, "bf16", "GPU", "v")
    assert k != autotune.signature(s, "f32", "GPU", "v")
    assert k != autotune.signature(s, "bf16", "GPU2", "v")
    assert k != autotune.signature(specs(4), "bf16", "GPU", "v")
    s2 = specs()
    s2[1].tau = 0.7
    s2[2].G = -4.8
    assert k == autotune.signature(s2, "bf16", "GPU", "v")
    s2[0].axisym = False
    assert k != autotune.signature(s2, "bf16", "GPU", "v")


def test_cache_off_always_measures(fake, monkeypatch):
    calls, path = fake
    monkeypatch.setenv("AMLBM_TUNE_CACHE", "off")
    autotune.tune(specs(), "f32")
    autotune.tune(specs(), "f32")
    assert len(calls) == 2 and not path.exists()


def test_corrupt_cache_file_is_ignored(fake):
    calls, path = fake
    path.write_text("{not json")
    r = autotune.tune(specs(), "bf16")
    assert not r["cached"] and len(calls) == 1
    assert autotune.tune(specs(), "bf16")["cached"]
