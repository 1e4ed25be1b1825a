"""Host logic of the autotuner (CPU only): size bins, cache keys, the cache file and re-applying
cached choices for one GPU model (the timing itself needs a GPU)."""
import json

import pytest

torch = pytest.importorskip("torch")
import paper_1707_05141_gb300 as bs  # noqa: E402
from paper_1707_05141_gb300 import autotune  # noqa: E402


def test_size_bins_and_keys():
    assert [autotune._bin(x) for x in (1, 2, 3, 4, 5, 64, 65, 128, 256, 1000)] == [0, 1, 2, 2, 3, 6, 7, 7, 8, 8]
    assert autotune._key("GB300", bs.F32, 64, 40) == "GB300|f32|6|6"
    assert autotune._key("GB300", bs.F64, 32, 100) == "GB300|f64|7|5"     # bins of max(m, n), min(m, n)


def test_candidates_are_every_register_variant_then_the_shared_tier():
    nreg = bs.jacobi_variants(bs.F32, 64, 64, bs.TIER_REGISTER)
    c = autotune.candidates(bs.F32, 64, 64)
    assert c == [bs.TIER_REGISTER | (v << 8) for v in range(1, nreg + 1)] + [bs.TIER_SHARED]
    assert autotune.candidates(bs.F32, 300, 300) == []                    # beyond both tiers


def test_cache_roundtrip_and_damaged_file(tmp_path, monkeypatch):
    path = tmp_path / "autotune.json"
    monkeypatch.setattr(autotune, "CACHE", str(path))
    assert autotune._load() == {}
    autotune._store({"a|f32|6|6": {"tier": 257}})
    assert autotune._load() == {"a|f32|6|6": {"tier": 257}}
    path.write_text("{broken")
    assert autotune._load() == {}


def test_apply_cache_only_for_this_gpu_model(tmp_path, monkeypatch):
    path = tmp_path / "autotune.json"
    path.write_text(json.dumps({"GB300|f32|6|5": {"tier": 1 | (3 << 8)}, "OTHER|f64|5|5": {"tier": 2}}))
    monkeypatch.setattr(autotune, "CACHE", str(path))
    monkeypatch.setattr(torch.cuda, "get_device_name", lambda device=None: "GB300")
    calls = []
    monkeypatch.setattr(autotune, "set_jacobi_choice", lambda *a: calls.append(a))
    assert autotune.apply_cache() == 1
    assert calls == [(bs.F32, 64, 32, 1 | (3 << 8))]
