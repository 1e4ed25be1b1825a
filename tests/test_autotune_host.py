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


def test_block_choice_arguments_and_cache_keys(tmp_path, monkeypatch):
    """The block tier's table (host checks only) and its keys: bins of max(m, n), min(m, n) up to
    16384 and the base method; a cached block entry is re-applied for the same GPU model."""
    L = bs.lib()
    assert L.bsvd_set_block_choice(0, 512, 512, 32, 10) == 0
    assert L.bsvd_set_block_choice(0, 512, 512, 0, 0) == 0                 # clears the entry
    assert L.bsvd_set_block_choice(2, 512, 512, 32, 0) == -1
    assert L.bsvd_set_block_choice(0, 20000, 512, 32, 0) == -2
    assert L.bsvd_set_block_choice(0, 512, 512, 24, 0) == -4
    assert L.bsvd_set_block_choice(0, 512, 512, 0, 3) == -5
    assert autotune._block_key("GB300", bs.F32, 512, 300, bs.BLOCK_GRAM | bs.BLOCK_QR_PRECONDITION) == \
        "block|GB300|f32|9|9|0"
    assert autotune._block_key("GB300", bs.F64, 4000, 20000, bs.BLOCK_DIRECT) == "block|GB300|f64|14|12|1"
    c = autotune.block_candidates(bs.F32, bs.BLOCK_GRAM)
    assert [w for w, _ in c] == [16, 16, 16, 32, 32, 32] and c[0][1] == 0 and c[3][1] == 0
    for (w, k), pre in zip(c[1:3] + c[4:6], (1, 0, 1, 0)):
        d = bs.jacobi_variant_desc(bs.F32, 2 * w, 2 * w, k)
        assert d["qr_precond"] == pre and d["carried_norms"]
    assert autotune.block_candidates(bs.F32, bs.BLOCK_DIRECT) == [(16, 0), (32, 0)]
    path = tmp_path / "autotune.json"
    path.write_text(json.dumps({"block|GB300|f32|9|9|0": {"block_width": 16, "inner_variant": 13},
                                "block|OTHER|f32|9|9|0": {"block_width": 32, "inner_variant": 0}}))
    monkeypatch.setattr(autotune, "CACHE", str(path))
    monkeypatch.setattr(torch.cuda, "get_device_name", lambda device=None: "GB300")
    calls = []
    monkeypatch.setattr(autotune, "set_block_choice", lambda *a: calls.append(a))
    assert autotune.apply_cache() == 1
    assert calls == [(bs.F32, 512, 512, 16, 13)]


def test_block_width_zero_resolves_through_the_table():
    """block_width = 0 in the workspace query takes the recorded block width for the size bin (the
    call resolves it the same way), and 32 when nothing is recorded (host only)."""
    L = bs.lib()
    w32 = L.batched_svd_block_jacobi_workspace(0, 10, 512, 512, 32, 0)
    w16 = L.batched_svd_block_jacobi_workspace(0, 10, 512, 512, 16, 0)
    assert w32 > 0 and w16 > 0 and w16 != w32
    try:
        assert L.bsvd_set_block_choice(0, 512, 512, 0, 0) == 0
        assert L.batched_svd_block_jacobi_workspace(0, 10, 512, 512, 0, 0) == w32
        assert L.bsvd_set_block_choice(0, 400, 300, 16, 0) == 0              # the same size bin (512, 512)
        assert L.batched_svd_block_jacobi_workspace(0, 10, 512, 512, 0, 0) == w16
        assert L.batched_svd_block_jacobi_workspace(0, 10, 200, 200, 0, 0) == \
            L.batched_svd_block_jacobi_workspace(0, 10, 200, 200, 32, 0)        # another bin: untouched
    finally:
        L.bsvd_set_block_choice(0, 512, 512, 0, 0)
