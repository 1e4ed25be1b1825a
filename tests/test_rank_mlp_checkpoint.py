"""The rank predictor's checkpoint format (CPU only): round trip, and every damaged form refused
with a ValueError (magic, header length, header, parameter count)."""
import json
import struct

import numpy as np
import pytest

pytest.importorskip("torch")
from paper_1707_05141_gb300 import MLP_PARAMS, rank_mlp  # noqa: E402


def test_roundtrip(tmp_path):
    p = rank_mlp.init_params(7)
    path = str(tmp_path / "w.bin")
    rank_mlp.save(path, p, {"tol": 1e-5, "note": "x"})
    q, hdr = rank_mlp.load(path)
    assert np.array_equal(p, q) and q.dtype == np.float32
    assert hdr["tol"] == 1e-5 and hdr["nparams"] == MLP_PARAMS and hdr["hidden"] == 64


def test_wrong_parameter_count_is_not_saved(tmp_path):
    with pytest.raises(ValueError):
        rank_mlp.save(str(tmp_path / "w.bin"), np.zeros(10, np.float32))


def _write(path, magic=rank_mlp.MAGIC, hdr=b'{"nparams": 5313}', hl=None, body=None):
    body = np.zeros(MLP_PARAMS, "<f4").tobytes() if body is None else body
    with open(path, "wb") as f:
        f.write(magic + struct.pack("<I", len(hdr) if hl is None else hl) + hdr + body)


@pytest.mark.parametrize("case", ["magic", "short", "hlen", "json", "notdict", "count", "truncated"])
def test_damaged_checkpoints_are_refused(tmp_path, case):
    path = str(tmp_path / "w.bin")
    if case == "magic":
        _write(path, magic=b"XXXXXXXX")
    elif case == "short":
        with open(path, "wb") as f:
            f.write(rank_mlp.MAGIC + b"\x01")
    elif case == "hlen":
        _write(path, hl=1 << 30)
    elif case == "json":
        _write(path, hdr=b"{not json")
    elif case == "notdict":
        _write(path, hdr=json.dumps([1, 2]).encode())
    elif case == "count":
        _write(path, hdr=b'{"nparams": 12}')
    else:
        _write(path, body=np.zeros(MLP_PARAMS - 1, "<f4").tobytes())
    with pytest.raises(ValueError):
        rank_mlp.load(path)
