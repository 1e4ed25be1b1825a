"""The C-ABI library builds, loads and exports every function that include/*.h declares (CPU only).

Only host-side argument checks are called here: they return before any CUDA call.
"""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
DECL = re.compile(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b([a-z_][a-z0-9_]*)\s*\(", re.M)


def declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        text = re.sub(r"^\s*#[^\n]*", "", text, flags=re.M)
        for m in DECL.finditer(text):
            if m.group(1) not in ("if", "while", "for", "return", "sizeof"):
                names.append(m.group(1))
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    import paper_1707_05141_gb300 as bs
    path = bs.build()
    return ctypes.CDLL(path), bs


def test_header_declares_the_three_entry_points():
    names = declared_functions()
    for want in ("batched_qr", "batched_svd_jacobi", "bsvd_version"):
        assert want in names, names


def test_every_declared_symbol_is_exported(lib):
    L, _ = lib
    for name in declared_functions():
        assert hasattr(L, name), name


def test_version_string(lib):
    _, bs = lib
    assert "sm_103a" in bs.version()


def test_host_argument_checks_without_gpu(lib):
    _, bs = lib
    L = bs.lib()
    z = None
    assert L.batched_qr(9, 1, 4, 4, z, z, z, z, z, z, z, z, z, z) == -1
    assert L.batched_qr(0, -3, 4, 4, z, z, z, z, z, z, z, z, z, z) == -2
    assert L.batched_qr(0, 1, 4, 8, z, z, z, z, z, z, z, z, z, z) == -4        # max_n > max_m
    assert L.batched_qr(0, 0, 4, 4, z, z, z, z, z, z, z, z, z, z) == 0         # empty batch: no-op
    assert L.batched_svd_jacobi(5, 1, 4, 4, z, z, z, z, z, z, z, z, z, 0.0, 0, 0, z, z, z) == -1
    assert L.batched_svd_jacobi(0, 1, 4, 4, z, z, z, z, z, z, z, z, z, 0.0, 0, 99, z, z, z) == -16
    assert L.batched_svd_jacobi(0, 1, 4, 4, z, z, z, z, z, z, z, z, z, 0.0, 0, 0, z, z, z) == -5
    assert L.batched_svd_jacobi(1, 0, 4, 4, z, z, z, z, z, z, z, z, z, 0.0, 0, 0, z, z, z) == 0
    assert L.batched_svd_jacobi(0, 1, 4, 4, z, z, z, z, z, z, z, z, z, 0.0, 0, 2 | (1 << 8), z, z, z) == -16
    # block Jacobi: unknown `method` bits are refused before anything is launched (the pointers
    # are never dereferenced: the checks return first)
    p = 64
    for bad in (1 << 21, 1 << 20, 2, -(1 << 30)):
        assert L.batched_svd_block_jacobi(0, 1, 64, 64, p, p, p, p, p, p, p, p, p, 0.0, 0, 32, bad, p, z, p, 1 << 20,
                                          z) == -17, bad


def test_variant_counts_and_tuning_table(lib):
    _, bs = lib
    L = bs.lib()
    assert L.bsvd_jacobi_variants(0, 64, 64, bs.TIER_REGISTER) >= 2
    assert L.bsvd_jacobi_variants(1, 32, 32, bs.TIER_REGISTER) >= 1
    assert L.bsvd_jacobi_variants(0, 256, 256, bs.TIER_REGISTER) == 0
    assert L.bsvd_jacobi_variants(0, 256, 128, bs.TIER_SHARED) == 1
    assert L.bsvd_jacobi_variants(1, 256, 128, bs.TIER_SHARED) == 0
    assert L.bsvd_jacobi_variants(3, 8, 8, bs.TIER_SHARED) == -1
    assert L.bsvd_set_jacobi_choice(0, 64, 64, bs.TIER_REGISTER | (2 << 8)) == 0
    assert L.bsvd_set_jacobi_choice(0, 64, 64, bs.TIER_AUTO) == 0
    assert L.bsvd_set_jacobi_choice(0, 512, 64, bs.TIER_AUTO) == -2
    assert L.bsvd_set_jacobi_choice(0, 64, 64, 7) == -4


def test_variant_descriptions(lib):
    """The k-th fitting register variant's shape; QR preconditioning only for square bounds, and
    listed after every unpreconditioned variant (so variant 0 -- the first -- never has it); the
    FP64-rotation-parameter variants (FP32 only) come after all the others."""
    _, bs = lib
    L = bs.lib()
    for code, (m, n) in [(0, (64, 64)), (0, (32, 32)), (1, (32, 32)), (1, (64, 64)), (0, (128, 48)), (1, (64, 60))]:
        nv = L.bsvd_jacobi_variants(code, m, n, bs.TIER_REGISTER)
        descs = [bs.jacobi_variant_desc(code, m, n, k) for k in range(1, nv + 1)]
        car = [d["carried_norms"] for d in descs]
        assert car == sorted(car), (code, m, n, car)             # carried-norm variants last
        p64 = [d["fp64_params"] for d in descs if not d["carried_norms"]]
        assert p64 == sorted(p64) and (code == 0 or not any(p64)), (code, m, n, p64)
        pre = [d["qr_precond"] for d in descs if not d["fp64_params"] and not d["carried_norms"]]
        assert pre == sorted(pre), (code, m, n, pre)             # preconditioned ones last
        assert any(pre) == (m == n), (code, m, n, pre)
        for d in descs:                                          # every one fits the bounds
            assert min(m, n) <= 2 * d["slots"] and max(m, n) <= d["parts"] * d["rows_a"]
            assert min(m, n) <= d["parts"] * d["rows_v"]
        with pytest.raises(bs.BsvdError):
            bs.jacobi_variant_desc(code, m, n, nv + 1)
    import ctypes
    d = (ctypes.c_int * 9)()
    assert L.bsvd_jacobi_variant_desc(2, 64, 64, 1, d) == -1
    assert L.bsvd_jacobi_variant_desc(0, -1, 64, 1, d) == -2
    assert L.bsvd_jacobi_variant_desc(0, 64, 64, 0, d) == -4
    assert L.bsvd_jacobi_variant_desc(0, 64, 64, 1, None) == -5


def test_blocked_qr_host_checks(lib):
    """The blocked QR's workspace query, height limit and argument checks (host only)."""
    _, bs = lib
    L = bs.lib()
    z = None
    assert L.batched_qr_blocked_max_rows(0) == 11976 and L.batched_qr_blocked_max_rows(1) == 5576
    assert L.batched_qr_blocked_max_rows(3) == -1
    w1 = L.batched_qr_blocked_workspace(0, 10, 1000, 200)
    w2 = L.batched_qr_blocked_workspace(0, 20, 1000, 200)
    assert 10 * 1000 * 200 * 4 <= w1 < w2 and L.batched_qr_blocked_workspace(1, 10, 1000, 200) > w1
    assert L.batched_qr_blocked_workspace(0, 10, 100, 200) == 0               # max_n > max_m
    args = (z, z, z, z, z, z, z, z, z, z, 0, z)
    assert L.batched_qr_blocked(7, 1, 64, 64, *args) == -1
    assert L.batched_qr_blocked(0, -1, 64, 64, *args) == -2
    assert L.batched_qr_blocked(0, 1, 64, 65, *args) == -4
    assert L.batched_qr_blocked(0, 0, 64, 64, *args) == 0                    # empty batch: no-op
    assert L.batched_qr_blocked(0, 1, 64, 64, *args) == -5
    p = ctypes.c_void_p(8)                                                     # never dereferenced
    assert L.batched_qr_blocked(0, 1, 64, 64, p, p, p, p, z, z, z, z, p, z, 0, z) == -14   # no workspace
    assert L.batched_qr_blocked(0, 1, 12000, 64, p, p, p, p, z, z, z, z, p, p, 0, z) == bs.ERR_UNSUPPORTED
