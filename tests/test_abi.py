"""CPU checks of the C ABI: the library loads, exports every entry point that
include/biharm.h declares, and its host-side FP64 setup (Eq. (matrix1d),
Sec. 4.1) agrees with the oracle.  No CUDA device is used."""
import os
import re

import numpy as np
import pytest
import scipy.linalg as sla

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    import paper_2412_05082_gb300 as bh
    if not os.path.exists(bh.LIB_PATH):
        from paper_2412_05082_gb300 import build
        build.build()
    return bh


def declared_functions():
    text = open(os.path.join(ROOT, "include", "biharm.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(bh_[A-Za-z0-9_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 15
    handle = lib.load()
    for name in names:
        assert hasattr(handle, name), name
    assert set(names) == set(lib.SIGNATURES), set(names) ^ set(lib.SIGNATURES)


def test_params_struct_matches_header(lib):
    import ctypes
    text = open(os.path.join(ROOT, "include", "biharm.h")).read()
    body = re.search(r"typedef struct \{(.*?)\} bh_params;", text, re.S).group(1)
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = re.findall(r"\b(int|double)\s+(\w+);", body)
    assert [f for _, f in fields] == [f for f, _ in lib.Params._fields_]
    for (ty, _), (_, ct) in zip(fields, lib.Params._fields_):
        assert ct == (ctypes.c_int if ty == "int" else ctypes.c_double)


def test_default_params_and_validation(lib):
    p = lib.default_params(2, 3, 4)
    assert (p.dim, p.degree, p.level, p.smoother, p.local_solver) == (2, 3, 4, lib.MVS_COLORED, lib.FDM)
    assert p.pre_steps == 1 and p.post_steps == 1 and p.gmres_restart == 50
    assert p.gmres_side == lib.RIGHT
    assert p.krylov == lib.GMRES
    for bad in [(1, 3, 4), (2, 1, 4), (2, 8, 4), (3, 2, 0)]:
        with pytest.raises(lib.BiharmError):
            lib.default_params(*bad)


@pytest.mark.parametrize("overrides,msg", [
    ({"krylov": 2}, "Krylov"),
    ({"krylov": 1}, "symmetric"),                       # CG with the multiplicative smoother
    ({"precision": 1, "gmres_side": 1}, "flexible"),   # FP32 V-cycle with left GMRES
    ({"precision": 2, "gmres_side": 1}, "flexible"),   # FP32 V-cycle, FP64 defects, left GMRES
    ({"precision": 3, "gmres_side": 1}, "flexible"),   # compensated FP32 defects, left GMRES
    ({"precision": 4}, "precision"),
])
def test_create_rejects_inconsistent_options_before_touching_a_device(lib, overrides, msg):
    # option checks run before device discovery, so they hold on a CPU-only host
    import types
    with pytest.raises(lib.BiharmError) as e:
        lib.Context(lib.default_params(2, 2, 3, **overrides), types.SimpleNamespace(cuda_stream=0))
    assert e.value.status == lib.BH_EINVAL and msg in str(e.value)


@pytest.mark.parametrize("k", range(2, 8))
def test_host_1d_matrices_match_oracle(lib, k):
    from oracle import kron
    cells = 4
    M, L, B = kron.global_1d(k, cells, full=True)   # h = 1/cells
    h = 1.0 / cells
    Ml, Ll, Bl = (lib.setup_1d(k, 0.0, cells, w) for w in range(3))  # h = 1
    assert np.allclose(Ml * h, M, rtol=0, atol=1e-14 * np.abs(M).max())
    assert np.allclose(Ll / h, L, rtol=0, atol=1e-13 * np.abs(L).max())
    assert np.allclose(Bl / h ** 3, B, rtol=0, atol=1e-12 * np.abs(B).max())


@pytest.mark.parametrize("k", range(2, 8))
def test_host_fdm_matches_oracle_patch_matrices(lib, k):
    from oracle import kron
    m = 2 * k - 1
    M5, _, B5 = kron.global_1d(k, 5, full=True)
    M2, _, B2 = kron.global_1d(k, 2, full=True)
    # patch type -> (matrices, first node) on lines of 5 (or 2) cells of size 1/5 (1/2)
    cases = {0: (M5, B5, k + 1, 5), 1: (M5, B5, 1, 5), 2: (M5, B5, 3 * k + 1, 5), 3: (M2, B2, 1, 2)}
    for t, (Mf, Bf, first, cells) in cases.items():
        s = slice(first, first + m)
        h = 1.0 / cells
        Mv, Bv = Mf[s, s] / h, Bf[s, s] * h ** 3          # back to cells of size 1
        S, lam = lib.setup_fdm(k, 0.0, t)
        assert np.allclose(S.T @ Mv @ S, np.eye(m), atol=1e-11)
        assert np.allclose(S.T @ Bv @ S, np.diag(lam), atol=1e-9 * lam.max())
        ref = sla.eigh(Bv, Mv, eigvals_only=True)
        assert np.allclose(np.sort(lam), ref, rtol=1e-11)
        if t == 0:
            # interior patches: the folded FDM needs even eigenvectors in
            # columns 0..k-1 and odd ones in k..m-1, exactly
            assert np.array_equal(S[::-1, :k], S[:, :k])
            assert np.array_equal(S[::-1, k:], -S[:, k:])


def test_no_cpu_fallback(lib):
    """Without a CUDA device the library refuses to build a hierarchy
    (BH_ECUDA), and the binding refuses host tensors: nothing runs on the CPU
    in their place."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")

    class NoStream:
        cuda_stream = 0

    with pytest.raises(lib.BiharmError) as e:
        lib.Context(lib.default_params(2, 2, 3), NoStream())
    assert e.value.status == lib.BH_ECUDA
    with pytest.raises(TypeError):
        lib._dev(torch.zeros(3, dtype=torch.float64), 3, "x")


def test_fault_injection_switch_on_the_host(lib):
    """bh_fault_inject_alloc is host-only: it takes non-negative counts and can
    be switched off again without a device."""
    lib.fault_inject_alloc(3, 1)
    lib.fault_inject_alloc(0, 0)
    with pytest.raises(lib.BiharmError) as e:
        lib.fault_inject_alloc(-1, 1)
    assert e.value.status == lib.BH_EINVAL
