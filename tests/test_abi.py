"""CPU checks of the C ABI: the library builds, loads, and exports every declared symbol;
host-side argument checks answer without touching a GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_1705_01893_gb300 import binding, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "mm.h")).read()
    decl = r"^(?:mm_status|void|const char\*)\s+(mm_\w+)\s*\("
    return sorted(set(re.findall(decl, text, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return binding.load()


def test_header_matches_binding():
    assert set(declared_symbols()) == set(binding.SIGNATURES)


def test_every_declared_symbol_exported(lib):
    for name in declared_symbols():
        assert hasattr(lib, name), name


def test_workspace_size_host_checks(lib):
    n = ctypes.c_size_t()
    off = np.array([0, 4096, 8192], dtype=np.int64)
    offp = off.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
    assert lib.mm_plan_workspace_size(2, offp, 100, 3, 0, ctypes.byref(n)) == binding.MM_OK
    assert n.value > 0 and n.value % 256 == 0
    # T-only needs less than IQU
    m = ctypes.c_size_t()
    assert lib.mm_plan_workspace_size(2, offp, 100, 1, 0, ctypes.byref(m)) == binding.MM_OK
    assert m.value < n.value
    # bad ncomp, bad weight dtype, bad n_pix
    assert lib.mm_plan_workspace_size(2, offp, 100, 2, 0, ctypes.byref(n)) == binding.MM_ERR_ARG
    assert lib.mm_plan_workspace_size(2, offp, 100, 3, 7, ctypes.byref(n)) == binding.MM_ERR_ARG
    assert lib.mm_plan_workspace_size(2, offp, 0, 3, 0, ctypes.byref(n)) == binding.MM_ERR_ARG
    assert b"n_pix" in lib.mm_last_error()
    # unsupported lengths: a prime factor other than 2, 3, 5; too long; too short; empty
    for bad in ([0, 4095], [0, 7 * 64], [0, 1 << 25], [0, 3], [0, 0]):
        o = np.array(bad, dtype=np.int64)
        r = lib.mm_plan_workspace_size(1, o.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), 10, 1,
                                       0, ctypes.byref(n))
        assert r in (binding.MM_ERR_UNSUPPORTED, binding.MM_ERR_ARG), bad
        assert r == (binding.MM_ERR_ARG if bad[1] == 0 else binding.MM_ERR_UNSUPPORTED), bad
    # 2-3-5-smooth lengths (even, odd, small powers of two) and unaligned starts are planned
    for good in ([0, 3000], [0, 3125], [0, 256], [0, 6000, 10096], [2, 4098]):
        o = np.array(good, dtype=np.int64)
        r = lib.mm_plan_workspace_size(len(good) - 1, o.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                       10, 3, 0, ctypes.byref(n))
        assert r == binding.MM_OK, good


def test_null_arguments_rejected_on_host(lib):
    h = ctypes.c_void_p()
    off = np.array([0, 1024], dtype=np.int64)
    offp = off.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
    # pix NULL
    r = lib.mm_plan_pointing(ctypes.byref(h), 1, offp, None, None, None, 0, 16, 1, 1e-3, None, 0, None)
    assert r == binding.MM_ERR_ARG
    assert lib.mm_messenger_iterate(None, None, 0, 0, None, None, None) == binding.MM_ERR_ARG
    lam = (ctypes.c_double * 1)(1.0)
    assert lib.mm_messenger_forward_ckpt(None, lam, 1, None, 1, None, None) == binding.MM_ERR_ARG
    assert lib.mm_messenger_adjoint_ckpt(None, lam, 1, None, None, None, None, 1, None, 0,
                                         None) == binding.MM_ERR_ARG
    lib.mm_plan_destroy(None)


def test_workspace_too_small_is_nomem(lib):
    h = ctypes.c_void_p()
    off = np.array([0, 1024], dtype=np.int64)
    offp = off.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
    fake = ctypes.c_void_p(0x1000)  # never dereferenced: the size check comes first
    r = lib.mm_plan_pointing(ctypes.byref(h), 1, offp, fake, None, None, 0, 16, 1, 1e-3,
                             ctypes.c_void_p(0x100000), 16, None)
    assert r == binding.MM_ERR_NOMEM
    assert b"workspace too small" in lib.mm_last_error()


def test_bounded_wait_check_rejects_bad_limits(lib):
    e = ctypes.c_int()
    assert lib.mm_check_bounded_wait(0, 0, ctypes.byref(e), None) == binding.MM_ERR_ARG
    assert lib.mm_check_bounded_wait((1 << 22) + 1, 0, ctypes.byref(e), None) == binding.MM_ERR_ARG
    assert lib.mm_check_bounded_wait(10, 0, None, None) == binding.MM_ERR_ARG


@pytest.mark.parametrize("m1,cb", [(512, 16), (1024, 8), (2048, 4)])
@pytest.mark.parametrize("count", list(range(1, 13)) + [16, 31])
def test_fused_item_list_order(lib, count, m1, cb):
    """The fused kernel's work list (host code, no GPU) for the three fused shapes (columns
    of 512, 1024 and 2048 points in tiles of 16, 8 and 4 columns, rows of 4096): each item
    exactly once, and every row job after all column tiles of its chunk, every inverse tile
    after all row jobs of its chunk -- the order that keeps the kernel free of deadlock."""
    items = binding.fused_item_list(m1, 4096, count)
    nA, nB = 4096 // cb, m1 // 2 + 1
    assert items.shape == (count * (2 * nA + nB), 3)
    assert len({tuple(r) for r in items}) == len(items)
    doneA = np.zeros(count, dtype=int)
    doneB = np.zeros(count, dtype=int)
    for kind, c, i in items:
        assert 0 <= c < count
        if kind == 0:
            assert 0 <= i < nA
            doneA[c] += 1
        elif kind == 1:
            assert 0 <= i < nB and doneA[c] == nA
            doneB[c] += 1
        else:
            assert kind == 2 and 0 <= i < nA and doneB[c] == nB
    assert (doneA == nA).all() and (doneB == nB).all()


def test_fused_item_list_rejects_bad_shapes(lib):
    n = ctypes.c_int()
    assert lib.mm_fused_item_list(512, 4096, 0, None, 0, ctypes.byref(n)) == binding.MM_ERR_ARG
    assert lib.mm_fused_item_list(500, 4096, 1, None, 0, ctypes.byref(n)) == binding.MM_ERR_ARG
    assert lib.mm_fused_item_list(512, 4008, 1, None, 0, ctypes.byref(n)) == binding.MM_ERR_ARG


def test_product_package_never_imports_the_oracle():
    """The CUDA path and the oracle share no code: nothing in the package imports oracle/."""
    pkg = os.path.join(ROOT, "paper_1705_01893_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(from|import)\s+oracle\b", text, flags=re.M), f
    assert "oracle" not in open(os.path.join(ROOT, "include", "mm.h")).read().lower()


def test_missing_library_raises_instead_of_falling_back(tmp_path):
    """No CPU fallback: loading a library that is not there is an error."""
    saved = binding._lib
    binding._lib = None
    try:
        with pytest.raises(RuntimeError):
            binding.load(str(tmp_path / "libmm.so"))
    finally:
        binding._lib = saved


def test_noalloc_binding_checks_arguments_before_any_call():
    """binned_map_noalloc checks types and sizes on the host before it passes a pointer (the
    kernels trust the sizes they are given); wrong arguments raise without a launch."""
    torch = pytest.importorskip("torch")
    n, npix = 64, 16
    pix = torch.zeros(n, dtype=torch.int32)
    tod = torch.zeros(n, dtype=torch.float32)
    c32, s32 = torch.zeros(n), torch.zeros(n)
    out = torch.zeros(npix, 3, dtype=torch.float64)
    with pytest.raises(ValueError):      # map_out too small for n_pix x ncomp
        binding.binned_map_noalloc(pix, c32, s32, tod, npix, 3, out[:npix - 1])
    with pytest.raises(TypeError):       # pixel indices not int32
        binding.binned_map_noalloc(pix.long(), c32, s32, tod, npix, 3, out)
    with pytest.raises(ValueError):      # tod shorter than pix
        binding.binned_map_noalloc(pix, c32, s32, tod[:-1], npix, 3, out)
    with pytest.raises(TypeError):       # weights of two precisions
        binding.binned_map_noalloc(pix, c32, s32.half(), tod, npix, 3, out)
    with pytest.raises(ValueError):      # weights shorter than pix
        binding.binned_map_noalloc(pix, c32[:-1], s32[:-1], tod, npix, 3, out)
    with pytest.raises(ValueError):      # weights given for a T-only map
        binding.binned_map_noalloc(pix, c32, s32, tod, npix, 1, out)
    with pytest.raises(TypeError):       # weights neither float32 nor float16
        binding.binned_map_noalloc(pix, c32.double(), s32.double(), tod, npix, 3, out)
    with pytest.raises(ValueError):      # map_out not float64
        binding.binned_map_noalloc(pix, c32, s32, tod, npix, 3, out.float())
    with pytest.raises(ValueError):      # correct arguments, but host tensors
        binding.binned_map_noalloc(pix, c32, s32, tod, npix, 3, out)


def test_noalloc_rejects_bad_rcond_on_the_host(lib):
    """rcond_min outside [0, 1] or NaN is an argument error, as for mm_plan_pointing (checked
    before any device work: the pointers below are never dereferenced)."""
    dummy = ctypes.c_void_p(16)
    for bad in (float("nan"), -0.5, 1.5):
        st = lib.mm_binned_map_noalloc(dummy, None, None, 0, dummy, 0, 16, 1, bad, dummy, None)
        assert st == binding.MM_ERR_ARG
        assert b"rcond_min" in lib.mm_last_error()


def test_wait_policy_host_checks(lib):
    """The wait policy is checked on the host: a NULL plan or a limit outside [1, 2^22] is an
    argument error."""
    assert lib.mm_plan_set_wait_policy(None, 1, 0) == binding.MM_ERR_ARG


def test_degenerate_plans_rejected_on_host(lib):
    """No chunk, a negative chunk count, offsets that decrease (an empty or negative chunk)
    and a NULL offsets array are argument errors, answered before any device work."""
    n = ctypes.c_size_t()

    def ws(off, nc):
        o = np.array(off, dtype=np.int64)
        return lib.mm_plan_workspace_size(nc, o.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                          10, 1, 0, ctypes.byref(n))
    assert ws([0], 0) == binding.MM_ERR_ARG and b"n_chunks" in lib.mm_last_error()
    assert ws([0, 4096], -1) == binding.MM_ERR_ARG
    assert ws([0, 4096, 2048], 2) == binding.MM_ERR_ARG and b"empty" in lib.mm_last_error()
    assert ws([0, 4096, 4096], 2) == binding.MM_ERR_ARG
    assert lib.mm_plan_workspace_size(1, None, 10, 1, 0, ctypes.byref(n)) == binding.MM_ERR_ARG
    # a plan may start at a non-zero offset (samples before it belong to no chunk)
    assert ws([5, 5 + 4096], 1) == binding.MM_OK
