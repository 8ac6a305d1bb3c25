"""Host-side checks of the C-ABI library that need no GPU: it loads, it exports
every entry point include/frag.h declares, and its plan logic (validation,
fragment sizes) agrees with the oracle's size arithmetic."""
import ctypes
import os
import re

import pytest

import oracle
import paper_1803_04880_b300 as fr

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    fr.build()
    return fr.lib()


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "frag.h")).read()
    return sorted(set(re.findall(r"^\s*(?:frag_status|int)\s+(frag_\w+)\s*\(", src, re.M)))


def test_exports_every_declared_symbol(L):
    names = declared_symbols()
    assert len(names) >= 20
    assert sorted(fr.EXPORTS) == names or set(fr.EXPORTS) <= set(names)
    for name in names:
        assert hasattr(L, name), name


def test_abi_version(L):
    assert L.frag_abi_version() == 2


@pytest.mark.parametrize("w,l,status", [(0, 1, fr.FRAG_EINVAL), (12, 3, fr.FRAG_EINVAL),
                                        (64, 0, fr.FRAG_EINVAL), (1024, 9, fr.FRAG_EINVAL),
                                        (64, 7, fr.FRAG_EINVAL), (384, 8, fr.FRAG_EINVAL)])
def test_plan_validation(L, w, l, status):
    h = ctypes.c_void_p()
    assert L.frag_plan_create(ctypes.byref(h), w, l, 0) == status
    assert "width" in fr.last_error() or "levels" in fr.last_error()


@pytest.mark.parametrize("w,l", [(64, 6), (128, 7), (256, 8), (8192, 8)])
def test_plans_of_six_to_eight_levels(L, w, l):
    """Every level count 1..8 makes a plan; its sizes are the oracle's."""
    p = fr.Plan(w, l)
    for n in (1, w * 3 + 1, w * (1 << l) * 5 - 7):
        assert p.sizes(n) == oracle.sizes(n, w, l)


def test_unknown_filter(L):
    h = ctypes.c_void_p()
    assert L.frag_plan_create(ctypes.byref(h), 64, 2, 7) == fr.FRAG_EUNSUPPORTED


@pytest.mark.parametrize("n,w,l", [(0, 64, 2), (1, 2, 1), (1000, 64, 3), (65536, 256, 1),
                                   (3 * 4096 * 4096 // 3, 4096, 3), (77777, 256, 5),
                                   (268435456, 8192, 4)])
def test_sizes_match_oracle(L, n, w, l):
    p = fr.Plan(w, l)
    H, pb, ub = p.sizes(n)
    assert (H, pb, ub) == oracle.sizes(n, w, l)


def test_null_arguments_are_rejected(L):
    p = fr.Plan(64, 2)
    assert L.frag_protect(p.handle, None, 0, None, 16, None, None, None) == fr.FRAG_EINVAL
    assert L.frag_recover(None, None, 0, None, None, 16, None, None) == fr.FRAG_EINVAL
    assert L.frag_get_error(None, 0) == fr.FRAG_EINVAL
    assert L.frag_batch_info(None, None, None) == fr.FRAG_EINVAL
    assert L.frag_check_wait_timeout(0, None) == fr.FRAG_EINVAL
    assert L.frag_check_box_wait_timeout(0, None) == fr.FRAG_EINVAL
    assert L.frag_batch_set_timing(None, 1) == fr.FRAG_EINVAL
    assert L.frag_batch_launch_times(None, None, None) == fr.FRAG_EINVAL
    assert L.frag_plan_set_path(None, 0) == fr.FRAG_EINVAL
    assert L.frag_plan_get_path(p.handle, None) == fr.FRAG_EINVAL
    # full-buffer AES-CTR: a NULL key is refused before any device work
    assert L.frag_aes128_ctr(None, 0, None, None, 16, None) == fr.FRAG_EINVAL


def test_packed_validation(L):
    import oracle
    p = fr.Plan(64, 2)
    with pytest.raises(fr.FragError):
        p.set_packed(True)  # not in block mode
    p.set_block(8)
    p.set_packed(True)
    assert p.packed()
    with pytest.raises(fr.FragError):
        p.set_block(0)  # packed plans keep their 8 x 8 blocks
    for n in (1, 64 * 8, 64 * 24 - 5, 64 * 4096):
        H, a, b, c = oracle.packed_sizes(n, 64)
        assert p.sizes(n) == (H, a, b + c)
        assert p.fragment_sizes(n) == (a, b, c)
    p.set_packed(False)
    assert not p.packed()
    q = fr.Plan(64, 3)
    q.set_block(8)
    with pytest.raises(fr.FragError):
        q.set_packed(True)  # the thesis's storage is for two levels
    # unpacked plans: the first public fragment is level L's three bands
    for W, Lv, n in ((64, 2, 64 * 30), (256, 3, 256 * 100 + 7)):
        r = fr.Plan(W, Lv)
        H, pb, ub = r.sizes(n)
        assert r.fragment_sizes(n) == (pb, 3 * pb, ub - 3 * pb)
    assert L.frag_plan_fragment_sizes(q.handle, 16, None) == fr.FRAG_EINVAL
    assert L.frag_plan_get_packed(q.handle, None) == fr.FRAG_EINVAL


def test_protect_public_validation(L):
    p = fr.Plan(64, 2)
    assert not p.protect_public()
    with pytest.raises(fr.FragError):
        p.set_protect_public(True)  # the keyed hashes work on the packed records
    p.set_block(8)
    p.set_packed(True)
    p.set_protect_public(True)
    assert p.protect_public()
    with pytest.raises(fr.FragError):
        p.set_packed(False)  # clear the keyed protection first
    assert p.fragment_sizes(64 * 24) == oracle_sizes(64 * 24, 64)  # the packed sizes
    p.set_protect_public(False)
    p.set_packed(False)
    assert not p.protect_public() and not p.packed()
    assert L.frag_plan_get_protect_public(p.handle, None) == fr.FRAG_EINVAL
    assert L.frag_plan_set_protect_public(None, 1) == fr.FRAG_EINVAL


def oracle_sizes(n, W):
    import oracle
    _, a, b, c = oracle.packed_sizes(n, W)
    return a, b, c


def test_block_validation(L):
    p = fr.Plan(64, 2)
    assert p.block() == 0
    p.set_block(8)
    assert p.block() == 8
    assert p.sizes(65)[0] == 8  # whole blocks: 2 rows pad to 8
    p.set_block(0)
    assert p.sizes(65)[0] == 4
    with pytest.raises(fr.FragError):
        fr.Plan(12, 2).set_block(8)  # width not a multiple of the block
    with pytest.raises(fr.FragError):
        fr.Plan(64, 4).set_block(8)  # block below 2^L
    with pytest.raises(fr.FragError):
        fr.Plan(64, 2).set_block(16)  # only 8 x 8 blocks on the CUDA path
    assert L.frag_plan_get_block(p.handle, None) == fr.FRAG_EINVAL


def test_path_validation(L):
    p = fr.Plan(256, 3)
    assert p.path() == fr.Plan.PATH_AUTO
    p.set_path(fr.Plan.PATH_LEVELS)
    assert p.path() == fr.Plan.PATH_LEVELS
    with pytest.raises(fr.FragError):
        p.set_path(7)


def test_sha2_constants_header_is_current():
    """The library's SHA-2 constants header is what its generator derives."""
    import subprocess
    import sys
    gen = os.path.join(os.path.dirname(fr.__file__), "csrc", "gen_sha2_constants.py")
    assert subprocess.run([sys.executable, gen, "--check"]).returncode == 0
