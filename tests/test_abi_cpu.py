"""C ABI checks that need no GPU: the library loads, exports every symbol the
header declares, and host-side validation returns the documented codes
(no call here reaches the CUDA runtime)."""
import ctypes

import numpy as np
import pytest

from rexlib import declared_symbols, ensure_built


@pytest.fixture(scope="module")
def rex():
    return ensure_built()


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for s in ("rex_init_process", "rex_set_params", "rex_reweight", "rex_me2", "rex_free_process",
              "rex_last_error"):
        assert s in syms


def test_library_exports_every_declared_symbol(rex):
    lib = rex.load()
    for s in declared_symbols():
        assert hasattr(lib, s), s
    assert set(rex.EXPORTS) == set(declared_symbols())
    assert "sm_103a" in rex.version()


def test_tooling_library_exports_its_header():
    """The measurement and test probes live in their own library, outside the reweighting ABI."""
    from rexlib import TOOLING_HEADER
    rex = ensure_built()
    lib = rex.load_tooling()
    syms = declared_symbols(TOOLING_HEADER)
    assert set(syms) == set(rex.TOOLING_EXPORTS)
    for s in syms:
        assert hasattr(lib, s), s
        assert s not in declared_symbols()


def test_init_errors(rex):
    lib = rex.load()
    h = ctypes.c_void_p()
    assert lib.rex_init_process(b"no_such_process", 0, ctypes.byref(h)) == rex.REX_EINVAL
    assert b"unknown process" in lib.rex_last_error()
    assert lib.rex_init_process(b"gg_ttxg", 7, ctypes.byref(h)) == rex.REX_EINVAL
    assert lib.rex_init_process(None, 0, ctypes.byref(h)) == rex.REX_EINVAL
    assert lib.rex_init_process(b"gg_ttxg", 0, None) == rex.REX_EINVAL
    assert lib.rex_init_process(b"ee_mumu", rex.MIXED, ctypes.byref(h)) == rex.REX_EUNSUPPORTED
    for name in (b"gg_ttxgg", b"qq_ttx", b"ee_mumu"):   # double-float: g g -> t t~ (g), q q~ -> t t~ g
        assert lib.rex_init_process(name, rex.DF64, ctypes.byref(h)) == rex.REX_EUNSUPPORTED
    for name in ("gg_ttx", "gg_ttxg", "qq_ttxg", "qg_ttxq"):
        p = rex.Process(name, rex.DF64)
        assert p.num_variants == 1 and p.variant == 0
        p.close()


@pytest.mark.parametrize("name,npart", [("ee_mumu", 4), ("gg_ttx", 4), ("gg_ttxg", 5), ("gg_ttxgg", 6), ("qq_ttx", 4), ("qq_ttxg", 5),
                                        ("qxq_ttxg", 5), ("qg_ttxq", 5), ("gq_ttxq", 5), ("qxg_ttxqx", 5),
                                        ("gqx_ttxqx", 5)])
def test_handle_lifecycle(rex, name, npart):
    p = rex.Process(name)
    assert p.npart == npart
    p.close()


def test_validation_before_any_device_work(rex):
    lib = rex.load()
    p = rex.Process("gg_ttxg")
    pts = (rex.Params * 1)(rex.params(dict(mt=171.0, alphas=0.118)))
    fake = ctypes.c_void_p(0x10000)     # never dereferenced: validation fails first
    # not initialised
    assert lib.rex_reweight(p._h, fake, fake, 10, pts, 1, fake, None) == rex.REX_ENOTINIT
    p.set_params(mt=173.0, alphas=0.118)
    assert lib.rex_reweight(p._h, fake, fake, -1, pts, 1, fake, None) == rex.REX_EINVAL
    assert lib.rex_reweight(p._h, fake, fake, 10, pts, -1, fake, None) == rex.REX_EINVAL
    assert lib.rex_reweight(p._h, None, fake, 10, pts, 1, fake, None) == rex.REX_EINVAL
    assert lib.rex_reweight(p._h, ctypes.c_void_p(0x10008), fake, 10, pts, 1, fake, None) == rex.REX_EINVAL
    assert b"aligned" in lib.rex_last_error()
    # empty work is a no-op that succeeds without touching the pointers
    assert lib.rex_reweight(p._h, None, None, 0, pts, 1, None, None) == rex.REX_OK
    assert lib.rex_reweight(p._h, None, None, 10, pts, 0, None, None) == rex.REX_OK
    # bad points
    bad = (rex.Params * 1)(rex.params(dict(mt=-1.0, alphas=0.118)))
    assert lib.rex_reweight(p._h, fake, fake, 10, bad, 1, fake, None) == rex.REX_EINVAL
    with pytest.raises(rex.RexError):
        p.set_params(mt=173.0, alphas=0.0)
    with pytest.raises(rex.RexError):
        p.set_flags(0x80)
    assert lib.rex_reweight(None, fake, fake, 10, pts, 1, fake, None) == rex.REX_EINVAL
    p.close()


def test_ee_point_validation(rex):
    p = rex.Process("ee_mumu")
    with pytest.raises(rex.RexError):
        p.set_params(mz=91.1876, wz=2.4952, sw2=1.5, alpha=1 / 132.507)
    p.set_params(mz=91.1876, wz=2.4952, sw2=0.2312, alpha=1 / 132.507)
    p.close()


def test_helicity_exclusive_validation_before_any_device_work(rex):
    lib = rex.load()
    pts = (rex.Params * 1)(rex.params(dict(mt=171.0, alphas=0.118)))
    fake = ctypes.c_void_p(0x10000)     # never dereferenced: validation fails first
    g = rex.Process("gg_ttxg")
    assert lib.rex_reweight_helicity(g._h, fake, fake, fake, 10, pts, 1, fake, None) == rex.REX_ENOTINIT
    g.set_params(mt=173.0, alphas=0.118)
    assert lib.rex_reweight_helicity(g._h, fake, None, fake, 10, pts, 1, fake, None) == rex.REX_EINVAL
    assert b"null helicity array" in lib.rex_last_error()
    q = rex.Process("qq_ttx")
    assert lib.rex_reweight_helicity(q._h, fake, fake, fake, 10, pts, 1, fake, None) == rex.REX_ENOTINIT
    q.set_params(mt=173.0, alphas=0.118)
    assert lib.rex_reweight_helicity(q._h, fake, None, fake, 10, pts, 1, fake, None) == rex.REX_EINVAL
    assert lib.rex_reweight_helicity(q._h, None, None, None, 0, pts, 1, None, None) == rex.REX_OK
    assert lib.rex_reweight_helicity(None, fake, fake, fake, 10, pts, 1, fake, None) == rex.REX_EINVAL
    x = rex.Process("qg_ttxq")       # a crossing evaluates the helicity sum only
    x.set_params(mt=173.0, alphas=0.118)
    assert lib.rex_reweight_helicity(x._h, fake, fake, fake, 10, pts, 1, fake, None) == rex.REX_EUNSUPPORTED
    assert b"direct channel only" in lib.rex_last_error()
    x.close()
    g.close()
    q.close()


def test_flop_counter_builds_and_counts_every_process():
    """The counting-scalar instantiation of the amplitude code (roofline flop counts)
    compiles against the current device routines and covers every QCD process."""
    from paper_2510_05100_b300 import flops
    counts = flops.counts()
    for proc in ("gg_ttx", "gg_ttxg", "gg_ttxgg", "qq_ttx", "qq_ttxg"):
        assert flops.per_event(proc, 5)["amp"] > 0, proc
    assert set(counts) >= {"gg_ttx", "gg_ttxg", "gg_ttxgg", "qq_ttx", "qq_ttxg"}


def test_injected_device_allocation_failure_is_reported(rex, monkeypatch):
    """The allocation-failure hook (REX_FAIL_DEVICE_ALLOC): the first library-owned
    device allocation of a handle fails as out of memory before any device is touched,
    and the call returns REX_ENOMEM with the cause in its message."""
    lib = rex.load()
    monkeypatch.setenv("REX_FAIL_DEVICE_ALLOC", "1")
    h = ctypes.c_void_p()
    assert lib.rex_xsec_create(4, ctypes.byref(h)) == rex.REX_ENOMEM
    assert not h.value
    assert b"out of memory" in lib.rex_xsec_last_error()
    assert lib.rex_surrogate_create(1, ctypes.byref(h)) == rex.REX_ENOMEM
    assert not h.value
    assert b"out of memory" in lib.rex_surrogate_last_error()


def test_tile_cost_calls_validate_their_handles(rex):
    lib = rex.load()
    p = rex.Process("gg_ttxg")
    us = ctypes.c_double(-1.0)
    assert lib.rex_multi_get_tile_cost(None, p._h, ctypes.byref(us)) == rex.REX_EINVAL
    assert lib.rex_multi_set_tile_cost(None, p._h, 1.0) == rex.REX_EINVAL
    assert us.value == -1.0
    p.close()
