"""Allocation failures on a B300, driven by the REX_FAIL_DEVICE_ALLOC hook: every
library-owned device allocation path returns REX_ENOMEM, releases what it had
allocated, and leaves the handle (or the library) usable once allocations succeed
again.  No device fault is involved: the hook fails the allocation before cudaMalloc."""
import numpy as np
import pytest

from rexlib import ensure_built
from paper_2510_05100_b300 import phase_space as ps

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ORIG = dict(mt=173.0, wt=0.0, alphas=0.118)


@pytest.fixture(scope="module")
def rex():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return ensure_built()


def free_bytes():
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


def test_handle_creation_fails_at_every_allocation_without_leaking(rex, monkeypatch):
    """x-section handles make 3 device allocations, surrogates 8, multi handles 1:
    failing at each one in turn, 20 times over, leaves the device's free memory where
    it was (a leak of the earlier buffers would show as 20 x their size)."""
    torch.cuda.init()
    rex.XSec(4).close()
    rex.Surrogate(1).close()
    rex.Multi(rex.MIXED).close()
    before = free_bytes()
    for kind, nalloc in (("xsec", 3), ("surrogate", 8), ("multi", 1)):
        for n in range(1, nalloc + 1):
            for rep in range(20):
                # "n" and "+n" read as the same n; a changed value restarts the count
                monkeypatch.setenv("REX_FAIL_DEVICE_ALLOC", f"{n}" if rep % 2 else f"+{n}")
                with pytest.raises(rex.RexError) as err:
                    if kind == "xsec":
                        rex.XSec(1 << 16)
                    elif kind == "surrogate":
                        rex.Surrogate(3)
                    else:
                        rex.Multi(rex.MIXED)
                assert err.value.code == rex.REX_ENOMEM
                assert "out of memory" in str(err.value)
        monkeypatch.delenv("REX_FAIL_DEVICE_ALLOC")
    after = free_bytes()
    assert before - after < 64 << 20, (before, after)
    rex.XSec(4).close()       # allocations succeed again
    rex.Surrogate(1).close()
    rex.Multi(rex.MIXED).close()


def test_workspace_failures_leave_the_handles_usable(rex, monkeypatch):
    """Buffers grown during a call (host-buffer staging of rex_reweight_host, the
    x-section partials, the surrogate's inference buffers): the call fails with
    REX_ENOMEM and the same handle works on the next call."""
    n = 4096
    pts = ps.grid_gg_ttxg()[:4]
    mom = ps.make_events("gg_ttxg", n, 5)
    w = np.ones(n)

    out = np.zeros((n, len(pts)))
    for fail_at in ("1", "2", "3"):      # a new handle's momenta, input weights, output weights
        proc = rex.Process("gg_ttxg")
        proc.set_params(ORIG)
        monkeypatch.setenv("REX_FAIL_DEVICE_ALLOC", fail_at)
        with pytest.raises(rex.RexError) as err:
            proc.reweight_host(mom, w, pts, out)
        assert err.value.code == rex.REX_ENOMEM
        monkeypatch.delenv("REX_FAIL_DEVICE_ALLOC")
        proc.reweight_host(mom, w, pts, out)     # the same handle, allocations succeeding
    ref = proc.reweight(torch.from_numpy(mom).cuda(), torch.from_numpy(w).cuda(), pts).cpu().numpy()
    assert np.array_equal(out, ref)

    xs = rex.XSec(len(pts))
    dw, dout = torch.from_numpy(w).cuda(), torch.from_numpy(ref).cuda()
    for fail_at in ("1", "2"):           # partial moments, partial scalars
        monkeypatch.setenv("REX_FAIL_DEVICE_ALLOC", fail_at)
        with pytest.raises(rex.RexError) as err:
            xs.accumulate(dw, dout)
        assert err.value.code == rex.REX_ENOMEM
    monkeypatch.delenv("REX_FAIL_DEVICE_ALLOC")
    xs.accumulate(dw, dout)
    st = xs.get_state()
    assert st[0] == n and st[5 * len(pts)] == n and np.all(np.isfinite(st))   # counted once, after the failures
    xs.close()

    sur = rex.Surrogate(2)
    sur.set_exact_alphas(0.118, 3)
    dm = torch.from_numpy(mom).cuda()
    pred = torch.empty((n, len(pts)), dtype=torch.float32, device="cuda")
    monkeypatch.setenv("REX_FAIL_DEVICE_ALLOC", "1")
    with pytest.raises(rex.RexError) as err:
        sur.reweight(dm, None, pts, pred=pred)
    assert err.value.code == rex.REX_ENOMEM
    monkeypatch.delenv("REX_FAIL_DEVICE_ALLOC")
    sur.reweight(dm, None, pts, pred=pred)
    assert torch.isfinite(pred).all()
    sur.close()
    proc.close()
