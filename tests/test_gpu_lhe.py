"""From an LHE file to a reweighted LHE file (needs a B300): the front-end's
extraction feeds the FP64 kernels, the new weights are written back, and the
written file is read with the oracle's reader."""
import re

import numpy as np
import pytest

from rexlib import ensure_built
from oracle import lhe as olhe
from oracle import reweight as oracle_rw
from paper_2510_05100_b300 import lhe_synth
from paper_2510_05100_b300 import phase_space as ps

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ORIG = dict(mt=173.0, wt=0.0, alphas=0.118)
# the q q~ and g g channels of p p -> t t~ share their weight ids, as in one reweighting run
GRIDS = {"gg_ttx": ps.grid_gg_ttx(), "qq_ttx": ps.grid_gg_ttx(), "gg_ttxg": ps.grid_gg_ttxg()}


@pytest.fixture(scope="module")
def rex():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return ensure_built()


def wid(pt):
    return "mt%.2f_as%.4f" % (pt["mt"], pt["alphas"])


def test_file_to_reweighted_file(rex, tmp_path):
    src, dst = str(tmp_path / "in.lhe"), str(tmp_path / "out.lhe")
    info = lhe_synth.write_lhe(src, {"gg_ttxg": 3000, "gg_ttx": 2000, "qq_ttx": 700, "ee_mumu": 100}, seed=5)
    L = rex.Lhe(src)
    gpu = {}
    for proc, pts in GRIDS.items():
        pin, pout = lhe_synth.PROCESSES[proc]
        mom, w, idx = L.extract(pin, pout)
        assert mom.shape[0] == info[proc][0].shape[0]
        p = rex.Process(proc, 0)
        p.set_params(ORIG)
        out = p.reweight(torch.from_numpy(mom).cuda(), torch.from_numpy(w).cuda(), pts).cpu().numpy()
        ref = oracle_rw.reweight(proc, mom[:8], w[:8], ORIG, pts)
        assert np.max(np.abs(out[:8] / ref - 1)) < 1e-12
        for j, pt in enumerate(pts):
            L.set_weights(wid(pt), idx, out[:, j])
        gpu[proc] = (idx, out)
    L.write(dst)
    L.close()
    doc = olhe.read(dst)
    text = doc["text"]
    ids = [wid(pt) for pts in GRIDS.values() for pt in pts]
    for i in ids:
        assert "<weight id='%s'>%s</weight>" % (i, i) in text
    pat = re.compile(r"<wgt id='([^']+)'> ([^ ]+) </wgt>")
    for proc, (idx, out) in gpu.items():
        pts = GRIDS[proc]
        for n in (0, 1, len(idx) // 2, len(idx) - 1):
            ev = doc["events"][idx[n]]
            found = dict(pat.findall(text[ev["start"]:ev["end"]]))
            for j, pt in enumerate(pts):
                assert float(found[wid(pt)]) == pytest.approx(out[n, j], rel=1e-10)   # %+.10e in the file
    # events of other processes get no weight lines
    _, _, eidx = olhe.extract(doc, *lhe_synth.PROCESSES["ee_mumu"])
    ev = doc["events"][eidx[0]]
    assert "<wgt" not in text[ev["start"]:ev["end"]]


def test_file_to_helicity_exclusive_weights(rex, tmp_path):
    """SPINUP read from the file feeds helicity-exclusive reweighting of q q~ -> t t~."""
    from rexlib import helicity_tolerance
    src = str(tmp_path / "hel.lhe")
    lhe_synth.write_lhe(src, {"qq_ttx": 600, "gg_ttx": 200}, seed=8, helicities=True)
    L = rex.Lhe(src)
    pin, pout = lhe_synth.PROCESSES["qq_ttx"]
    mom, w, idx = L.extract(pin, pout)
    hel = L.extract_helicities(pin, pout)
    L.close()
    p = rex.Process("qq_ttx", 0)
    p.set_params(ORIG)
    pts = GRIDS["qq_ttx"]
    out = p.reweight_helicity(torch.from_numpy(mom).cuda(), torch.from_numpy(hel).cuda(),
                              torch.from_numpy(w).cuda(), pts).cpu().numpy()
    ref = oracle_rw.reweight_helicity("qq_ttx", mom, hel, w, ORIG, pts)
    zero = ref[:, 0] == 0.0
    assert np.any(zero) and np.all(out[zero] == 0.0)
    bound = helicity_tolerance("qq_ttx", mom, hel, ORIG, pts, 1e-12, np.finfo(np.float64).eps / 2)
    err = np.abs(out - ref) / np.where(ref != 0.0, np.abs(ref), 1.0)
    assert np.all(err[~zero] < bound[~zero])


def test_pp_ttxj_file_every_channel(rex, tmp_path):
    """A p p -> t t~ + jet file with g g, q q~, q g and q~ g events in random beam order:
    each channel extracted by its PDG codes (incoming parton order as listed) and
    reweighted by its own process against the oracle."""
    src = str(tmp_path / "ppj.lhe")
    counts = {"gg_ttxg": 300, "qq_ttxg": 90, "qg_ttxq": 150, "qxg_ttxqx": 70}
    info = lhe_synth.write_lhe(src, counts, seed=6)
    pts = GRIDS["gg_ttxg"]
    L = rex.Lhe(src)
    for proc in counts:
        pin, pout = lhe_synth.PROCESSES[proc]
        mom, w, idx = L.extract(pin, pout)
        assert mom.shape[0] == counts[proc]
        gen, wgen, pos = info[proc]
        order = np.argsort(pos)
        assert np.array_equal(mom, gen[order]) and np.array_equal(w, wgen[order])
        p = rex.Process(proc, 0)
        p.set_params(ORIG)
        out = p.reweight(torch.from_numpy(mom).cuda(), torch.from_numpy(w).cuda(), pts).cpu().numpy()
        ref = oracle_rw.reweight(proc, mom[:8], w[:8], ORIG, pts)
        assert np.max(np.abs(out[:8] / ref - 1)) < 1e-12, proc
        p.close()
    L.close()


def test_file_to_helicity_exclusive_weights_gg_ttxg(rex, tmp_path):
    """SPINUP read from the file feeds helicity-exclusive reweighting of g g -> t t~ g."""
    from rexlib import helicity_tolerance
    src = str(tmp_path / "hel_gg.lhe")
    lhe_synth.write_lhe(src, {"gg_ttxg": 120, "qq_ttx": 40}, seed=9, helicities=True)
    L = rex.Lhe(src)
    pin, pout = lhe_synth.PROCESSES["gg_ttxg"]
    mom, w, idx = L.extract(pin, pout)
    hel = L.extract_helicities(pin, pout)
    L.close()
    p = rex.Process("gg_ttxg", 0)
    p.set_params(ORIG)
    pts = GRIDS["gg_ttxg"]
    out = p.reweight_helicity(torch.from_numpy(mom).cuda(), torch.from_numpy(hel).cuda(),
                              torch.from_numpy(w).cuda(), pts).cpu().numpy()
    # the reference in extended precision: the oracle's own FP64 rounding of small helicity
    # terms exceeds their bound (see test_gpu_helicity.extended_reference)
    ref = np.asarray(oracle_rw.reweight_helicity("gg_ttxg", mom.astype(np.longdouble), hel, w, ORIG, pts),
                     dtype=np.float64)
    bound = helicity_tolerance("gg_ttxg", mom, hel, ORIG, pts, 1e-12, np.finfo(np.float64).eps / 2)
    err = np.abs(out - ref) / np.abs(ref)
    assert np.all(err < bound)
