"""The native LHE front-end (rex_lhe_*) against the LHE oracle: process extraction
with parton reindexing and the weight writer, on the hand-written fixture and on
synthetic multi-process files (CPU; the front-end is host code)."""
import os

import numpy as np
import pytest

from rexlib import ensure_built
from oracle import lhe as olhe
from paper_2510_05100_b300 import lhe_synth

HERE = os.path.dirname(os.path.abspath(__file__))
TINY = os.path.join(HERE, "golden", "tiny.lhe")
SIGS = [([21, 21], [6, -6, 21]), ([21, 21], [6, -6]), ([21, 21], [6, -6, 21, 21]), ([-11, 11], [-13, 13]),
        ([21, 21], [-6, 21, 6])]


@pytest.fixture(scope="module")
def rex():
    return ensure_built()


@pytest.fixture(scope="module")
def synth(tmp_path_factory):
    path = str(tmp_path_factory.mktemp("lhe") / "synth.lhe")
    info = lhe_synth.write_lhe(path, {"gg_ttxg": 6000, "gg_ttx": 3000, "ee_mumu": 700, "gg_ttxgg": 500,
                                      "qq_ttx": 800, "qq_ttxg": 400, "qg_ttxq": 300, "qxg_ttxqx": 200}, seed=11,
                               with_initrwgt=True)
    return path, info


def same(a, b):
    return all(np.array_equal(x, y) for x, y in zip(a, b))


def test_fixture_matches_the_oracle(rex):
    L = rex.Lhe(TINY)
    doc = olhe.read(TINY)
    assert L.num_events == 3
    for pin, pout in SIGS:
        assert same(L.extract(pin, pout), olhe.extract(doc, pin, pout)), (pin, pout)
    L.close()


@pytest.mark.parametrize("threads", [1, 8])
def test_synthetic_file_matches_the_oracle_and_the_generator(rex, synth, threads):
    path, info = synth
    L = rex.Lhe(path, nthreads=threads)
    doc = olhe.read(path)
    assert L.num_events == len(doc["events"]) == 11900
    for proc, (pin, pout) in lhe_synth.PROCESSES.items():
        got = L.extract(pin, pout)
        assert same(got, olhe.extract(doc, pin, pout)), proc
        mom, w, pos = info[proc]
        order = np.argsort(pos)
        assert np.array_equal(got[0], mom[order]) and np.array_equal(got[1], w[order])
        assert np.array_equal(got[2], pos[order])
    L.close()


def test_writer_matches_the_oracle_text(rex, synth, tmp_path):
    path, _ = synth
    L = rex.Lhe(path)
    doc = olhe.read(path)
    g = np.random.default_rng(3)
    weights = []
    for wid, (pin, pout) in (("mt171", ([21, 21], [6, -6, 21])), ("mt171", ([21, 21], [6, -6])),
                             ("as0.12", ([21, 21], [6, -6, 21]))):
        _, w, idx = L.extract(pin, pout)
        vals = w * g.uniform(0.5, 2.0, w.size)
        L.set_weights(wid, idx, vals)
        weights.append((wid, idx, vals))
    out = str(tmp_path / "out.lhe")
    L.write(out)
    # the oracle takes one (id, index, values) list per id
    merged = {}
    for wid, idx, vals in weights:
        a, b = merged.get(wid, (np.empty(0, np.int64), np.empty(0)))
        merged[wid] = (np.concatenate([a, idx]), np.concatenate([b, vals]))
    ref = olhe.write(doc, [(wid, *merged[wid]) for wid in ("mt171", "as0.12")])
    assert open(out).read() == ref
    # the written file reads back to the same events
    L2 = rex.Lhe(out)
    for pin, pout in SIGS:
        assert same(L2.extract(pin, pout), L.extract(pin, pout))
    L.close()
    L2.close()


def test_header_is_created_when_missing(rex, tmp_path):
    text = open(TINY).read()
    start, end = text.index("<header>"), text.index("</header>") + len("</header>\n")
    path = str(tmp_path / "noheader.lhe")
    open(path, "w").write(text[:start] + text[end:])
    L = rex.Lhe(path)
    L.set_weights("w1", [0, 1, 2], [1.0, 2.0, 3.0])
    out = str(tmp_path / "noheader_out.lhe")
    L.write(out)
    assert open(out).read() == olhe.write(olhe.read(path), [("w1", [0, 1, 2], [1.0, 2.0, 3.0])])
    L.close()


def test_errors(rex, tmp_path):
    with pytest.raises(rex.RexError):
        rex.Lhe(str(tmp_path / "missing.lhe"))
    bad = str(tmp_path / "bad.lhe")
    open(bad, "w").write(open(TINY).read().replace("</event>\n</LesHouchesEvents>", ""))
    with pytest.raises(rex.RexError):
        rex.Lhe(bad)
    L = rex.Lhe(TINY)
    with pytest.raises(rex.RexError):
        L.set_weights("x", [3], [1.0])            # index out of range
    with pytest.raises(rex.RexError):
        L.set_weights("it's", [0], [1.0])         # markup in the id
    L.close()


def test_helicity_column(rex, tmp_path):
    """SPINUP of the fixture (pinned by hand for its first event) and of a synthetic file with
    random helicities: the native reader against the oracle reader and the generator."""
    L = rex.Lhe(TINY)
    doc = olhe.read(TINY)
    for pin, pout in SIGS:
        assert np.array_equal(L.extract_helicities(pin, pout), olhe.extract_helicities(doc, pin, pout))
    # first event: g(+1) g(-1) -> t(+1) t~(-1) g(+1), in the order g g t t~ g
    assert L.extract_helicities([21, 21], [6, -6, 21])[0].tolist() == [1, -1, 1, -1, 1]
    L.close()
    path = str(tmp_path / "hel.lhe")
    info = lhe_synth.write_lhe(path, {"qq_ttx": 700, "ee_mumu": 300, "gg_ttxg": 500}, seed=13, helicities=True)
    L = rex.Lhe(path)
    doc = olhe.read(path)
    for proc in info:
        pin, pout = lhe_synth.PROCESSES[proc]
        got = L.extract_helicities(pin, pout)
        assert np.array_equal(got, olhe.extract_helicities(doc, pin, pout))
        mom, w, pos, hel = info[proc]
        assert np.array_equal(got, hel[np.argsort(pos)])
    L.close()
    # without the option every particle is written as unknown (9)
    path2 = str(tmp_path / "nohel.lhe")
    lhe_synth.write_lhe(path2, {"qq_ttx": 10}, seed=14)
    L = rex.Lhe(path2)
    assert np.all(L.extract_helicities([2, -2], [6, -6]) == 9)
    L.close()
