"""The LHE oracle against a hand-written fixture (tests/golden/tiny.lhe): the values
below are typed from the fixture's text, and the expected writer output is spelled
out literally."""
import os

import numpy as np

from oracle import lhe

HERE = os.path.dirname(os.path.abspath(__file__))
TINY = os.path.join(HERE, "golden", "tiny.lhe")


def test_reads_the_fixture():
    doc = lhe.read(TINY)
    assert len(doc["events"]) == 3
    e0, e1, e2 = doc["events"]
    assert e0["head"][:3] == [5, 1, 0.25] and e1["head"][:3] == [4, 2, -0.125] and e2["head"][0] == 6
    assert e0["particles"][2][:2] == [6, 1] and e0["particles"][2][6:11] == [10.0, 20.0, 30.0, 200.0, 173.0]
    assert e2["particles"][5][:2] == [25, 2]          # an intermediate (status 2) particle


def test_extracts_and_reindexes_a_process():
    doc = lhe.read(TINY)
    mom, w, idx = lhe.extract(doc, [21, 21], [6, -6, 21])
    assert list(idx) == [0, 2] and list(w) == [0.25, 0.75]
    # event 0 is written g g t g t~; event 2 g g g t~ t (plus a status-2 Higgs, ignored)
    assert np.array_equal(mom[0], [[300, 0, 0, 300], [250, 0, 0, -250], [200, 10, 20, 30],
                                   [290, -5, -24, 0], [60, -5, 4, 20]])
    assert np.array_equal(mom[1][2], [696, 9, -2, -3]) and np.array_equal(mom[1][3], [300, -10, 0, 0])
    assert np.array_equal(mom[1][4], [4, 1, 2, 3])
    mom2, w2, idx2 = lhe.extract(doc, [21, 21], [6, -6])
    assert list(idx2) == [1] and list(w2) == [-0.125]
    assert np.array_equal(mom2[0][2], [400, -100, 0, -50]) and np.array_equal(mom2[0][3], [400, 100, 0, 50])
    assert lhe.extract(doc, [11, -11], [13, -13])[0].shape == (0, 4, 4)


def test_writes_weights_into_events_and_header():
    doc = lhe.read(TINY)
    out = lhe.write(doc, [("rw1", [0, 2], [1.5, -2.0]), ("rw2", [1], [3.0])])
    assert ("<initrwgt>\n<weightgroup name='rex_b300'>\n<weight id='rw1'>rw1</weight>\n"
            "<weight id='rw2'>rw2</weight>\n</weightgroup>\n</initrwgt>\n</header>") in out
    # event 0 had no <rwgt>: a new block before </event>
    assert ("# a comment line\n<rwgt>\n<wgt id='rw1'> +1.5000000000e+00 </wgt>\n</rwgt>\n</event>") in out
    # event 1 had one: the new weight goes inside it, after the existing one
    assert ("<wgt id='old'> +1.0000000000e+00 </wgt>\n<wgt id='rw2'> +3.0000000000e+00 </wgt>\n</rwgt>") in out
    assert "<wgt id='rw1'> -2.0000000000e+00 </wgt>" in out
    # everything else is untouched
    assert out.replace("<wgt id='rw1'> +1.5000000000e+00 </wgt>\n", "").count("<event>") == 3
    rd = lhe.read(TINY)
    assert lhe.write(rd, []) == rd["text"]
