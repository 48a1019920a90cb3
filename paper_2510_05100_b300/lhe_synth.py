"""Synthetic LHE v3 files for the front-end's tests and benchmark.

An input generator (no matrix-element arithmetic): seeded events of several
processes (momenta from phase_space.make_events) are written interleaved in a
seeded random order.  Each event's final-state particles are written in a seeded
random order between different PDG codes, identical codes keeping their
generated order, so that a reader that reindexes to the process order recovers
the generated arrays exactly.  Momenta and masses are written with 17
significant digits (exact round trip).  Some events carry an extra status-2
particle, a comment line, or an existing <rwgt> block.  With helicities=True every
particle gets a seeded random helicity +1/-1 in the SPINUP column (9, unknown,
otherwise).
"""
from __future__ import annotations

import numpy as np

from . import phase_space as ps

# PDG codes of the incoming and outgoing particles of each process, in the
# particle order of the momentum arrays
PROCESSES = {
    "ee_mumu": ([-11, 11], [-13, 13]),
    "gg_ttx": ([21, 21], [6, -6]),
    "gg_ttxg": ([21, 21], [6, -6, 21]),
    "gg_ttxgg": ([21, 21], [6, -6, 21, 21]),
    "qq_ttx": ([2, -2], [6, -6]),
    "qq_ttxg": ([2, -2], [6, -6, 21]),
    "qg_ttxq": ([2, 21], [6, -6, 2]),
    "qxg_ttxqx": ([-2, 21], [6, -6, -2]),
}
_MASS = {6: 173.0, -6: 173.0}


def _order(codes: list, rng) -> list:
    """A random permutation of positions that keeps identical codes in order."""
    perm = list(rng.permutation(len(codes)))
    # the k-th slot (in file order) holding code c gets the k-th particle with code c
    out, seen = [], {}
    slots = [codes[p] for p in perm]
    for c in slots:
        k = seen.get(c, 0)
        seen[c] = k + 1
        out.append([i for i, x in enumerate(codes) if x == c][k])
    return out


def write_lhe(path: str, counts: dict, seed: int = 0, with_initrwgt: bool = False, helicities: bool = False) -> dict:
    """Write a synthetic LHE file.  counts: {process name: number of events}.

    Returns {process: (momenta [n][npart][4], weights [n], file positions [n])},
    the arrays in generation order with each event's position in the file; with
    helicities=True a fourth array, the int8 helicities [n][npart]."""
    rng = np.random.default_rng(seed)
    data = {}
    labels = []
    for i, (proc, n) in enumerate(sorted(counts.items())):
        mom = ps.make_events(proc, n, seed * 100 + i + 1)
        w = rng.uniform(0.5, 1.5, n)
        w[rng.random(n) < 0.01] *= -1.0
        hel = (rng.choice(np.array([-1, 1], dtype=np.int8), size=mom.shape[:2]) if helicities
               else np.full(mom.shape[:2], 9, dtype=np.int8))
        data[proc] = (mom, w, hel)
        labels += [(proc, j) for j in range(n)]
    order = rng.permutation(len(labels))
    pos = {proc: np.empty(n, dtype=np.int64) for proc, n in counts.items()}
    out = ['<LesHouchesEvents version="3.0">\n<header>\n<!-- synthetic events -->\n']
    if with_initrwgt:
        out.append("<initrwgt>\n<weightgroup name='old'>\n<weight id='old'>old</weight>\n</weightgroup>\n"
                   "</initrwgt>\n")
    out.append("</header>\n<init>\n2212 2212 6.5e+03 6.5e+03 0 0 247000 247000 -4 1\n"
               "1.0e+02 1.0e+00 1.0e+02 1\n</init>\n")
    for fpos, lab in enumerate(order):
        proc, j = labels[lab]
        pos[proc][j] = fpos
        mom, w, hel = data[proc]
        pin, pout = PROCESSES[proc]
        extra = proc == "gg_ttxg" and rng.random() < 0.1
        lines = []
        ins = _order(pin, rng)
        outs = _order(pout, rng)
        rows = [(pin[k], -1, k) for k in ins] + [(pout[k], 1, len(pin) + k) for k in outs]
        nup = len(rows) + (1 if extra else 0)
        lines.append(" %d 1 %+.16e %.8e %.8e %.8e" % (nup, w[j], 173.0, 7.546771e-3, 0.118))
        for code, st, r in rows:
            e, px, py, pz = mom[j, r]
            moth = (0, 0) if st == -1 else (1, 2)
            lines.append(" %d %d %d %d %d %d %+.16e %+.16e %+.16e %.16e %.16e 0.0000e+00 %.4e"
                         % (code, st, moth[0], moth[1], 501 + r, 0, px, py, pz, e, _MASS.get(code, 0.0),
                            float(hel[j, r])))
        if extra:
            lines.append(" 25 2 1 2 0 0 +0.0 +0.0 +0.0 1.25e+02 1.25e+02 0.0000e+00 0.0000e+00")
        u = rng.random()
        if u < 0.05:
            lines.append("# synthetic comment")
        elif with_initrwgt and u < 0.5:
            lines.append("<rwgt>\n<wgt id='old'> %+.10e </wgt>\n</rwgt>" % w[j])
        out.append("<event>\n" + "\n".join(lines) + "\n</event>\n")
    out.append("</LesHouchesEvents>\n")
    with open(path, "w") as f:
        f.write("".join(out))
    if helicities:
        return {proc: (data[proc][0], data[proc][1], pos[proc], data[proc][2]) for proc in counts}
    return {proc: (data[proc][0], data[proc][1], pos[proc]) for proc in counts}
