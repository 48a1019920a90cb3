"""LHE v3 reading, process extraction and weight writing (oracle; test
infrastructure only).

The front-end that sits before and after the reweighting path (paper Sec. 2:
events read from an LHE file, sorted into processes by comparing their external
legs (eventBelongs), partons reindexed to the process's order, transposed to a
structure of arrays; Sec. 3.1: new weights appended to every event and declared
in the header's <initrwgt> block).  Plain Python over the file text:

read(path)            the file text and, per event, its text span, its first
                      line (nUP idPrUP xWgtUP scalUP aQEDUP aQCDUP) and its nUP
                      particle lines (idUP iStUP mothUP1 mothUP2 iColUP1 iColUP2
                      px py pz E m vTimUP spinUP);
extract(doc, in, out) the events whose status -1 particles carry the PDG codes
                      `in` and whose status +1 particles carry `out` (as
                      multisets; other statuses are ignored), with momenta
                      (E, px, py, pz) in the requested order (identical codes in
                      file order), the event weights xWgtUP and the event indices;
extract_helicities(doc, in, out)
                      the same events' SPINUP values rounded to integers, in the
                      same particle order (9, unknown, where a line lacks it);
write(doc, weights)   the file text with, for every weight id (in the order
                      given) and every event that has a value for it, a line
                      "<wgt id='ID'> %+.10e </wgt>" inside the event's last
                      <rwgt> block (a new block before </event> if it has none),
                      and the header's <initrwgt> extended by a
                      "<weightgroup name='rex_b300'>" of "<weight id='ID'>ID</weight>"
                      lines (a new <initrwgt> before </header>, or a new header
                      before <init> if the file has none).
"""
from __future__ import annotations

import re

import numpy as np

_EVENT = re.compile(r"<event(?=[\s>])")
_INIT = re.compile(r"<init(?=[\s>])")
GROUP_NAME = "rex_b300"


def read(path: str) -> dict:
    with open(path, "r") as f:
        text = f.read()
    events = []
    pos = _INIT.search(text).start()
    while True:
        m = _EVENT.search(text, pos)
        if not m:
            break
        start = m.start()
        end = text.index("</event>", start) + len("</event>")
        body = text[text.index(">", start) + 1:end - len("</event>")]
        lines = [ln for ln in body.split("\n") if ln.strip()]
        head = lines[0].split()
        nup = int(head[0])
        parts = []
        for ln in lines[1:1 + nup]:
            f = ln.split()
            parts.append([int(f[0]), int(f[1]), int(f[2]), int(f[3]), int(f[4]), int(f[5])]
                         + [float(x) for x in f[6:13]])
        events.append({"start": start, "end": end,
                       "head": [nup, int(head[1]), float(head[2]), float(head[3]), float(head[4]), float(head[5])],
                       "particles": parts})
        pos = end
    return {"text": text, "events": events}


def extract(doc: dict, pdg_in, pdg_out):
    pdg_in, pdg_out = list(pdg_in), list(pdg_out)
    mom, w, idx = [], [], []
    for i, ev in enumerate(doc["events"]):
        ins = [p for p in ev["particles"] if p[1] == -1]
        outs = [p for p in ev["particles"] if p[1] == 1]
        if sorted(p[0] for p in ins) != sorted(pdg_in) or sorted(p[0] for p in outs) != sorted(pdg_out):
            continue
        row = []
        for group, wanted in ((ins, pdg_in), (outs, pdg_out)):
            used = [False] * len(group)
            for code in wanted:
                k = next(k for k, p in enumerate(group) if not used[k] and p[0] == code)
                used[k] = True
                p = group[k]
                row.append([p[9], p[6], p[7], p[8]])          # E, px, py, pz
        mom.append(row)
        w.append(ev["head"][2])
        idx.append(i)
    n = len(pdg_in) + len(pdg_out)
    return (np.array(mom, dtype=np.float64).reshape(len(mom), n, 4), np.array(w, dtype=np.float64),
            np.array(idx, dtype=np.int64))


def extract_helicities(doc: dict, pdg_in, pdg_out) -> np.ndarray:
    pdg_in, pdg_out = list(pdg_in), list(pdg_out)
    rows = []
    for ev in doc["events"]:
        ins = [p for p in ev["particles"] if p[1] == -1]
        outs = [p for p in ev["particles"] if p[1] == 1]
        if sorted(p[0] for p in ins) != sorted(pdg_in) or sorted(p[0] for p in outs) != sorted(pdg_out):
            continue
        row = []
        for group, wanted in ((ins, pdg_in), (outs, pdg_out)):
            used = [False] * len(group)
            for code in wanted:
                k = next(k for k, p in enumerate(group) if not used[k] and p[0] == code)
                used[k] = True
                row.append(int(round(group[k][12])) if len(group[k]) > 12 else 9)
        rows.append(row)
    return np.array(rows, dtype=np.int8).reshape(len(rows), len(pdg_in) + len(pdg_out))


def write(doc: dict, weights: list) -> str:
    """weights: list of (id, index array, value array), in the order ids appear."""
    text = doc["text"]
    ids = [wid for wid, _, _ in weights]
    per_event = {}
    for wid, index, values in weights:
        for i, v in zip(index, values):
            per_event.setdefault(int(i), []).append((wid, float(v)))
    out = []
    # header: the text before the <init> block
    init_at = _INIT.search(text).start()
    header = text[:init_at]
    if ids:
        group = ("<weightgroup name='%s'>\n" % GROUP_NAME
                 + "".join("<weight id='%s'>%s</weight>\n" % (i, i) for i in ids) + "</weightgroup>\n")
        if "</initrwgt>" in header:
            k = header.index("</initrwgt>")
            header = header[:k] + group + header[k:]
        elif "</header>" in header:
            k = header.index("</header>")
            header = header[:k] + "<initrwgt>\n" + group + "</initrwgt>\n" + header[k:]
        else:
            header = header + "<header>\n<initrwgt>\n" + group + "</initrwgt>\n</header>\n"
    out.append(header)
    prev = init_at
    for i, ev in enumerate(doc["events"]):
        out.append(text[prev:ev["start"]])
        etext = text[ev["start"]:ev["end"]]
        vals = per_event.get(i)
        if vals:
            # weights in the order of the ids
            order = {wid: n for n, wid in enumerate(ids)}
            vals = sorted(vals, key=lambda t: order[t[0]])
            lines = "".join("<wgt id='%s'> %+.10e </wgt>\n" % (wid, v) for wid, v in vals)
            if "</rwgt>" in etext:
                k = etext.rindex("</rwgt>")
                etext = etext[:k] + lines + etext[k:]
            else:
                k = etext.rindex("</event>")
                etext = etext[:k] + "<rwgt>\n" + lines + "</rwgt>\n" + etext[k:]
        out.append(etext)
        prev = ev["end"]
    out.append(text[prev:])
    return "".join(out)
