"""Algorithmic flop counts of the amplitude code, for roofline figures.

Compiles and runs csrc/tools/flopcount.cpp (the generated amplitude routines
instantiated with a counting scalar type) with the host compiler and caches the
result under _build/.  Counts are per call of each routine:
  event_setup                  once per event
  mass_setup                   once per (event, mass slot)
  polarisations, gluon_currents once per (event, gluon polarisation configuration)
  quark_line_amp / _acc        once per (event, gluon polarisation, mass slot);
                               amplitude arithmetic / colour+helicity accumulation.
"""
from __future__ import annotations

import functools
import json
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "csrc", "tools", "flopcount.cpp")
GEN = os.path.join(HERE, "csrc", "generated", "qcd_amplitudes.cuh")
BUILD = os.path.join(os.path.dirname(HERE), "_build")


@functools.lru_cache(maxsize=None)
def counts() -> dict:
    os.makedirs(BUILD, exist_ok=True)
    exe = os.path.join(BUILD, "flopcount")
    newest = max(os.path.getmtime(SRC), os.path.getmtime(GEN),
                 *(os.path.getmtime(os.path.join(HERE, "csrc", f))
                   for f in ("helas.cuh", "qq_amplitude.cuh", "qqg_amplitude.cuh")))
    if not os.path.exists(exe) or os.path.getmtime(exe) < newest:
        subprocess.run(["g++", "-O0", "-std=c++17", "-o", exe, SRC], check=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    return json.loads(out)


def per_event(proc: str, nmass: int, exclusive: bool = False) -> dict:
    """Flops of one event evaluated at ``nmass`` distinct mass slots.

    'amp': amplitude arithmetic (FP64 in REX_FP64, FP32 in REX_MIXED);
    'acc': colour/helicity accumulation (FP64 in both modes).
    exclusive: the helicity-exclusive g g tile, whose lanes evaluate the quark line
    for the event's own antitop helicity only (its colour form counted as the summed
    tile's; the warp shuffles that combine the lanes' jamps are not counted).
    """
    c = counts()[proc]
    nh = c["nghel"]
    line = c["quark_line_amp_one_antitop"] if exclusive else c["quark_line_amp"]
    amp = (c["event_setup"] + nmass * c["mass_setup"]
           + nh * (c["gluon_currents"] + c["polarisations"] + nmass * line))
    acc = nh * nmass * c["quark_line_acc"]
    return {"amp": amp, "acc": acc, "total": amp + acc}
