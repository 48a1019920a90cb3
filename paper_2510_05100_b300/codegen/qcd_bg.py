"""Emit unrolled CUDA for g g -> t t~ + k g as colour-ordered Berends-Giele recursion.

Colour decomposition (one quark line, n gluons, t^a = lambda^a/2):

    M = g_s^n  sum_{s in S_n} (t^{a_s1} ... t^{a_sn})_{i j}  A(s)

with i the top colour and j the antitop colour, s read from the top end of the
line.  The colour-ordered amplitudes ("jamps") A(s) follow from colour-ordered
Feynman rules, obtained from the standard ones by f^{abc} t^c = -i [t^a, t^b]:

* gluon current of an ordered sequence  (outgoing momenta P_X, P_Y, ...):
      J(s) = -1/P_s^2 [ sum_{s = X Y}   V3(X, Y)  +  sum_{s = X Y Z}  V4(X, Y, Z) ]
      V3(X,Y) = (J_X.J_Y)(P_Y - P_X) - (J_X.(P_X + 2 P_Y)) J_Y + (J_Y.(2 P_X + P_Y)) J_X
      V4(X,Y,Z) = (J_X.J_Y) J_Z + (J_Y.J_Z) J_X - 2 (J_X.J_Z) J_Y
  (reflection: J(reversed s) = (-1)^(|s|+1) J(s));
* off-shell antitop line after absorbing the ordered suffix Y:
      psi(Y) = -(q-slash + m)/(q^2 - m^2 + i m Gamma)  sum_{Y = B Y'} (gamma.J_B) psi(Y'),
      q = -(p_tbar + P_Y),  psi(empty) = v(p_tbar);
* jamp:  A(s) = ubar(p_t) sum_{s = B Y} (gamma.J_B) psi(Y).

|M|^2 summed over colours = g_s^(2n) sum_{s,s'} conj(A_s) C_{ss'} A_s' with C the
exact flow colour matrix (``colour_flow``).  Gluon indices: 0, 1 incoming
(outgoing momentum -k), 2.. outgoing.
"""
from __future__ import annotations

import itertools

from .colour_flow import flow_basis, integer_colour_matrix


def _canon(seq: tuple) -> tuple:
    return seq if len(seq) == 1 or seq[0] < seq[-1] else tuple(reversed(seq))


def _sign(seq: tuple) -> int:
    if len(seq) == 1 or seq[0] < seq[-1]:
        return 1
    return 1 if len(seq) % 2 == 1 else -1


def _jn(seq: tuple) -> str:
    return "J" + "".join(str(g) for g in _canon(seq))


def _pn(s) -> str:
    return "P" + "".join(str(g) for g in sorted(s))


def _psin(seq: tuple) -> str:
    return "psi" + "".join(str(g) for g in seq)


class _W:
    def __init__(self):
        self.lines = []

    def __call__(self, s="", ind=1):
        self.lines.append("  " * ind + s if s else "")

    def text(self):
        return "\n".join(self.lines)


def emit_process(name: str, ngluon: int) -> str:
    n = ngluon
    flows = flow_basis(n)
    cint, cden = integer_colour_matrix(n)
    gl = list(range(n))
    canon_seqs = []
    for ln in range(2, n + 1):
        for seq in itertools.permutations(gl, ln):
            if _canon(seq) == seq:
                canon_seqs.append(seq)
    sets = sorted({frozenset(s) for s in canon_seqs}, key=lambda s: (len(s), sorted(s)))
    suffixes = [seq for ln in range(1, n) for seq in itertools.permutations(gl, ln)]
    suffix_sets = sorted({frozenset(s) for s in suffixes}, key=lambda s: (len(s), sorted(s)))

    w = _W()
    w(f"// ---- {name}: g g -> t t~ + {n - 2} g, {n} gluons, {len(flows)} colour flows", 0)
    w(f"// Generated by paper_2510_05100_b300/codegen/qcd_bg.py; do not edit.", 0)
    w(f"struct {name}_info {{", 0)
    w(f"static constexpr int NGLUON = {n};")
    w(f"static constexpr int NFLOW = {len(flows)};")
    w(f"static constexpr int NGHEL = {2 ** n};")
    w(f"static constexpr int COLOUR_DEN = {cden};")
    w("};", 0)
    w("", 0)
    # colour matrix as a table for the tensor-core path / host
    w(f"// exact flow colour matrix C = {name}_colour / {cden}; flows (top end first):", 0)
    for k, f in enumerate(flows):
        w(f"//   flow {k}: {f}", 0)
    w(f"constexpr int {name}_colour[{len(flows)}][{len(flows)}] = {{", 0)
    for row in cint:
        w("{" + ", ".join(str(v) for v in row) + "},")
    w("};", 0)
    w("", 0)

    # ---------------- gluon state (mass independent)
    w(f"template <typename R>", 0)
    w(f"struct {name}_gluons {{", 0)
    for g in gl:
        w(f"R J{g}[4];")
    for s in canon_seqs:
        w(f"R {_jn(s)}[4];")
    for st in suffix_sets:
        w(f"R Q{''.join(str(g) for g in sorted(st))}[4];   // -(p_tbar + P)")
    w("};", 0)
    w("", 0)
    w("// gluon currents for one gluon polarisation configuration (mass independent)", 0)
    w(f"template <typename R>", 0)
    w(f"__device__ __forceinline__ void {name}_gluon_state(const R (&pg)[{n}][4], "
      f"const R (&eps)[{n}][4], const R (&ptb)[4], {name}_gluons<R>& st) {{", 0)
    for g in gl:
        w(f"const R* P{g} = pg[{g}];")
        w(f"#pragma unroll", 0)
        w(f"for (int m = 0; m < 4; ++m) st.J{g}[m] = eps[{g}][m];")
    for s in sets:
        if len(s) < 2:
            continue
        nm = _pn(s)
        terms = " + ".join(f"pg[{g}][m]" for g in sorted(s))
        w(f"R {nm}[4];")
        w(f"#pragma unroll", 0)
        w(f"for (int m = 0; m < 4; ++m) {nm}[m] = {terms};")
    for s in canon_seqs:
        w(f"{{  // J({','.join(map(str, s))})")
        w(f"R t[4] = {{R(0), R(0), R(0), R(0)}};", 2)
        for i in range(1, len(s)):
            x, y = s[:i], s[i:]
            sg = _sign(x) * _sign(y)
            w(f"vvv_acc(R({sg}), st.{_jn(x)}, {_pn(x) if len(x) > 1 else 'P%d' % x[0]}, "
              f"st.{_jn(y)}, {_pn(y) if len(y) > 1 else 'P%d' % y[0]}, t);", 2)
        for i in range(1, len(s)):
            for j in range(i + 1, len(s)):
                x, y, z = s[:i], s[i:j], s[j:]
                sg = _sign(x) * _sign(y) * _sign(z)
                w(f"vvvv_acc(R({sg}), st.{_jn(x)}, st.{_jn(y)}, st.{_jn(z)}, t);", 2)
        pn = _pn(s)
        w(f"const R f = R(-1) / mdot({pn}, {pn});", 2)
        w(f"#pragma unroll", 0)
        w(f"for (int m = 0; m < 4; ++m) st.{_jn(s)}[m] = f * t[m];", 2)
        w("}")
    for st_ in suffix_sets:
        nm = "Q" + "".join(str(g) for g in sorted(st_))
        terms = " + ".join(f"pg[{g}][m]" for g in sorted(st_))
        w(f"#pragma unroll", 0)
        w(f"for (int m = 0; m < 4; ++m) st.{nm}[m] = -(ptb[m] + {terms});")
    w("}", 0)
    w("", 0)

    # ---------------- quark line for one mass: sum over top/antitop helicities
    w("// sum over top and antitop helicities of sum_{s,s'} conj(A_s) Cint_{ss'} A_s'", 0)
    w("// for one (mass, width); Cint = C * COLOUR_DEN.  WIDTH selects complex denominators.", 0)
    w("// The quadratic form of one helicity is evaluated in CS (a positive-definite form:", 0)
    w("// no cancellation), and the helicity sum is accumulated in ACC.", 0)
    w(f"template <typename R, typename ACC, bool WIDTH, typename CS = ACC>", 0)
    w(f"__device__ __forceinline__ ACC {name}_quark_line(const {name}_gluons<R>& st, "
      f"const R (&pt)[4], const R (&ptb)[4], R mt, R wt) {{", 0)
    w("ACC total = ACC(0);")
    # propagator denominators
    for st_ in suffix_sets:
        nm = "".join(str(g) for g in sorted(st_))
        w(f"const R d{nm} = mdot(st.Q{nm}, st.Q{nm}) - mt * mt;")
        w(f"R id{nm}r, id{nm}i;")
        w(f"if (WIDTH) {{ const R im = mt * wt; const R nn = R(1) / (d{nm} * d{nm} + im * im); "
          f"id{nm}r = d{nm} * nn; id{nm}i = -im * nn; }} else {{ id{nm}r = R(1) / d{nm}; id{nm}i = R(0); }}")
    w("cx<R> ut[2][4];")
    w("spinor_u(pt, mt, -1, ut[0]);")
    w("spinor_u(pt, mt, +1, ut[1]);")
    w("#pragma unroll 1", 0)
    w("for (int hb = 0; hb < 2; ++hb) {")
    w("cx<R> v[4];", 2)
    w("spinor_v(ptb, mt, hb == 0 ? -1 : +1, v);", 2)
    for seq in suffixes:
        nm = _psin(seq)
        key = "".join(str(g) for g in sorted(seq))
        w(f"cx<R> {nm}[4];", 2)
        w("{", 2)
        w("cx<R> t[4] = {};", 3)
        for i in range(1, len(seq) + 1):
            b, rest = seq[:i], seq[i:]
            src = _psin(rest) if rest else "v"
            w(f"slash_acc(R({_sign(b)}), st.{_jn(b)}, {src}, t);", 3)
        w(f"if (WIDTH) fermion_prop(st.Q{key}, mt, cx<R>{{id{key}r, id{key}i}}, t, {nm});", 3)
        w(f"else fermion_prop_real(st.Q{key}, mt, id{key}r, t, {nm});", 3)
        w("}", 2)
    nf = len(flows)
    w(f"cx<R> A[2][{nf}];", 2)
    for k, f in enumerate(flows):
        w("{", 2)
        w("cx<R> x[4] = {};", 3)
        for i in range(1, n + 1):
            b, rest = f[:i], f[i:]
            src = _psin(rest) if rest else "v"
            w(f"slash_acc(R({_sign(b)}), st.{_jn(b)}, {src}, x);", 3)
        w(f"A[0][{k}] = ubar_dot(ut[0], x);", 3)
        w(f"A[1][{k}] = ubar_dot(ut[1], x);", 3)
        w("}", 2)
    w("#pragma unroll", 0)
    w("for (int ht = 0; ht < 2; ++ht) {", 2)
    w("CS s = CS(0);", 3)
    for i in range(nf):
        w(f"s += CS({cint[i][i]}) * (CS(A[ht][{i}].re) * CS(A[ht][{i}].re) + "
          f"CS(A[ht][{i}].im) * CS(A[ht][{i}].im));", 3)
    for i in range(nf):
        for j in range(i + 1, nf):
            c = cint[i][j]
            if c == 0:
                continue
            w(f"s += CS({2 * c}) * (CS(A[ht][{i}].re) * CS(A[ht][{j}].re) + "
              f"CS(A[ht][{i}].im) * CS(A[ht][{j}].im));", 3)
    w("total += ACC(s);", 3)
    w("}", 2)
    w("}")
    w("return total;")
    w("}", 0)
    w("", 0)
    return w.text()


PROCESSES = [("gg_ttx", 2), ("gg_ttxg", 3), ("gg_ttxgg", 4)]


def emit_all() -> str:
    parts = [
        "// Colour-ordered Berends-Giele amplitudes for g g -> t t~ + k g (k = 0, 1, 2).",
        "// Generated by paper_2510_05100_b300/codegen/qcd_bg.py (python -m",
        "// paper_2510_05100_b300.codegen); do not edit.",
        "#pragma once",
        '#include "../helas.cuh"',
        "",
        "namespace rex {",
        "",
    ]
    for name, n in PROCESSES:
        parts.append(emit_process(name, n))
    parts.append("}  // namespace rex")
    parts.append("")
    return "\n".join(parts)
