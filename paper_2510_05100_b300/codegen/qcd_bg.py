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


def _sn(st) -> str:
    return "".join(str(g) for g in sorted(st))


def emit_process(name: str, ngluon: int) -> str:
    n = ngluon
    flows = flow_basis(n)
    fidx = {f: i for i, f in enumerate(flows)}
    cint, cden = integer_colour_matrix(n)
    gl = list(range(n))
    canon_seqs = [seq for ln in range(2, n + 1) for seq in itertools.permutations(gl, ln)
                  if _canon(seq) == seq]
    gsets = sorted({frozenset(s) for s in canon_seqs}, key=lambda s: (len(s), sorted(s)))
    gidx = {st: i for i, st in enumerate(gsets)}
    suffix_sets = sorted({frozenset(c) for ln in range(1, n) for c in itertools.combinations(gl, ln)},
                         key=lambda s: (len(s), sorted(s)))
    sidx = {st: i for i, st in enumerate(suffix_sets)}
    nsuf, ngs = len(suffix_sets), len(gsets)

    def pref(seq):   # momentum sum of a gluon sequence, as an expression
        return f"ev.pg[{seq[0]}]" if len(seq) == 1 else f"ev.ps[{gidx[frozenset(seq)]}]"

    w = _W()
    w(f"// ---- {name}: g g -> t t~ + {n - 2} g, {n} gluons, {len(flows)} colour flows", 0)
    w(f"struct {name}_info {{", 0)
    w(f"static constexpr int NGLUON = {n};")
    w(f"static constexpr int NFLOW = {len(flows)};")
    w(f"static constexpr int NGHEL = {2 ** n};")
    w(f"static constexpr int COLOUR_DEN = {cden};")
    w(f"static constexpr int NSUFFIX = {nsuf};   // gluon sets absorbed on the antitop side")
    w(f"static constexpr int NGSET = {ngs};      // gluon sets of two or more (internal gluons)")
    w("};", 0)
    w("", 0)
    w(f"// exact flow colour matrix C = {name}_colour / {cden}; flows (top end first):", 0)
    for k, f in enumerate(flows):
        w(f"//   flow {k}: {f}", 0)
    w(f"constexpr int {name}_colour[{len(flows)}][{len(flows)}] = {{", 0)
    for row in cint:
        w("{" + ", ".join(str(v) for v in row) + "},")
    w("};", 0)
    w("#if defined(__CUDACC__)", 0)
    w(f"// device copy for lane-indexed reads (tensor-core colour form)", 0)
    w(f"__constant__ int {name}_colour_dev[{len(flows)}][{len(flows)}] = {{", 0)
    for row in cint:
        w("{" + ", ".join(str(v) for v in row) + "},")
    w("};", 0)
    w("#endif", 0)
    w("", 0)
    w("// gluon sets (internal gluon lines): " + ", ".join(f"{i}={{{_sn(st)}}}" for st, i in gidx.items()), 0)
    w("// suffix sets (off-shell antitop lines): " + ", ".join(f"{i}={{{_sn(st)}}}" for st, i in sidx.items()), 0)

    # ---------------- event-level data, filled cooperatively by the event's lanes
    npart = n + 2
    vecs = [f"g{g}" for g in gl] + ["tb"]            # dot-product vectors: pg[0..n-1], p_tbar
    dots = [(i, j) for i in range(n + 1) for j in range(i, n + 1)]
    didx = {d: k for k, d in enumerate(dots)}

    def dot(i, j):
        return f"ev.dd[{didx[(min(i, j), max(i, j))]}]"

    def inv_sq(members):     # (sum of vectors)^2 from the dot table
        terms = [dot(i, i) for i in members]
        terms += [f"2.0 * {dot(i, j)}" for a_, i in enumerate(members) for j in members[a_ + 1:]]
        return " + ".join(terms)

    w("template <typename R>", 0)
    w(f"struct {name}_event {{", 0)
    w(f"R praw[{npart * 4}];     // particle momenta converted to R")
    w(f"double dd[{len(dots)}];  // FP64 dot products of (pg_0..pg_{n - 1}, p_tbar)")
    w(f"R pg[{n}][4];          // outgoing-convention gluon momenta (incoming: -k)")
    w("R pt[4], ptb[4];       // top, antitop")
    w(f"R ps[{ngs}][4];        // momentum sum of each gluon set")
    w(f"R fg[{ngs}];           // -1 / P^2 of each gluon set (P^2 in FP64)")
    w(f"R q[{nsuf}][4];        // -(p_tbar + P) of each suffix set")
    w(f"double q2[{nsuf}];     // q^2 in FP64 (the exact mode's mass slot subtracts m^2 in FP64)")
    w(f"R qm[{nsuf}];          // q^2 - m0^2 (FP64, then R): the mixed mode's slot adds m0^2 - m^2 in R")
    w("cx<R> cht[2][2], chb[2][2];   // helicity 2-spinors chi-, chi+ of top / antitop")
    w("R wpt, iwpt, wptb, iwptb;     // omega_+ and 1/omega_+ of top / antitop")
    w("};", 0)
    w("", 0)
    w("template <typename R>", 0)
    w(f"struct {name}_mass {{   // one (event, mass slot), shared memory", 0)
    w("cx<R> ut[2][4];        // u(p_t) for top helicity -, +")
    w("cx<R> v[2][4];         // v(p_tbar) for antitop helicity -, +")
    w(f"R idr[{nsuf}], idi[{nsuf}];   // 1/(q^2 - m^2 + i m Gamma), real and imaginary parts")
    w("R m;")
    w("};", 0)
    w("", 0)
    w("template <typename R>", 0)
    w(f"struct {name}_gluons {{   // colour-ordered gluon currents of one polarisation configuration", 0)
    for g in gl:
        w(f"R J{g}[4];")
    for sq in canon_seqs:
        w(f"R {_jn(sq)}[4];")
    w("};", 0)
    w("", 0)

    # event setup, phase 1 (all lanes): conversion and FP64 dot products
    w("// Event setup, phase 1, run by every lane l of nl lanes of the event: convert the", 0)
    w("// FP64 momenta p (global, [npart][4], rows g g t t~ g..) to R and form the FP64", 0)
    w("// dot products of the outgoing-convention vectors.  The invariants that cancel for", 0)
    w("// soft or collinear gluons are built from these FP64 products.", 0)
    w("template <typename R>", 0)
    w(f"__device__ __forceinline__ void {name}_event_phase1(const double* __restrict__ p, "
      f"{name}_event<R>& ev, int l, int nl) {{", 0)
    w(f"for (int i = l; i < {npart * 4}; i += nl) ev.praw[i] = to_r<R>(__ldg(p + i));")
    w(f"for (int k = l; k < {len(dots)}; k += nl) {{")
    w("int a = 0, b = 0;", 2)
    w("switch (k) {", 2)
    for (i, j), k in didx.items():
        w(f"case {k}: a = {i}; b = {j}; break;", 3)
    w("}", 2)
    w("// vector index -> (row, sign): gluons 0, 1 are incoming (-k), the antitop is row 3", 2)
    w(f"const int ra = a == {n} ? 3 : (a < 2 ? a : a + 2), rb = b == {n} ? 3 : (b < 2 ? b : b + 2);", 2)
    w("const double sa = (a < 2) ? -1.0 : 1.0, sb = (b < 2) ? -1.0 : 1.0;", 2)
    w("const double* x = p + 4 * ra;", 2)
    w("const double* y = p + 4 * rb;", 2)
    w("ev.dd[k] = sa * sb * (__ldg(x) * __ldg(y) - __ldg(x + 1) * __ldg(y + 1) - __ldg(x + 2) * __ldg(y + 2)"
      " - __ldg(x + 3) * __ldg(y + 3));", 2)
    w("}")
    w("}", 0)
    w("", 0)

    # event setup, phase 2
    w("// Event setup, phase 2 (after a barrier): lanes form the FP64 invariants (q^2 also", 0)
    w("// less m02, the square of the launch's reference mass); lane 0 builds the R-typed", 0)
    w("// vectors and the top/antitop spinor bases.", 0)
    w("template <typename R>", 0)
    w(f"__device__ __forceinline__ void {name}_event_phase2({name}_event<R>& ev, double m02, int l, int nl) {{", 0)
    ninv = ngs + nsuf
    w(f"for (int k = l; k < {ninv}; k += nl) {{")
    w("switch (k) {", 2)
    for st, i in gidx.items():
        w(f"case {i}: ev.fg[{i}] = R(-1) / to_r<R>({inv_sq(sorted(st))}); break;", 3)
    for st, i in sidx.items():
        w(f"case {ngs + i}: ev.q2[{i}] = {inv_sq(sorted(st) + [n])}; ev.qm[{i}] = to_r<R>(ev.q2[{i}] - m02); break;", 3)
    w("}", 2)
    w("}")
    w("if (l == 0) {")
    w("#pragma unroll", 0)
    w("for (int m = 0; m < 4; ++m) {", 2)
    w("ev.pg[0][m] = -ev.praw[0 + m];", 3)
    w("ev.pg[1][m] = -ev.praw[4 + m];", 3)
    for g in range(2, n):
        w(f"ev.pg[{g}][m] = ev.praw[{4 * (g + 2)} + m];", 3)
    w("ev.pt[m] = ev.praw[8 + m];", 3)
    w("ev.ptb[m] = ev.praw[12 + m];", 3)
    w("}", 2)
    for st, i in gidx.items():
        terms = " + ".join(f"ev.pg[{g}][m]" for g in sorted(st))
        w("#pragma unroll", 0)
        w(f"for (int m = 0; m < 4; ++m) ev.ps[{i}][m] = {terms};", 2)
    for st, i in sidx.items():
        terms = " + ".join(f"ev.pg[{g}][m]" for g in sorted(st))
        w("#pragma unroll", 0)
        w(f"for (int m = 0; m < 4; ++m) ev.q[{i}][m] = -(ev.ptb[m] + {terms});", 2)
    w("R pabs;", 2)
    w("omegas(ev.pt, R(0), &pabs, &ev.wpt, &ev.iwpt);", 2)
    w("ev.iwpt = R(1) / ev.wpt;", 2)
    w("chi_pair(ev.pt, pabs, ev.cht[1], ev.cht[0]);", 2)
    w("omegas(ev.ptb, R(0), &pabs, &ev.wptb, &ev.iwptb);", 2)
    w("ev.iwptb = R(1) / ev.wptb;", 2)
    w("chi_pair(ev.ptb, pabs, ev.chb[1], ev.chb[0]);", 2)
    w("}")
    w("}", 0)
    w("", 0)

    # mass setup
    w("// Per (event, mass), run by every lane l of nl: inverse propagator denominators,", 0)
    w("// q^2 - m^2 in FP64 in the exact mode; in the mixed mode (R = float) (q^2 - m0^2) +", 0)
    w("// (m0^2 - m^2) in R with dm2 = m0^2 - m^2 from the launch's slot table, so the slot", 0)
    w("// loop issues no FP64 instruction (exact at the reference mass, where dm2 = 0, and", 0)
    w("// free of cancellation elsewhere); lane 0 builds the top spinors.", 0)
    w("template <typename R, bool WIDTH>", 0)
    w(f"__device__ __forceinline__ void {name}_mass_setup(const {name}_event<R>& ev, double mt, double wt, R dm2, "
      f"{name}_mass<R>& mm, int l, int nl) {{", 0)
    w("constexpr bool F32 = std::is_same<R, float>::value;")
    w("const double m2 = mt * mt;")
    w("const R mw = F32 ? to_r<R>(mt) * to_r<R>(wt) : R(mt * wt);")
    w(f"for (int i = l; i < {nsuf}; i += nl) {{")
    w("const R d = F32 ? ev.qm[i] + dm2 : R(ev.q2[i] - m2);", 2)
    w("if (WIDTH) { const R nn = R(1) / (d * d + mw * mw); mm.idr[i] = d * nn; mm.idi[i] = -mw * nn; }", 2)
    w("else { mm.idr[i] = R(1) / d; mm.idi[i] = R(0); }", 2)
    w("}")
    w("if (l == 0) {")
    w("const R mr = to_r<R>(mt);", 2)
    w("mm.m = mr;", 2)
    w("spinor_u_from(ev.cht, ev.wpt, mr * ev.iwpt, mm.ut);", 2)
    w("spinor_v_from(ev.chb, ev.wptb, mr * ev.iwptb, mm.v);", 2)
    w("}")
    w("}", 0)
    w("", 0)

    # gluon currents
    w("// colour-ordered gluon currents for one polarisation configuration (mass independent)", 0)
    w("template <typename R>", 0)
    w(f"__device__ __forceinline__ void {name}_gluon_currents(const {name}_event<R>& ev, "
      f"const R (&eps)[{n}][4], {name}_gluons<R>& J) {{", 0)
    for g in gl:
        w("#pragma unroll", 0)
        w(f"for (int m = 0; m < 4; ++m) J.J{g}[m] = eps[{g}][m];")
    for sq in canon_seqs:
        w(f"{{  // J({','.join(map(str, sq))})")
        w("R t[4] = {R(0), R(0), R(0), R(0)};", 2)
        for i in range(1, len(sq)):
            x, y = sq[:i], sq[i:]
            w(f"vvv_acc(R({_sign(x) * _sign(y)}), J.{_jn(x)}, {pref(x)}, J.{_jn(y)}, {pref(y)}, t);", 2)
        for i in range(1, len(sq)):
            for j in range(i + 1, len(sq)):
                x, y, z = sq[:i], sq[i:j], sq[j:]
                w(f"vvvv_acc(R({_sign(x) * _sign(y) * _sign(z)}), J.{_jn(x)}, J.{_jn(y)}, J.{_jn(z)}, t);", 2)
        w(f"const R f = ev.fg[{gidx[frozenset(sq)]}];", 2)
        w("#pragma unroll", 0)
        w(f"for (int m = 0; m < 4; ++m) J.{_jn(sq)}[m] = f * t[m];", 2)
        w("}")
    w("}", 0)
    w("", 0)

    # quark line with depth-first emission of the antitop-side currents
    nf = len(flows)
    w("// sum over top helicities and antitop helicities hb in [hb_lo, hb_hi) (0: -, 1: +) of", 0)
    w("// sum_{s,s'} conj(A_s) Cint_{ss'} A_s' (Cint = C * COLOUR_DEN).  The antitop-side", 0)
    w("// currents psi(Y) are emitted depth-first over suffixes Y, so only one per depth is live.", 0)
    w("// The colour form of one helicity is evaluated in CS, the helicity sum in ACC.", 0)
    w("// FORM, if given, replaces the scalar colour form: form(A) returns this lane's", 0)
    w("// contribution for both top helicities (e.g. the tensor-core form).", 0)
    w("template <typename R, typename ACC, bool WIDTH, typename CS = ACC, typename FORM = NoColourForm>", 0)
    w(f"__device__ __forceinline__ ACC {name}_quark_line(const {name}_event<R>& ev, const {name}_mass<R>& mm, "
      f"const {name}_gluons<R>& J, int hb_lo = 0, int hb_hi = 2, const FORM& form = FORM()) {{", 0)
    w("ACC total = ACC(0);")
    w("#pragma unroll 1", 0)
    w("for (int hb = hb_lo; hb < hb_hi; ++hb) {")
    w("const cx<R>* v = mm.v[hb];", 2)
    w(f"cx<R> A[2][{nf}];", 2)

    def prop(seq, dst, ind):
        i = sidx[frozenset(seq)]
        w(f"if (WIDTH) fermion_prop(ev.q[{i}], mm.m, cx<R>{{mm.idr[{i}], mm.idi[{i}]}}, t, {dst});", ind)
        w(f"else fermion_prop_real(ev.q[{i}], mm.m, mm.idr[{i}], t, {dst});", ind)

    def emit_psi(seq, ind):
        nm = _psin(seq)
        w(f"cx<R> {nm}[4];", ind)
        w("{", ind)
        w("cx<R> t[4] = {};", ind + 1)
        for i in range(1, len(seq) + 1):
            bl, rest = seq[:i], seq[i:]
            w(f"slash_acc(R({_sign(bl)}), J.{_jn(bl)}, {_psin(rest) if rest else 'v'}, t);", ind + 1)
        prop(seq, nm, ind + 1)
        w("}", ind)

    def emit_flow(f, ind):
        k = fidx[f]
        w(f"{{  // flow {k} = {f}", ind)
        w("cx<R> x[4] = {};", ind + 1)
        for i in range(1, n + 1):
            bl, rest = f[:i], f[i:]
            w(f"slash_acc(R({_sign(bl)}), J.{_jn(bl)}, {_psin(rest) if rest else 'v'}, x);", ind + 1)
        w(f"A[0][{k}] = ubar_dot(mm.ut[0], x);", ind + 1)
        w(f"A[1][{k}] = ubar_dot(mm.ut[1], x);", ind + 1)
        w("}", ind)

    def dfs(suffix, ind):
        for g in gl:
            if g in suffix:
                continue
            new = (g,) + suffix
            if len(new) == n:
                emit_flow(new, ind)
            else:
                w("{", ind)
                emit_psi(new, ind + 1)
                dfs(new, ind + 1)
                w("}", ind)

    dfs((), 2)
    w("if constexpr (!std::is_same<FORM, NoColourForm>::value) {", 2)
    w("total += ACC(form(A));", 3)
    w("} else {", 2)
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
        "//",
        "// Per process: <name>_event (event-level data, filled once per event),",
        "// <name>_mass (per event and mass slot), <name>_gluons (gluon currents of one",
        "// polarisation configuration) and the routines that fill them, then",
        "// <name>_quark_line: jamps and their colour form summed over top helicities.",
        "#pragma once",
        "#include <type_traits>",
        "",
        '#include "../helas.cuh"',
        "",
        "namespace rex {",
        "",
        "// marker: no replacement colour form (use the scalar quadratic form)",
        "struct NoColourForm {};",
        "",
    ]
    for name, n in PROCESSES:
        parts.append(emit_process(name, n))
    parts.append("}  // namespace rex")
    parts.append("")
    return "\n".join(parts)
