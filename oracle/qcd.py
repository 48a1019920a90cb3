"""g g -> t t~ + n g (n = 0, 1, 2) from explicit Feynman diagrams (oracle).

Feynman rules (Peskin & Schroeder Fig. 16.7, Feynman gauge, all gluon momenta
flowing into the vertex):

* quark-gluon vertex          i g gamma^mu t^a
* quark propagator            i (q-slash + m) / (q^2 - m^2 + i m Gamma)
* gluon propagator            -i g_{mu nu} delta^{ab} / q^2
* three-gluon vertex          g f^{abc} [ g^{mu nu}(k-p)^rho + g^{nu rho}(p-q)^mu + g^{rho mu}(q-k)^nu ]
* four-gluon vertex           -i g^2 [ f^{abe}f^{cde}(g^{mu rho}g^{nu sigma} - g^{mu sigma}g^{nu rho})
                                     + f^{ace}f^{bde}(g^{mu nu}g^{rho sigma} - g^{mu sigma}g^{nu rho})
                                     + f^{ade}f^{bce}(g^{mu nu}g^{rho sigma} - g^{mu rho}g^{nu sigma}) ]

Every tree diagram with one open top line and n+2 external gluons is
enumerated: the gluons are split into an ordered sequence of clusters along
the top line (ordered set partitions); every cluster of two or more gluons is
any tree of three- and four-gluon vertices with those leaves.  This gives 3,
16 and 123 diagrams for n = 0, 1, 2.  A diagram containing a four-gluon vertex
splits into three terms, one per colour structure of that vertex.

For each term t the colour factor K_t[a_1..a_{n+2}, i, j] is built as an
explicit tensor from t^a and f^abc; the kinematic part L_t (per event) is
evaluated with explicit 4x4 Dirac matrices.  Then

    sum_colours |M|^2 = sum_{t,t'} conj(L_t) G_{tt'} L_t',   G = conj(K) K^T

is the sum over every colour index, with no colour-flow decomposition.
Averaging: 1/4 for the gluon spins, 1/64 for the gluon colours, 1/k! for k
identical final-state gluons.

Particle order in the momentum array: g(1) g(2) t(3) t~(4) g(5) [g(6)].
Incoming gluons are treated as outgoing with momentum -k and polarisation
eps(k); outgoing gluons carry eps^*(k).
"""
from __future__ import annotations

import functools
import itertools
import math
import string
from dataclasses import dataclass

import numpy as np

from .colour import F, T
from .lorentz import bar, mdot, polarisation, slash, spinor_u, spinor_v


# ----------------------------------------------------------------------------
# diagram enumeration
# ----------------------------------------------------------------------------
@dataclass(frozen=True)
class Leaf:
    g: int


@dataclass(frozen=True)
class Node3:
    x: object
    y: object


@dataclass(frozen=True)
class Node4:
    x: object
    y: object
    z: object
    term: int = -1     # 0, 1, 2 after expansion into colour terms


def leaves(t) -> tuple:
    if isinstance(t, Leaf):
        return (t.g,)
    if isinstance(t, Node3):
        return tuple(sorted(leaves(t.x) + leaves(t.y)))
    return tuple(sorted(leaves(t.x) + leaves(t.y) + leaves(t.z)))


def _unordered_partitions(items: tuple, k: int):
    """All partitions of ``items`` into k non-empty unordered blocks."""
    if k < 1 or len(items) < k:
        return
    if k == 1:
        yield (items,)
        return
    first, rest = items[0], items[1:]
    # first element's block = {first} + subset of rest
    for r in range(0, len(rest) + 1):
        for sub in itertools.combinations(rest, r):
            block = (first,) + sub
            remaining = tuple(x for x in rest if x not in sub)
            for others in _unordered_partitions(remaining, k - 1):
                yield (block,) + others


@functools.lru_cache(maxsize=None)
def gluon_trees(s: tuple) -> tuple:
    """Every tree of 3- and 4-gluon vertices whose leaves are the gluons in ``s``."""
    if len(s) == 1:
        return (Leaf(s[0]),)
    out = []
    for a, b in _unordered_partitions(s, 2):
        for ta in gluon_trees(a):
            for tb in gluon_trees(b):
                out.append(Node3(ta, tb))
    for a, b, c in _unordered_partitions(s, 3):
        for ta in gluon_trees(a):
            for tb in gluon_trees(b):
                for tc in gluon_trees(c):
                    out.append(Node4(ta, tb, tc))
    return tuple(out)


def _ordered_partitions(items: tuple):
    for k in range(1, len(items) + 1):
        for blocks in _unordered_partitions(items, k):
            for perm in itertools.permutations(blocks):
                yield perm


def diagrams(ngluon: int) -> list:
    """All tree diagrams: tuples of cluster trees along the top line (t end first)."""
    out = []
    for blocks in _ordered_partitions(tuple(range(ngluon))):
        for trees in itertools.product(*(gluon_trees(b) for b in blocks)):
            out.append(tuple(trees))
    return out


def _expand(t) -> list:
    """Replace each four-gluon vertex by its three colour terms."""
    if isinstance(t, Leaf):
        return [t]
    if isinstance(t, Node3):
        return [Node3(x, y) for x in _expand(t.x) for y in _expand(t.y)]
    return [Node4(x, y, z, term) for x in _expand(t.x) for y in _expand(t.y)
            for z in _expand(t.z) for term in range(3)]


@functools.lru_cache(maxsize=None)
def diagram_terms(ngluon: int) -> tuple:
    out = []
    for d in diagrams(ngluon):
        for combo in itertools.product(*(_expand(t) for t in d)):
            out.append(tuple(combo))
    return tuple(out)


# ----------------------------------------------------------------------------
# colour factors as explicit tensors
# ----------------------------------------------------------------------------
_DELTA8 = np.eye(8)


def _einsum_labelled(ops, out_labels):
    """einsum over (array, labels) pairs with arbitrary hashable labels."""
    letters = {}
    pool = iter(string.ascii_letters)

    def let(lbl):
        if lbl not in letters:
            letters[lbl] = next(pool)
        return letters[lbl]

    subs = []
    arrays = []
    for arr, labels in ops:
        subs.append("".join(let(l) for l in labels))
        arrays.append(arr)
    spec = ",".join(subs) + "->" + "".join(let(l) for l in out_labels)
    return np.einsum(spec, *arrays, optimize=True)


def _tree_colour(t, root):
    """(tensor, labels): colour factor of a gluon tree with free adjoint index ``root``."""
    if isinstance(t, Leaf):
        return _DELTA8, [("g", t.g), root]
    if isinstance(t, Node3):
        rx, ry = ("int", id(t), "x"), ("int", id(t), "y")
        cx, lx = _tree_colour(t.x, rx)
        cy, ly = _tree_colour(t.y, ry)
        out = [l for l in lx if l != rx] + [l for l in ly if l != ry] + [root]
        return _einsum_labelled([(cx, lx), (cy, ly), (F, [rx, ry, root])], out), out
    rx, ry, rz, q = (("int", id(t), s) for s in "xyzq")
    cx, lx = _tree_colour(t.x, rx)
    cy, ly = _tree_colour(t.y, ry)
    cz, lz = _tree_colour(t.z, rz)
    if t.term == 0:      # f^{x y q} f^{z e q}
        ff = [(F, [rx, ry, q]), (F, [rz, root, q])]
    elif t.term == 1:    # f^{x z q} f^{y e q}
        ff = [(F, [rx, rz, q]), (F, [ry, root, q])]
    else:                # f^{x e q} f^{y z q}
        ff = [(F, [rx, root, q]), (F, [ry, rz, q])]
    out = ([l for l in lx if l != rx] + [l for l in ly if l != ry]
           + [l for l in lz if l != rz] + [root])
    return _einsum_labelled([(cx, lx), (cy, ly), (cz, lz)] + ff, out), out


def term_colour(term: tuple, ngluon: int) -> np.ndarray:
    """K[a_1..a_n, i, j]: colour factor of a diagram term (t end = row index i)."""
    ops = []
    for k, tree in enumerate(term):
        root = ("root", k)
        c, lab = _tree_colour(tree, root)
        ops.append((c, lab))
        ops.append((T, [root, ("q", k), ("q", k + 1)]))
    out = [("g", g) for g in range(ngluon)] + [("q", 0), ("q", len(term))]
    return _einsum_labelled(ops, out)


@functools.lru_cache(maxsize=None)
def colour_matrix(ngluon: int) -> np.ndarray:
    """G_{tt'} = sum over all colour indices of conj(K_t) K_t'."""
    terms = diagram_terms(ngluon)
    k = np.stack([term_colour(t, ngluon).reshape(-1) for t in terms])
    return k.conj() @ k.T


# ----------------------------------------------------------------------------
# kinematic part
# ----------------------------------------------------------------------------
class _Kinematics:
    def __init__(self, p_out, eps, g):
        self.p_out = p_out          # list of [N,4] outgoing-convention gluon momenta
        self.eps = eps              # list of [N,4] complex polarisations
        self.g = g
        self.cache = {}

    def current(self, t):
        """(J, P): off-shell current (propagator included) and its outgoing momentum."""
        key = t
        if key in self.cache:
            return self.cache[key]
        g = self.g
        if isinstance(t, Leaf):
            res = (self.eps[t.g], self.p_out[t.g])
        elif isinstance(t, Node3):
            jx, px = self.current(t.x)
            jy, py = self.current(t.y)
            kx, ky, ke = -px, -py, px + py          # incoming momenta at the vertex
            vert = g * (mdot(jx, jy)[:, None] * (kx - ky)
                        + mdot(jx, ky - ke)[:, None] * jy
                        + mdot(jy, ke - kx)[:, None] * jx)
            p = px + py
            res = ((-1j / mdot(p, p))[:, None] * vert, p)
        else:
            jx, px = self.current(t.x)
            jy, py = self.current(t.y)
            jz, pz = self.current(t.z)
            if t.term == 0:
                lor = mdot(jx, jz)[:, None] * jy - mdot(jy, jz)[:, None] * jx
            elif t.term == 1:
                lor = mdot(jx, jy)[:, None] * jz - mdot(jy, jz)[:, None] * jx
            else:
                lor = mdot(jx, jy)[:, None] * jz - mdot(jx, jz)[:, None] * jy
            p = px + py + pz
            res = ((-1j * g * g) * (-1j / mdot(p, p))[:, None] * lor, p)
        self.cache[key] = res
        return res


def _matvec(m, v):
    return np.einsum("nij,nj->ni", m, v)


def _line_amplitude(term, kin, ubar_t, v_tb, p_t, mt, wt):
    """ubar(t) (i g J1-slash) S(q1) (i g J2-slash) ... (i g Jm-slash) v(t~)."""
    g = kin.g
    cur = [kin.current(tr) for tr in term]
    qs = []
    q = p_t.copy()
    for k in range(len(term) - 1):
        q = q + cur[k][1]
        qs.append(q)
    psi = v_tb
    for k in range(len(term) - 1, -1, -1):
        psi = 1j * g * _matvec(slash(cur[k][0]), psi)
        if k > 0:
            qk = qs[k - 1]
            den = mdot(qk, qk) - mt * mt + 1j * mt * wt
            num = slash(qk) + mt * np.eye(4)
            psi = (1j / den)[:, None] * _matvec(num, psi)
    return np.einsum("ni,ni->n", ubar_t, psi)


def _real(p) -> np.ndarray:
    """Momenta as a real array: FP64, unless they are given in extended precision
    (np.longdouble), which is then kept through every step.  The extended path only
    measures the FP64 evaluation's own rounding error (pins of the condition estimate)."""
    p = np.asarray(p)
    return p if p.dtype == np.longdouble else p.astype(np.float64)


def me2_helicity(p: np.ndarray, mt: float, wt: float, alphas: float,
                 hel_g: tuple, lt: int, ltb: int) -> np.ndarray:
    """Colour-summed |M|^2 (not averaged) for one physical helicity configuration.

    hel_g: helicities of the gluons in row order (g1, g2, g5, ...); lt, ltb:
    helicities of the outgoing top and antitop.
    """
    p = _real(p)
    npart = p.shape[1]
    ngl = npart - 2
    g = math.sqrt(4.0 * math.pi * alphas)
    terms = diagram_terms(ngl)
    gmat = colour_matrix(ngl)
    gl_rows = [0, 1] + list(range(4, npart))
    p_out = [-p[:, 0], -p[:, 1]] + [p[:, r] for r in range(4, npart)]
    eps = []
    for k, (row, lam) in enumerate(zip(gl_rows, hel_g)):
        e = polarisation(p[:, row], lam)
        eps.append(e if k < 2 else e.conj())
    kin = _Kinematics(p_out, eps, g)
    ubar_t = bar(spinor_u(p[:, 2], mt, lt))
    v_tb = spinor_v(p[:, 3], mt, ltb)
    amps = np.stack([_line_amplitude(t, kin, ubar_t, v_tb, p[:, 2], mt, wt)
                     for t in terms], axis=1)
    return np.real(np.einsum("ns,st,nt->n", amps.conj(), gmat, amps))


def me2_helicity_per_event(p: np.ndarray, mt: float, wt: float, alphas: float, hel: np.ndarray) -> np.ndarray:
    """Each event's own helicity term of me2, averaged as me2 is (so that the sum over
    every configuration gives me2): hel[N, npart] in particle order g g t t~ g.., +1 / -1
    (a positive entry reads as +1).  Events are grouped by configuration and each group
    evaluated with me2_helicity."""
    p = _real(p)
    hel = np.where(np.asarray(hel) > 0, 1, -1)
    nev, npart, _ = p.shape
    ngl = npart - 2
    gl_rows = [0, 1] + list(range(4, npart))
    out = np.zeros(nev, dtype=p.dtype)
    configs, inverse = np.unique(hel, axis=0, return_inverse=True)
    for c, h in enumerate(configs):
        idx = np.nonzero(inverse.reshape(-1) == c)[0]
        out[idx] = me2_helicity(p[idx], mt, wt, alphas, tuple(int(h[r]) for r in gl_rows), int(h[2]), int(h[3]))
    return out / (4.0 * 64.0 * math.factorial(ngl - 2))


def me2(p: np.ndarray, mt: float, wt: float, alphas: float) -> np.ndarray:
    """Spin/colour summed and averaged |M|^2 for g g -> t t~ + n g, one point.

    p: [N, 4+n, 4] physical momenta (E, px, py, pz); rows g g t t~ g...
    """
    p = _real(p)
    nev, npart, _ = p.shape
    ngl = npart - 2
    nfinal_g = ngl - 2
    g = math.sqrt(4.0 * math.pi * alphas)
    terms = diagram_terms(ngl)
    gmat = colour_matrix(ngl)
    gl_rows = [0, 1] + list(range(4, npart))
    p_out = [-p[:, 0], -p[:, 1]] + [p[:, r] for r in range(4, npart)]
    p_t, p_tb = p[:, 2], p[:, 3]
    total = np.zeros(nev, dtype=p.dtype)
    for hel_g in itertools.product((-1, 1), repeat=ngl):
        eps = []
        for k, (row, lam) in enumerate(zip(gl_rows, hel_g)):
            e = polarisation(p[:, row], lam)
            eps.append(e if k < 2 else e.conj())
        kin = _Kinematics(p_out, eps, g)
        for lt in (-1, 1):
            ubar_t = bar(spinor_u(p_t, mt, lt))
            for ltb in (-1, 1):
                v_tb = spinor_v(p_tb, mt, ltb)
                amps = np.stack([_line_amplitude(t, kin, ubar_t, v_tb, p_t, mt, wt)
                                 for t in terms], axis=1)      # [N, terms]
                total += np.real(np.einsum("ns,st,nt->n", amps.conj(), gmat, amps))
    avg = 1.0 / (4.0 * 64.0 * math.factorial(nfinal_g))
    return total * avg


def gauge_check(p: np.ndarray, mt: float, which: int, hel_g: tuple, lt: int, ltb: int,
                alphas: float = 0.118) -> tuple[float, float]:
    """Colour-summed |M|^2 with gluon ``which``'s polarisation replaced by its momentum,
    and the same with the physical polarisation, for one helicity configuration.

    Returns (sum over events of the gauge-replaced value, sum of the physical one).
    """
    p = _real(p)
    npart = p.shape[1]
    ngl = npart - 2
    g = math.sqrt(4.0 * math.pi * alphas)
    terms = diagram_terms(ngl)
    gmat = colour_matrix(ngl)
    gl_rows = [0, 1] + list(range(4, npart))
    p_out = [-p[:, 0], -p[:, 1]] + [p[:, r] for r in range(4, npart)]
    p_t, p_tb = p[:, 2], p[:, 3]
    res = []
    for replace in (True, False):
        eps = []
        for k, (row, lam) in enumerate(zip(gl_rows, hel_g)):
            e = polarisation(p[:, row], lam)
            e = e if k < 2 else e.conj()
            if replace and k == which:
                e = p[:, row].astype(complex)
            eps.append(e)
        kin = _Kinematics(p_out, eps, g)
        ubar_t = bar(spinor_u(p_t, mt, lt))
        v_tb = spinor_v(p_tb, mt, ltb)
        amps = np.stack([_line_amplitude(t, kin, ubar_t, v_tb, p_t, mt, wt=0.0)
                         for t in terms], axis=1)
        res.append(np.real(np.einsum("ns,st,nt->n", amps.conj(), gmat, amps)))
    return res[0], res[1]


def condition(p: np.ndarray, mt: float, wt: float, alphas: float) -> np.ndarray:
    """Condition estimate of me2: kappa = sum_h sum_st |Re(A_s* G_st A_t)| / |M|^2 over
    every helicity configuration h and every pair (s, t) of diagram terms, the same
    terms me2 adds.  kappa >= 1; a result whose terms cancel has kappa >> 1, and a
    relative rounding error up to ~ eps * kappa is then expected of any evaluation
    order (a diagnostic for the tolerance rule, not a physical quantity)."""
    p = _real(p)
    nev, npart, _ = p.shape
    ngl = npart - 2
    g = math.sqrt(4.0 * math.pi * alphas)
    terms = diagram_terms(ngl)
    gmat = colour_matrix(ngl)
    gl_rows = [0, 1] + list(range(4, npart))
    p_out = [-p[:, 0], -p[:, 1]] + [p[:, r] for r in range(4, npart)]
    p_t, p_tb = p[:, 2], p[:, 3]
    total = np.zeros(nev, dtype=p.dtype)
    absum = np.zeros(nev, dtype=p.dtype)
    for hel_g in itertools.product((-1, 1), repeat=ngl):
        eps = []
        for k, (row, lam) in enumerate(zip(gl_rows, hel_g)):
            e = polarisation(p[:, row], lam)
            eps.append(e if k < 2 else e.conj())
        kin = _Kinematics(p_out, eps, g)
        for lt in (-1, 1):
            ubar_t = bar(spinor_u(p_t, mt, lt))
            for ltb in (-1, 1):
                v_tb = spinor_v(p_tb, mt, ltb)
                amps = np.stack([_line_amplitude(t, kin, ubar_t, v_tb, p_t, mt, wt)
                                 for t in terms], axis=1)
                pair = np.real(amps.conj()[:, :, None] * gmat[None, :, :] * amps[:, None, :])
                total += pair.sum(axis=(1, 2))
                absum += np.abs(pair).sum(axis=(1, 2))
    return absum / np.abs(total)
