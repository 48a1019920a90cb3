"""Independent physics results used to pin the oracle (no oracle code used here).

* e+e- -> mu+mu- via photon + Z: textbook helicity amplitudes for massless
  fermions (Peskin & Schroeder Sec. 5.2; the Z adds a chiral coupling and a
  Breit-Wigner propagator).
* g g -> Q Q~ and q q~ -> Q Q~: the Combridge (1979) formulas as printed in
  Ellis, Stirling & Webber, "QCD and collider physics", Ch. 10 (spin and colour
  averaged); for q q~ -> Q Q~ also the trace form of the same result, which
  holds for any on-shell heavy-quark momenta (momentum conservation unused).
* g g -> q q~ + n g, massless: colour-ordered Parke-Taylor amplitudes in the
  spinor-helicity formalism (Mangano & Parke, Phys. Rept. 200 (1991) 301;
  Dixon, TASI 1995 lectures, hep-ph/9601359) with the colour decomposition
  into ordered products of generators, summed over colours with a colour
  matrix computed here from its own Gell-Mann matrices.
"""
from __future__ import annotations

import itertools
import math

import numpy as np


def mdot(a, b):
    return a[..., 0] * b[..., 0] - (a[..., 1:] * b[..., 1:]).sum(-1)


# ----------------------------------------------------------------------------
# e+ e- -> mu+ mu-
# ----------------------------------------------------------------------------
def ee_mumu_closed_form(p, mz, wz, sw2, alpha):
    """(e^4/4) sum_{l,l'} |Q^2 + g_l g_l' s/(sW^2 cW^2 (s - mZ^2 + i mZ GZ))|^2 (1 + eta cos)^2."""
    e2 = 4.0 * math.pi * alpha
    cw2 = 1.0 - sw2
    gl, gr = -0.5 + sw2, sw2
    s = mdot(p[:, 0] + p[:, 1], p[:, 0] + p[:, 1])
    n_e = p[:, 1, 1:] / np.linalg.norm(p[:, 1, 1:], axis=1)[:, None]
    n_mu = p[:, 3, 1:] / np.linalg.norm(p[:, 3, 1:], axis=1)[:, None]
    c = (n_e * n_mu).sum(1)
    prop = s / (s - mz * mz + 1j * mz * wz)
    tot = 0.0
    for i, ge in enumerate((gl, gr)):
        for j, gm in enumerate((gl, gr)):
            eta = 1.0 if i == j else -1.0
            tot = tot + np.abs(1.0 + ge * gm / (sw2 * cw2) * prop) ** 2 * (1.0 + eta * c) ** 2
    return e2 * e2 / 4.0 * tot


def ee_mumu_helicity_closed_form(p, hel, mz, wz, sw2, alpha):
    """One helicity configuration (l1, l2, l3, l4) of e+ e- mu+ mu-, with the same 1/4:
    (e^4/4) |Q^2 + g_X g_Y s/(sW^2 cW^2 (s - mZ^2 + i mZ GZ))|^2 (1 + eta cos)^2, X (Y) the
    chirality of the e- (mu-): L for helicity -1; eta = +1 if X == Y; 0 unless the e+ and
    the mu+ have the helicities opposite to the e- and the mu-."""
    e2 = 4.0 * math.pi * alpha
    cw2 = 1.0 - sw2
    g = {-1: -0.5 + sw2, 1: sw2}
    s = mdot(p[:, 0] + p[:, 1], p[:, 0] + p[:, 1])
    n_e = p[:, 1, 1:] / np.linalg.norm(p[:, 1, 1:], axis=1)[:, None]
    n_mu = p[:, 3, 1:] / np.linalg.norm(p[:, 3, 1:], axis=1)[:, None]
    c = (n_e * n_mu).sum(1)
    prop = s / (s - mz * mz + 1j * mz * wz)
    out = np.zeros(p.shape[0])
    for i, (l1, l2, l3, l4) in enumerate(hel):
        if l1 != -l2 or l3 != -l4:
            continue
        eta = 1.0 if l2 == l4 else -1.0
        out[i] = e2 * e2 / 4.0 * abs(1.0 + g[l2] * g[l4] / (sw2 * cw2) * prop[i]) ** 2 * (1.0 + eta * c[i]) ** 2
    return out


def qq_qq_helicity_cm(p, hel, m, alphas):
    """q q~ -> Q Q~ per helicity configuration (l1, l2, l3, l4) in the centre-of-mass frame,
    spin average 1/4 and colour included: g_s^4/18 (1 + l1 l3 cos)^2 when l3 = -l4 and
    g_s^4/18 (1 - beta^2) sin^2 when l3 = l4; 0 unless l2 = -l1 (massless q, q~).  cos is
    the angle between q and Q, beta the velocity of Q.  The 16 terms add up to the
    Combridge form."""
    gs2 = 4.0 * math.pi * alphas
    nq = p[:, 0, 1:] / np.linalg.norm(p[:, 0, 1:], axis=1)[:, None]
    pq = np.linalg.norm(p[:, 2, 1:], axis=1)
    nQ = p[:, 2, 1:] / pq[:, None]
    c = (nq * nQ).sum(1)
    beta2 = (pq / p[:, 2, 0]) ** 2
    out = np.zeros(p.shape[0])
    for i, (l1, l2, l3, l4) in enumerate(hel):
        if l2 != -l1:
            continue
        if l3 == -l4:
            out[i] = gs2 * gs2 / 18.0 * (1.0 + l1 * l3 * c[i]) ** 2
        else:
            out[i] = gs2 * gs2 / 18.0 * (1.0 - beta2[i]) * (1.0 - c[i] * c[i])
    return out


def qed_limit_closed_form(p, alpha):
    """e^4 (1 + cos^2 theta): pure photon exchange (Peskin & Schroeder eq. 5.10)."""
    e2 = 4.0 * math.pi * alpha
    n_e = p[:, 1, 1:] / np.linalg.norm(p[:, 1, 1:], axis=1)[:, None]
    n_mu = p[:, 3, 1:] / np.linalg.norm(p[:, 3, 1:], axis=1)[:, None]
    c = (n_e * n_mu).sum(1)
    return e2 * e2 * (1.0 + c * c)


# ----------------------------------------------------------------------------
# g g -> Q Q~ (Combridge)
# ----------------------------------------------------------------------------
def gg_qq_combridge(p, m, alphas):
    """g_s^4 (1/(6 t1 t2) - 3/8)(t1^2 + t2^2 + rho - rho^2/(4 t1 t2)), t_i = 2 k_i.p_Q / s."""
    gs2 = 4.0 * math.pi * alphas
    k1, k2, pq = p[:, 0], p[:, 1], p[:, 2]
    s = mdot(k1 + k2, k1 + k2)
    t1 = 2.0 * mdot(k1, pq) / s
    t2 = 2.0 * mdot(k2, pq) / s
    rho = 4.0 * m * m / s
    return gs2 * gs2 * (1.0 / (6.0 * t1 * t2) - 3.0 / 8.0) * (t1 * t1 + t2 * t2 + rho
                                                              - rho * rho / (4.0 * t1 * t2))


def qq_qq_combridge(p, m, alphas):
    """q q~ -> Q Q~: g_s^4 (4/9)(t1^2 + t2^2 + rho/2), t_i = 2 k_i.p_Q / s, rho = 4 m^2 / s."""
    gs2 = 4.0 * math.pi * alphas
    k1, k2, pq = p[:, 0], p[:, 1], p[:, 2]
    s = mdot(k1 + k2, k1 + k2)
    t1 = 2.0 * mdot(k1, pq) / s
    t2 = 2.0 * mdot(k2, pq) / s
    return gs2 * gs2 * 4.0 / 9.0 * (t1 * t1 + t2 * t2 + 2.0 * m * m / s)


def qq_qq_trace(k1, k2, pq, pqb, m, alphas):
    """The same |M|^2 from the Dirac traces, (1/36) g^4 * 2 * 32 [(k1.pq)(k2.pqb) +
    (k1.pqb)(k2.pq) + m^2 k1.k2] / s^2, for massless k1, k2 and any pq, pqb of mass m."""
    gs2 = 4.0 * math.pi * alphas
    s = mdot(k1 + k2, k1 + k2)
    tr = 32.0 * (mdot(k1, pq) * mdot(k2, pqb) + mdot(k1, pqb) * mdot(k2, pq) + m * m * mdot(k1, k2))
    return gs2 * gs2 * 2.0 * tr / (36.0 * s * s)


def light_cone_mass_shift(p, m):
    """The momentum of mass m with the direction and the light-cone component E + |p| of p:
    E' + |p'| = E + |p|, E' - |p'| = m^2 / (E + |p|)."""
    a = np.linalg.norm(p[..., 1:], axis=-1)
    plus = p[..., 0] + a
    minus = m * m / plus
    out = np.empty_like(p)
    out[..., 0] = 0.5 * (plus + minus)
    out[..., 1:] = p[..., 1:] * (0.5 * (plus - minus) / a)[..., None]
    return out


# ----------------------------------------------------------------------------
# spinor helicity, Parke-Taylor
# ----------------------------------------------------------------------------
def _lam(k):
    """Holomorphic and anti-holomorphic spinors of a massless momentum (needs k^+ > 0).

    Negative-energy momenta (crossed incoming particles) use lambda(-k) times i;
    the constant phase is common to all colour orderings and drops out of
    the colour-summed |M|^2.
    """
    neg = k[..., 0] < 0
    kk = np.where(neg[..., None], -k, k)
    kp = kk[..., 0] + kk[..., 3]
    sq = np.sqrt(kp)
    lam = np.stack([sq + 0j, (kk[..., 1] + 1j * kk[..., 2]) / sq], axis=-1)
    lamt = np.stack([sq + 0j, (kk[..., 1] - 1j * kk[..., 2]) / sq], axis=-1)
    ph = np.where(neg, 1j, 1.0)
    return lam * ph[..., None], lamt * ph[..., None]


def _angle(li, lj):
    return li[..., 0] * lj[..., 1] - li[..., 1] * lj[..., 0]


def _t_matrices():
    """Generators t^a = lambda^a/2 built from the su(3) basis (own construction)."""
    t = []
    for (i, j) in ((0, 1), (0, 2), (1, 2)):
        s = np.zeros((3, 3), complex)
        s[i, j] = s[j, i] = 0.5
        a = np.zeros((3, 3), complex)
        a[i, j] = -0.5j
        a[j, i] = 0.5j
        t += [s, a]
    d3 = np.diag([0.5, -0.5, 0.0]).astype(complex)
    d8 = np.diag([1.0, 1.0, -2.0]).astype(complex) / (2.0 * math.sqrt(3.0))
    return np.array(t + [d3, d8])


def flow_colour_matrix(ngl):
    """C_{s,s'} = sum_colours conj((t^s1..t^sn)_{ij}) (t^s'1..t^s'n)_{ij} over orderings s."""
    t = _t_matrices()
    perms = list(itertools.permutations(range(ngl)))
    words = []
    for perm in perms:
        # tensor over (a_1..a_n, i, j) of the ordered product t^{a_perm0} ... t^{a_perm(n-1)}
        idx = [chr(ord("a") + g) for g in range(ngl)]
        chain = ",".join(f"{idx[g]}{chr(ord('p') + k)}{chr(ord('p') + k + 1)}"
                         for k, g in enumerate(perm))
        out = "".join(idx) + "p" + chr(ord("p") + ngl)
        words.append(np.einsum(chain + "->" + out, *([t] * ngl)).reshape(-1))
    w = np.array(words)
    return perms, (w.conj() @ w.T).real


def parke_taylor_helicity(p, alphas, q_hel, qb_hel, gl_hel_out):
    """Colour-summed |A|^2 (not averaged) for one all-outgoing helicity configuration.

    p: [N, 4+n, 4] rows g g q q~ g...; gl_hel_out: outgoing-convention helicities
    of the gluons in row order (an incoming gluon of helicity h is an outgoing
    one of helicity -h).  Returns None when the configuration is neither MHV
    nor anti-MHV (no Parke-Taylor formula); vanishing configurations give 0.
    """
    nev, npart, _ = p.shape
    ngl = npart - 2
    if q_hel == qb_hel:
        return np.zeros(nev)          # helicity conserved along a massless quark line
    nneg = sum(1 for h in gl_hel_out if h < 0)
    if nneg in (0, ngl):
        return np.zeros(nev)
    if nneg == 1:
        pick, special = 0, list(gl_hel_out).index(-1)   # MHV: angle brackets
    elif nneg == ngl - 1:
        pick, special = 1, list(gl_hel_out).index(1)    # anti-MHV: square brackets
    else:
        return None
    out_mom = [-p[:, 0], -p[:, 1]] + [p[:, r] for r in range(4, npart)]
    lq, lqb = _lam(p[:, 2]), _lam(p[:, 3])
    lg = [_lam(k) for k in out_mom]
    br = lambda a, b: _angle(a[pick], b[pick])
    li = lg[special]
    # MHV: A(qbar-, q+, .., i-, ..) ~ <qbar i>^3 <q i>;  A(qbar+, q-, ..) ~ <q i>^3 <qbar i>.
    # anti-MHV is the parity conjugate (angle -> square, all helicities flipped).
    qbar_minus_mhv = (qb_hel < 0) if pick == 0 else (qb_hel > 0)
    if qbar_minus_mhv:
        num = br(lqb, li) ** 3 * br(lq, li)
    else:
        num = br(lq, li) ** 3 * br(lqb, li)
    perms, cmat = flow_colour_matrix(ngl)
    amps = []
    for perm in perms:
        chain = [lqb, lq] + [lg[g] for g in perm]
        den = np.ones(nev, complex)
        for k in range(len(chain)):
            den = den * br(chain[k], chain[(k + 1) % len(chain)])
        amps.append(1j * num / den)
    a = np.stack(amps, axis=1)
    gs2 = 4.0 * math.pi * alphas
    # T^a = sqrt(2) t^a in the colour decomposition: a factor 2 per generator in |M|^2
    return np.real(np.einsum("ns,st,nt->n", a.conj(), cmat, a)) * gs2 ** ngl * 2.0 ** ngl


def parke_taylor_me2(p, alphas):
    """Colour-summed, averaged |M|^2 of g g -> q q~ + n g (n <= 1), massless quarks."""
    nev, npart, _ = p.shape
    ngl = npart - 2
    assert ngl <= 3, "beyond five partons not every helicity amplitude is MHV"
    total = np.zeros(nev)
    for gh in itertools.product((-1, 1), repeat=ngl):
        for qh in (-1, 1):
            v = parke_taylor_helicity(p, alphas, qh, -qh, gh)
            total += v
    avg = 1.0 / (4.0 * 64.0 * math.factorial(ngl - 2))
    return total * avg


def random_rotation(seed):
    g = np.random.default_rng(seed)
    q, r = np.linalg.qr(g.normal(size=(3, 3)))
    q = q * np.sign(np.diag(r))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q


def rotate(p, rot):
    out = p.copy()
    out[..., 1:] = p[..., 1:] @ rot.T
    return out


def boost(p, beta):
    b = np.asarray(beta, dtype=np.float64)
    b2 = b @ b
    gam = 1.0 / math.sqrt(1.0 - b2)
    bp = p[..., 1:] @ b
    out = p.copy()
    out[..., 0] = gam * (p[..., 0] + bp)
    out[..., 1:] = p[..., 1:] + ((gam - 1.0) * bp / b2)[..., None] * b + (gam * p[..., 0])[..., None] * b
    return out


# ----------------------------------------------------------------------------
# soft-gluon limit of q q~ -> Q Q~ g
# ----------------------------------------------------------------------------
def qq_qq_colour_correlators():
    """C_ij = <B| T_i . T_j |B> / <B|B> for the Born colour tensor
    B[i1, j2, i3, j4] = sum_b (t^b)_{j2 i1} (t^b)_{i3 j4} of q(1) q~(2) -> Q(3) Q~(4).
    Insertions: an outgoing quark's index takes t^c from the left, an outgoing
    antiquark's -t^c from the right; an incoming quark counts as an outgoing
    antiquark and an incoming antiquark as an outgoing quark.  Returns C [4, 4] and
    the colour-conservation residual max |sum_i T_i B|."""
    t = _t_matrices()
    born = np.einsum("bji,bkl->ijkl", t, t)
    ins = [
        lambda c: -np.einsum("xi,xjkl->ijkl", t[c], born),   # q in: index i1
        lambda c: np.einsum("jx,ixkl->ijkl", t[c], born),    # q~ in: index j2
        lambda c: np.einsum("kx,ijxl->ijkl", t[c], born),    # Q out: index i3
        lambda c: -np.einsum("xl,ijkx->ijkl", t[c], born),   # Q~ out: index j4
    ]
    norm = np.real(np.sum(born.conj() * born))
    corr = np.zeros((4, 4))
    resid = 0.0
    for c in range(8):
        tb = [f(c) for f in ins]
        resid = max(resid, float(np.max(np.abs(sum(tb)))))
        for i in range(4):
            for j in range(4):
                corr[i, j] += np.real(np.sum(tb[i].conj() * tb[j])) / norm
    return corr, resid


def soft_eikonal(p, k, corr, alphas):
    """-g^2 sum_{i,j} C_ij (p_i.p_j) / ((p_i.k)(p_j.k)) over the four hard legs (physical
    momenta; the sign flips of incoming legs cancel in each term)."""
    gs2 = 4.0 * math.pi * alphas
    tot = 0.0
    for i in range(4):
        for j in range(4):
            tot = tot + corr[i, j] * mdot(p[:, i], p[:, j]) / (mdot(p[:, i], k) * mdot(p[:, j], k))
    return -gs2 * tot


def soft_qq_ttg_events(n, seed, m, sqrt_s, omega_frac):
    """q q~ -> Q Q~ g with a soft gluon of energy omega_frac * sqrt(s), exact momentum
    conservation and on-shell Q: the Q Q~ pair recoils against the gluon and decays at
    seeded angles in its rest frame.  Returns (events [n, 5, 4], Born events [n, 4, 4]
    with the same angles at omega = 0)."""
    rng = np.random.default_rng(seed)
    e = sqrt_s / 2.0
    p1 = np.array([e, 0.0, 0.0, e])
    p2 = np.array([e, 0.0, 0.0, -e])
    out, born = [], []
    for _ in range(n):
        ck, phk = rng.uniform(-0.9, 0.9), rng.uniform(0, 2 * math.pi)
        nk = np.array([math.sqrt(1 - ck * ck) * math.cos(phk), math.sqrt(1 - ck * ck) * math.sin(phk), ck])
        ct, pht = rng.uniform(-0.9, 0.9), rng.uniform(0, 2 * math.pi)
        nt = np.array([math.sqrt(1 - ct * ct) * math.cos(pht), math.sqrt(1 - ct * ct) * math.sin(pht), ct])
        rows = []
        for om in (omega_frac * sqrt_s, 0.0):
            k = np.concatenate([[om], om * nk])
            pp = np.concatenate([[sqrt_s - om], -om * nk])
            mm = math.sqrt(pp[0] ** 2 - pp[1:] @ pp[1:])
            q = math.sqrt(mm * mm / 4.0 - m * m)
            t_rest = np.concatenate([[mm / 2.0], q * nt])
            tb_rest = np.concatenate([[mm / 2.0], -q * nt])
            beta = pp[1:] / pp[0]
            if om > 0.0:
                t_lab = boost(t_rest[None], beta)[0]
                tb_lab = boost(tb_rest[None], beta)[0]
            else:
                t_lab, tb_lab = t_rest, tb_rest
            rows.append((k, t_lab, tb_lab))
        (k, t_lab, tb_lab), (_, t0, tb0) = rows
        out.append([p1, p2, t_lab, tb_lab, k])
        born.append([p1, p2, t0, tb0])
    return np.array(out), np.array(born)


# ----------------------------------------------------------------------------
# initial-state collinear limit of q g -> Q Q~ q (g -> q q~ splitting)
# ----------------------------------------------------------------------------
def collinear_initial_events(n, seed, m, sqrt_s, x, theta):
    """a(pa) g(pb) -> Q Q~ c(pc) in the centre-of-mass frame, pa along +z, pb along -z,
    the outgoing light parton c of energy (1 - x) E_b at angle theta to pb (seeded
    azimuth), the Q Q~ pair recoiling and decaying at seeded angles in its rest frame.
    Returns events [n, 5, 4] in the order (pa, pb, Q, Q~, pc)."""
    rng = np.random.default_rng(seed)
    e = sqrt_s / 2.0
    pa = np.array([e, 0.0, 0.0, e])
    pb = np.array([e, 0.0, 0.0, -e])
    out = []
    for _ in range(n):
        phi = rng.uniform(0, 2 * math.pi)
        ec = (1.0 - x) * e
        pc = ec * np.array([1.0, math.sin(theta) * math.cos(phi), math.sin(theta) * math.sin(phi), -math.cos(theta)])
        qq = pa + pb - pc
        mm = math.sqrt(qq[0] ** 2 - qq[1:] @ qq[1:])
        q = math.sqrt(mm * mm / 4.0 - m * m)
        ct, pht = rng.uniform(-0.9, 0.9), rng.uniform(0, 2 * math.pi)
        nt = np.array([math.sqrt(1 - ct * ct) * math.cos(pht), math.sqrt(1 - ct * ct) * math.sin(pht), ct])
        t_rest = np.concatenate([[mm / 2.0], q * nt])
        tb_rest = np.concatenate([[mm / 2.0], -q * nt])
        beta = qq[1:] / qq[0]
        out.append([pa, pb, boost(t_rest[None], beta)[0], boost(tb_rest[None], beta)[0], pc])
    return np.array(out)


def splitting_g_to_qq(x):
    """The spin- and colour-averaged g -> q q~ splitting function T_R (x^2 + (1 - x)^2),
    T_R = 1/2 (Altarelli & Parisi, Nucl. Phys. B126 (1977) 298)."""
    return 0.5 * (x * x + (1.0 - x) ** 2)


def forward_quark_events(nphi, seed, m, sqrt_s, x, theta):
    """q(pa) g(pb) -> Q Q~ q(pc) with the outgoing quark of energy (1 - x) E_a at angle
    theta to pa (along +z), at nphi equally spaced azimuths around pa (which averages
    out the cos(2 phi) spin correlation of a gluon entering the hard process); the Q Q~
    pair recoils and decays at one seeded rest-frame direction for all azimuths.
    Returns events [nphi, 5, 4] in the order (pa, pb, Q, Q~, pc)."""
    rng = np.random.default_rng(seed)
    e = sqrt_s / 2.0
    pa = np.array([e, 0.0, 0.0, e])
    pb = np.array([e, 0.0, 0.0, -e])
    ct, pht = rng.uniform(-0.9, 0.9), rng.uniform(0, 2 * math.pi)
    nt = np.array([math.sqrt(1 - ct * ct) * math.cos(pht), math.sqrt(1 - ct * ct) * math.sin(pht), ct])
    out = []
    for k in range(nphi):
        phi = 2.0 * math.pi * k / nphi + 0.3
        ec = (1.0 - x) * e
        pc = ec * np.array([1.0, math.sin(theta) * math.cos(phi), math.sin(theta) * math.sin(phi), math.cos(theta)])
        qq = pa + pb - pc
        mm = math.sqrt(qq[0] ** 2 - qq[1:] @ qq[1:])
        q = math.sqrt(mm * mm / 4.0 - m * m)
        t_rest = np.concatenate([[mm / 2.0], q * nt])
        tb_rest = np.concatenate([[mm / 2.0], -q * nt])
        beta = qq[1:] / qq[0]
        out.append([pa, pb, boost(t_rest[None], beta)[0], boost(tb_rest[None], beta)[0], pc])
    return np.array(out)


def splitting_q_to_g(x):
    """The q -> g splitting function C_F (1 + (1 - x)^2) / x, x the gluon's momentum
    fraction (Altarelli & Parisi, Nucl. Phys. B126 (1977) 298)."""
    return (4.0 / 3.0) * (1.0 + (1.0 - x) ** 2) / x


# ----------------------------------------------------------------------------
# g g -> Q Q~ diagram by diagram, for the condition estimate
# ----------------------------------------------------------------------------
def _dirac_rep_gammas():
    """gamma^mu in the Dirac (standard) representation: gamma^0 = diag(1, 1, -1, -1),
    gamma^i = [[0, sigma_i], [-sigma_i, 0]] (a different basis from the oracle's chiral one)."""
    sig = [np.array([[0, 1], [1, 0]], complex), np.array([[0, -1j], [1j, 0]], complex),
           np.array([[1, 0], [0, -1]], complex)]
    g = np.zeros((4, 4, 4), complex)
    g[0] = np.diag([1, 1, -1, -1]).astype(complex)
    for i in range(3):
        g[i + 1, :2, 2:] = sig[i]
        g[i + 1, 2:, :2] = -sig[i]
    return g, sig


def _helicity_two_spinors(n, sig):
    """Eigenvectors of n.sigma for eigenvalues +1 and -1, from a numerical eigensolver
    (their phases are arbitrary; the quantities built from them do not depend on phases)."""
    m = n[0] * sig[0] + n[1] * sig[1] + n[2] * sig[2]
    val, vec = np.linalg.eigh(m)
    return {+1: vec[:, 1], -1: vec[:, 0]}


def _circular_polarisations(k):
    """(e1 + i lam e2)/sqrt(2) with e1, e2, k-hat right-handed and orthonormal; zero time
    component.  Any such e1 gives the helicity vectors up to a phase."""
    n = k[1:] / np.linalg.norm(k[1:])
    ref = np.array([1.0, 0.0, 0.0]) if abs(n[0]) < 0.9 else np.array([0.0, 1.0, 0.0])
    e1 = ref - (ref @ n) * n
    e1 /= np.linalg.norm(e1)
    e2 = np.cross(n, e1)
    return {lam: np.concatenate([[0.0], (e1 + 1j * lam * e2) / math.sqrt(2.0)]) for lam in (1, -1)}


def gg_qq_pair_terms(p, m, alphas):
    """For one event g(k1) g(k2) -> Q(p1) Q~(p2) with on-shell heavy quarks: the terms
    x[h, s, t] = Re(conj(A_s) G_st A_t) of the colour- and helicity-summed |M|^2, for the
    three diagrams (t-channel colour t^a t^b, u-channel t^b t^a, s-channel f^abc t^c) and
    the 16 helicity configurations h.  Written from the Feynman rules (quark-gluon vertex
    i g gamma^mu t^a, gluon propagator -i g_{mu nu}/q^2, three-gluon vertex g f^abc [...],
    all momenta incoming) in the Dirac representation, with helicity spinors
    u = (sqrt(E+m) chi, lam sqrt(E-m) chi), v = (-lam sqrt(E-m) eta, sqrt(E+m) eta),
    eta = chi_{-lam}, and G_st = sum over colours of conj(K_s) K_t."""
    gam, sig = _dirac_rep_gammas()
    metric = np.array([1.0, -1.0, -1.0, -1.0])
    g = math.sqrt(4.0 * math.pi * alphas)
    k1, k2, p1, p2 = p[0], p[1], p[2], p[3]

    def slash_(a):
        return np.einsum("m,mij->ij", (a * metric).astype(complex), gam)

    def dot(a, b):
        return a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3]

    def u_spinor(q, lam):
        e, a = q[0], np.linalg.norm(q[1:])
        chi = _helicity_two_spinors(q[1:] / a, sig)[lam]
        return np.concatenate([math.sqrt(e + m) * chi, lam * math.sqrt(e - m) * chi])

    def v_spinor(q, lam):
        e, a = q[0], np.linalg.norm(q[1:])
        eta = _helicity_two_spinors(q[1:] / a, sig)[-lam]
        return np.concatenate([-lam * math.sqrt(e - m) * eta, math.sqrt(e + m) * eta])

    def prop(q):
        return (slash_(q) + m * np.eye(4)) / (dot(q, q) - m * m)

    t = _t_matrices()
    f = np.real(-2j * np.einsum("aij,bjk,cki->abc", t, t, t) + 2j * np.einsum("bij,ajk,cki->abc", t, t, t))
    kcol = [np.einsum("aik,bkj->abij", t, t), np.einsum("bik,akj->abij", t, t),
            np.einsum("abc,cij->abij", f, t)]
    gmat = np.array([[np.sum(np.conj(ks) * kt) for kt in kcol] for ks in kcol])
    eps1, eps2 = _circular_polarisations(k1), _circular_polarisations(k2)
    s = dot(k1 + k2, k1 + k2)
    out = []
    for l1, l2, lq, lqb in itertools.product((1, -1), repeat=4):
        e1, e2 = eps1[l1], eps2[l2]
        ubar = np.conj(u_spinor(p1, lq)) @ gam[0]
        v = v_spinor(p2, lqb)
        a_t = -1j * g * g * ubar @ slash_(e1) @ prop(p1 - k1) @ slash_(e2) @ v
        a_u = -1j * g * g * ubar @ slash_(e2) @ prop(p1 - k2) @ slash_(e1) @ v
        vert = dot(e1, e2) * (k1 - k2) + 2.0 * dot(e1, k2) * e2 - 2.0 * dot(e2, k1) * e1
        a_s = g * g * (ubar @ slash_(vert) @ v) / s
        amp = np.array([a_t, a_u, a_s])
        out.append(np.real(np.conj(amp)[:, None] * gmat * amp[None, :]))
    return np.array(out)
