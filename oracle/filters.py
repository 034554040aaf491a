"""Daubechies-16 least-asymmetric filters and the operator filters built on them (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

What the paper fixes (Sec. II.B, "Daubechies wavelets in BigDFT" and Fig. Daub_16):
the basis is the orthogonal, least-asymmetric Daubechies family of order 2m = 16;
scaling function phi and wavelet psi are supported on [1-m, m] = [-7, 8]; the family
reproduces low-degree polynomials exactly.  The paper prints no coefficient and
delegates the operator filters to the BigDFT literature, so this module derives every
number from the mathematics, in multi-precision arithmetic (mpmath), and rounds to
FP64 once, when the table ``filters_d16.txt`` is written.

Readings taken where the paper is silent:

* low-pass filter h_j, j = -7..8 (sum h = sqrt 2): spectral factor of the Daubechies
  polynomial P(y) = sum_{k<8} C(7+k, k) y^k, |H(w)|^2 = 2 cos^16(w/2) P(sin^2(w/2)).
  "Least asymmetric" = among the 16 real factorizations, the one whose non-binomial
  factor Q(e^{-iw}) has the smallest maximal deviation of its unwrapped phase from the
  chord joining w = 0 and w = pi (Daubechies, Ten Lectures, Sec. 8.1.1).  A factor and
  its mirror image tie; the tie is broken by taking the orientation whose scaling
  function has first moment M_1 <= 1/2.
* high-pass filter g_j = (-1)^j h_{1-j}, same support.
* "polynomials up to 8th order" is read as degree <= 7 (m = 8 vanishing moments).
* moments M_p = int x^p phi(x) dx from the refinement equation.
* magic filter w_l, l = -7..8: the 16-tap filter with the moments of phi,
  sum_l w_l l^p = M_p for p = 0..15; u_j = sum_k w_{j-k} c_k maps scaling
  coefficients to point values (window centred on supp phi since M_1 ~ 0.16).
* moment overlaps F^p(l) = int x^p phi(x) phi(x - l) dx, p <= 4, |l| <= 14, from the
  refinement equation (the multiplication operators x^p of the quartic confining
  potential, Sec. "Support function optimization": evaluated by convolutions like the
  kinetic energy).
* kinetic filters: Galerkin connection coefficients r_l = int phi(x) phi''(x-l) dx,
  |l| <= 14, from r_l = 4 sum_{i,j} h_i h_j r_{2l+j-i} with sum_l l^2 r_l = 2
  (Beylkin 1992); the scale-h blocks T_XY(l) = 4 sum_{k,k'} X_k Y_k' r_{2l+k'-k},
  X, Y in {h, g}, so that <X_i| d^2/dx^2 |Y_j> = T_XY(j - i) (unit spacing).
"""
from __future__ import annotations

import itertools
import os
from dataclasses import dataclass

import numpy as np

TABLE_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "filters_d16.txt")

M_ORDER = 8            # m: number of vanishing moments; filter length 2m = 16
H_LO = 1 - M_ORDER     # support of h, g, phi, psi: [-7, 8]
MAGIC_LO = -7          # magic filter taps l = -7..8
KIN_HALF = 2 * M_ORDER - 2  # r_l nonzero for |l| <= 14


# ----------------------------------------------------------------------------
# multi-precision derivation (needs mpmath; used to write the table)
# ----------------------------------------------------------------------------

def _mp():
    import mpmath
    return mpmath


def _polymul(p, q):
    out = [0] * (len(p) + len(q) - 1)
    for i, a in enumerate(p):
        for j, b in enumerate(q):
            out[i + j] += a * b
    return out


def daubechies_candidates(dps: int = 60):
    """All real spectral factors h (j = -7..8) of the order-16 Daubechies filter.

    Returns a list of (phase_deviation, first_moment, h) with mpmath numbers.
    Sec. II.B (order 2m = 16); construction: Daubechies, Ten Lectures, Sec. 6.1.
    """
    mp = _mp()
    mp.mp.dps = dps
    m = M_ORDER
    # P(y) = sum_{k<m} C(m-1+k, k) y^k
    pcoef = [mp.binomial(m - 1 + k, k) for k in range(m)]
    yroots = mp.polyroots(pcoef[::-1], maxsteps=400, extraprec=4 * dps)
    tiny = mp.mpf(10) ** (-(dps // 2))
    groups = [("r", y) for y in yroots if abs(mp.im(y)) < tiny]
    groups += [("c", y) for y in yroots if mp.im(y) >= tiny]

    def zpair(y):
        # y = sin^2(w/2) = (2 - z - 1/z)/4  <=>  z^2 - (2 - 4y) z + 1 = 0
        b = 2 - 4 * y
        d = mp.sqrt(b * b - 4)
        z1, z2 = (b + d) / 2, (b - d) / 2
        return (z1, z2) if abs(z1) < abs(z2) else (z2, z1)

    out = []
    for bits in itertools.product([0, 1], repeat=len(groups)):
        zs = []
        for bit, (kind, y) in zip(bits, groups):
            z = zpair(y)[bit]
            if kind == "r":
                zs.append(mp.re(z))
            else:
                zs += [z, mp.conj(z)]
        q = [mp.mpf(1)]
        for z in zs:
            q = _polymul(q, [-z, 1])
        q = [mp.re(c) for c in q]
        if sum(q) < 0:
            q = [-c for c in q]
        poly = list(q)
        for _ in range(m):
            poly = _polymul(poly, [1, 1])
        s = sum(poly)
        h = [c * mp.sqrt(2) / s for c in poly]
        dev = phase_deviation(q)
        m1 = mp.sqrt(2) / 2 * sum((j + H_LO) * h[j] for j in range(2 * m))
        out.append((dev, m1, h))
    return out


def phase_deviation(q, samples: int = 1024):
    """Max deviation of the unwrapped phase of Q(e^{-iw}) = sum_k q_k e^{-ikw} from the
    chord through w = 0 and w = pi (least-asymmetry criterion, see module doc)."""
    mp = _mp()
    th = []
    prev = mp.mpf(0)
    for k in range(samples + 1):
        w = mp.pi * k / samples
        a = mp.arg(sum(c * mp.expj(-w * i) for i, c in enumerate(q)))
        while a - prev > mp.pi:
            a -= 2 * mp.pi
        while a - prev < -mp.pi:
            a += 2 * mp.pi
        th.append(a)
        prev = a
    return max(abs(th[k] - th[samples] * k / samples) for k in range(samples + 1))


def least_asymmetric_h(dps: int = 60):
    """h_j, j = -7..8, of the least-asymmetric order-16 Daubechies filter (Sec. II.B)."""
    mp = _mp()
    cands = daubechies_candidates(dps)
    best = min(c[0] for c in cands)
    tied = [c for c in cands if abs(c[0] - best) < mp.mpf(10) ** -20]
    tied = [c for c in tied if c[1] <= mp.mpf(1) / 2]
    assert len(tied) == 1, "least-asymmetric factor not unique"
    return tied[0][2]


def high_pass(h):
    """g_j = (-1)^j h_{1-j}, j = -7..8 (quadrature mirror filter, same support)."""
    n = len(h)
    return [(-1) ** (j) * h[(1 - j) - H_LO] for j in range(H_LO, H_LO + n)]


def moments(h, pmax: int = 2 * M_ORDER - 1):
    """M_p = int x^p phi(x) dx, p = 0..pmax, from the refinement equation
    phi(x) = sqrt2 sum_j h_j phi(2x - j):
    M_p (1 - 2^-p) = 2^(-p-1) sqrt2 sum_{i<p} C(p,i) M_i sum_j h_j j^(p-i),  M_0 = 1."""
    mp = _mp()
    js = list(range(H_LO, H_LO + len(h)))
    hm = [sum(hj * mp.mpf(j) ** q for hj, j in zip(h, js)) for q in range(pmax + 1)]
    M = [mp.mpf(1)]
    for p in range(1, pmax + 1):
        acc = sum(mp.binomial(p, i) * M[i] * hm[p - i] for i in range(p))
        M.append(mp.sqrt(2) * acc / (2 ** (p + 1) * (1 - mp.mpf(2) ** (-p))))
    return M


def magic_filter(M, lo: int = MAGIC_LO):
    """w_l, l = lo..lo+15, with sum_l w_l l^p = M_p, p = 0..15 (Vandermonde solve)."""
    mp = _mp()
    n = len(M)
    A = mp.matrix(n, n)
    for p in range(n):
        for k in range(n):
            A[p, k] = mp.mpf(lo + k) ** p
    b = mp.matrix([M[p] for p in range(n)])
    x = mp.lu_solve(A, b)
    return [x[k] for k in range(n)]


def connection_coefficients(h):
    """r_l = int phi(x) phi''(x - l) dx, l = -14..14 (Beylkin 1992).

    Two-scale relation r_l = 4 sum_n a_n r_{2l+n}, a_n = sum_i h_i h_{i+n}; the
    eigen-system is singular (left null vector l^2), so the row l = 14 is replaced by
    the normalization sum_l l^2 r_l = 2 (from d^2/dx^2 x^2 = 2)."""
    mp = _mp()
    L = KIN_HALF
    n = len(h)
    a = {}
    for d in range(-(n - 1), n):
        a[d] = sum(h[i] * h[i + d] for i in range(n) if 0 <= i + d < n)
    size = 2 * L + 1
    A = mp.matrix(size, size)
    for li, l in enumerate(range(-L, L + 1)):
        for mi, m in enumerate(range(-L, L + 1)):
            A[li, mi] = (1 if li == mi else 0) - 4 * a.get(m - 2 * l, 0)
    b = mp.matrix([0] * size)
    for mi, m in enumerate(range(-L, L + 1)):
        A[size - 1, mi] = mp.mpf(m) ** 2
    b[size - 1] = 2
    x = mp.lu_solve(A, b)
    return [x[k] for k in range(size)]


def kinetic_blocks(h, g, r):
    """T_XY(l), l = -14..14, for X, Y in {h, g}: <X_0|d^2|Y_l> = 4 sum X_k Y_k' r_{2l+k'-k}."""
    L = KIN_HALF
    rr = {l: r[l + L] for l in range(-L, L + 1)}
    js = list(range(H_LO, H_LO + len(h)))
    out = {}
    for nx, X in (("h", h), ("g", g)):
        for ny, Y in (("h", h), ("g", g)):
            blk = []
            for l in range(-L, L + 1):
                s = 0
                for k, xk in zip(js, X):
                    for kp, yk in zip(js, Y):
                        s += xk * yk * rr.get(2 * l + kp - k, 0)
                blk.append(4 * s)
            out[nx + ny] = blk
    return out


def moment_overlaps(h, pmax: int = 4):
    """F^p(l) = int x^p phi(x) phi(x - l) dx, p = 0..pmax, l = -14..14: the Galerkin
    entries of the multiplication operators x^p between scaling functions, which the
    quartic confining potential a (r - R)^4 of the support-function optimization needs
    ("evaluated via convolutions in the same manner as the kinetic energy").

    Refinement equation in both factors, then x = (s + a)/2:
      F^p(l) = 2^-p sum_{a,b} h_a h_b sum_{q<=p} C(p,q) a^(p-q) F^q(2l + b - a),
    i.e. (I - 2^-p T) F^p = 2^-p sum_{q<p} ..., with (T F)(l) = sum_n A_n F(2l + n) and
    A_n = sum_a h_a h_{a+n}.  F^0(l) = delta_l0 (orthonormal translates); for p >= 1 the
    matrix I - 2^-p T is regular (T has spectral radius 1)."""
    mp = _mp()
    L = KIN_HALF
    n = len(h)
    js = list(range(H_LO, H_LO + n))
    A = {}
    for d in range(-(n - 1), n):
        A[d] = sum(h[i] * h[i + d] for i in range(n) if 0 <= i + d < n)
    size = 2 * L + 1
    F = [[mp.mpf(1) if l == 0 else mp.mpf(0) for l in range(-L, L + 1)]]
    for p in range(1, pmax + 1):
        M = mp.matrix(size, size)
        b = mp.matrix([0] * size)
        for li, l in enumerate(range(-L, L + 1)):
            for mi, m in enumerate(range(-L, L + 1)):
                M[li, mi] = (1 if li == mi else 0) - mp.mpf(2) ** (-p) * A.get(m - 2 * l, 0)
            acc = mp.mpf(0)
            for q in range(p):
                for ja, ha in zip(js, h):
                    for jb, hb in zip(js, h):
                        idx = 2 * l + jb - ja
                        if -L <= idx <= L:
                            acc += mp.binomial(p, q) * mp.mpf(ja) ** (p - q) * ha * hb * F[q][idx + L]
            b[li] = mp.mpf(2) ** (-p) * acc
        x = mp.lu_solve(M, b)
        F.append([x[k] for k in range(size)])
    return F


def derive(dps: int = 60):
    """Every table entry in mpmath precision: dict name -> (lo, [values])."""
    h = least_asymmetric_h(dps)
    g = high_pass(h)
    M = moments(h)
    w = magic_filter(M)
    r = connection_coefficients(h)
    T = kinetic_blocks(h, g, r)
    tab = {
        "h": (H_LO, h),
        "g": (H_LO, g),
        "moments": (0, M),
        "magic": (MAGIC_LO, w),
        "kin_r": (-KIN_HALF, r),
    }
    for k, v in T.items():
        tab["kin_" + k] = (-KIN_HALF, v)
    for p, v in enumerate(moment_overlaps(h)):
        tab["movl_%d" % p] = (-KIN_HALF, v)
    return tab


def write_table(path: str = TABLE_PATH, dps: int = 60) -> None:
    """Write the FP64 table (40 significant digits, rounded to FP64 when read)."""
    mp = _mp()
    tab = derive(dps)
    lines = [
        "# Daubechies-16 least-asymmetric filters and derived operator filters.",
        "# Written by `python -m oracle.filters --write` (mpmath, %d digits)." % dps,
        "# Format: '<name> <first index> <count>' then one value per line.",
    ]
    for name, (lo, vals) in tab.items():
        lines.append("%s %d %d" % (name, lo, len(vals)))
        lines += [mp.nstr(v, 40, min_fixed=-1, max_fixed=0) if v != 0 else "0" for v in vals]
    with open(path, "w") as f:
        f.write("\n".join(lines) + "\n")


# ----------------------------------------------------------------------------
# FP64 table used by the oracle
# ----------------------------------------------------------------------------

@dataclass(frozen=True)
class Filters:
    """FP64 filter table; every array is indexed from its ``*_lo`` index."""
    h: np.ndarray        # j = -7..8
    g: np.ndarray        # j = -7..8
    moments: np.ndarray  # p = 0..15
    magic: np.ndarray    # l = -7..8
    kin_r: np.ndarray    # l = -14..14
    kin: dict            # "hh","hg","gh","gg" -> l = -14..14
    h_lo: int = H_LO
    magic_lo: int = MAGIC_LO
    kin_lo: int = -KIN_HALF
    movl: np.ndarray = None   # [p][l + 14]: int x^p phi(x) phi(x - l) dx, p = 0..4


def read_table(path: str = TABLE_PATH) -> dict:
    tab = {}
    with open(path) as f:
        rows = [ln.strip() for ln in f if ln.strip() and not ln.startswith("#")]
    i = 0
    while i < len(rows):
        name, lo, n = rows[i].split()
        lo, n = int(lo), int(n)
        tab[name] = (lo, np.array([float(v) for v in rows[i + 1:i + 1 + n]], dtype=np.float64))
        i += 1 + n
    return tab


_CACHE = {}


def load(path: str = TABLE_PATH) -> Filters:
    if path not in _CACHE:
        t = read_table(path)
        _CACHE[path] = Filters(
            h=t["h"][1], g=t["g"][1], moments=t["moments"][1], magic=t["magic"][1],
            kin_r=t["kin_r"][1],
            kin={k: t["kin_" + k][1] for k in ("hh", "hg", "gh", "gg")},
            movl=np.array([t["movl_%d" % p][1] for p in range(5)]),
        )
    return _CACHE[path]


if __name__ == "__main__":
    import sys
    if "--write" in sys.argv:
        write_table()
        print("wrote", TABLE_PATH)
