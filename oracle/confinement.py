"""Quartic confining potential a (r - R)^4 and the preconditioning equation (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Paper: Sec. "Support function optimization".  During the first iterations of the outer
loop each support function alpha sees its own Hamiltonian H_alpha = H_KS +
a_alpha (r - R_alpha)^4 (the text before Eq. trace); the confining term can be
"evaluated via convolutions in the same manner as the kinetic energy"; the gradient is
preconditioned by solving Eq. precond,
  (-1/2 nabla^2 + a_alpha (r - R_alpha)^4 - eps_alpha) g_prec = -g,
approximately, with eps_alpha an approximation of Lambda_alpha,alpha.

Readings taken where the paper is silent:

* the quartic is represented exactly in the two-level basis (its Galerkin matrix):
  (r - R)^4 = sum_d X_d^4 + 2 sum_{d<e} X_d^2 X_e^2 with X_d = x_d - R_d; each term is a
  product of 1D multiplication operators along single dimensions (identity along the
  others), and the 1D matrix between basis functions chi^b_i (b = 0 scaling, 1 wavelet,
  coarse point i, spacing h) is
    <chi^b_i | (x - R)^m | chi^b'_j> = (h/2)^m sum_{k,k'} X_k Y_k' sum_p C(m,p)
                                        (2i + k - 2c)^(m-p) F^p(2(j-i) + k' - k),
  X, Y = h or g (the filters of b, b'), c = R/h, F^p the moment overlaps
  int x^p phi(x) phi(x - l) dx (filters.moment_overlaps);
* the equation is solved on L(alpha): A = P_L (T + Q - eps) P_L (T the kinetic operator
  of hamiltonian.kinetic3d, Q the confinement), by conjugate gradients from
  g_prec = 0 for a fixed number of iterations; eps_alpha < 0 (a bound state) keeps A
  positive definite.
"""
from __future__ import annotations

import math

import numpy as np

from . import filters as _filters
from . import hamiltonian as _H

HALF = 14   # band of the 1D blocks: |j - i| <= 14


def quartic_block_1d(m, b, bp, i_idx, j_idx, c, h, F):
    """Matrix [len(i_idx), len(j_idx)] of <chi^b_i | (x - R)^m | chi^b'_j>, c = R / h.

    Entry (i, j) = (h/2)^m sum_p C(m,p) sum_{k,k'} X_k (2i + k - 2c)^(m-p) Y_k'
    F^p(2(j - i) + k' - k): for each offset j - i the sum over k' is one product with Y,
    the sum over k one product with the powers of (2i + k - 2c), all i at once."""
    X = F.h if b == 0 else F.g
    Y = F.h if bp == 0 else F.g
    ks = np.arange(F.h_lo, F.h_lo + len(F.h))
    i_idx = np.asarray(i_idx)
    j_idx = np.asarray(j_idx)
    out = np.zeros((len(i_idx), len(j_idx)))
    base = 2.0 * i_idx[:, None] + ks[None, :] - 2.0 * c                 # [i, k]
    for d in range(-HALF, HALF + 1):
        lmat = 2 * d + ks[None, :] - ks[:, None]                         # [k, k']
        ok = np.abs(lmat) <= HALF
        col = np.zeros(len(i_idx))
        for p in range(m + 1):
            Fp = np.where(ok, F.movl[p][np.clip(lmat + HALF, 0, 2 * HALF)], 0.0)
            col += math.comb(m, p) * ((base ** (m - p)) * X[None, :]) @ (Fp @ Y)
        # place entry (i, j = i + d) where j is one of the requested columns
        pos = np.searchsorted(j_idx, i_idx + d)
        hit = (pos < len(j_idx)) & (j_idx[np.minimum(pos, len(j_idx) - 1)] == i_idx + d)
        out[np.nonzero(hit)[0], pos[hit]] = col[hit]
    return out * (h / 2.0) ** m


_BLOCKS = {}


def _blocks(d_lo, n, c, h, F):
    """The 1D blocks of (x - R)^2 and (x - R)^4 on the index range [d_lo, d_lo + n)."""
    key = (int(d_lo), int(n), float(c), float(h), id(F))
    if key not in _BLOCKS:
        idx = np.arange(d_lo, d_lo + n)
        _BLOCKS[key] = {m: {(b, bp): quartic_block_1d(m, b, bp, idx, idx, c, h, F)
                            for b in (0, 1) for bp in (0, 1)} for m in (2, 4)}
    return _BLOCKS[key]


def _apply_1d(arr, axis, blocks):
    """Apply a 1D two-level operator along ``axis`` of the 8-type array ``arr``:
    out[t] = sum_b' B_{b b'} arr[t with bit b'] along the axis, b the bit of t."""
    out = np.zeros_like(arr)
    for t in range(8):
        b = (t >> axis) & 1
        for bp in (0, 1):
            src = (t & ~(1 << axis)) | (bp << axis)
            B = blocks[(b, bp)]
            out[t] += np.moveaxis(np.tensordot(B, arr[src], axes=([1], [axis])), 0, axis)
    return out


def confine3d(c, lo, centre, a, h, F=None):
    """Q c = a (r - R)^4 c (Galerkin) for dense type arrays c[t, x, y, z] on the coarse
    block at ``lo``.  Returns (out, out_lo): the block widened by 14 on every side."""
    F = F or _filters.load()
    n = c.shape[1:]
    P = [n[d] + 2 * HALF for d in range(3)]
    cp = np.zeros((8,) + tuple(P))
    cp[:, HALF:HALF + n[0], HALF:HALF + n[1], HALF:HALF + n[2]] = c
    out_lo = [lo[d] - HALF for d in range(3)]
    cc = [centre[d] / h for d in range(3)]
    blocks = {}
    for d in range(3):
        bd = _blocks(out_lo[d], P[d], cc[d], h, F)
        for m in (2, 4):
            blocks[d, m] = bd[m]
    total = np.zeros_like(cp)
    for d in range(3):
        total += _apply_1d(cp, d, blocks[d, 4])
    for d in range(3):
        for e in range(d + 1, 3):
            total += 2.0 * _apply_1d(_apply_1d(cp, d, blocks[d, 2]), e, blocks[e, 2])
    return a * total, out_lo


def _box_of(geo, f):
    L = geo.L[geo.sf_atom[f]]
    return L, list(L.lo), tuple(L.hi - L.lo + 1)


def confinement_energy_and_action(geo, f, phi_f, a, F=None):
    """(Q phi on L'(f) compressed, <phi|Q phi>) for the quartic centred on f's atom."""
    F = F or _filters.load()
    L, lo, shape = _box_of(geo, f)
    Lp = geo.Lp[geo.sf_atom[f]]
    N = geo.desc.N
    c = _H.uncompress(N, L, np.asarray(phi_f, np.float64), lo, shape)
    q, qlo = confine3d(c, lo, geo.desc.pos[geo.sf_atom[f]], a, geo.desc.h, F)
    e = float(np.sum(c * q[(slice(None),) + tuple(slice(HALF, HALF + s) for s in shape)]))
    blo = [min(qlo[d], Lp.lo[d]) for d in range(3)]
    bhi = [max(qlo[d] + q.shape[d + 1], Lp.hi[d] + 1) for d in range(3)]
    tot = np.zeros((8,) + tuple(bhi[d] - blo[d] for d in range(3)))
    _H._place(tot, blo, q, qlo)
    return _H.compress(N, Lp, tot, blo), e


def precond_operator(geo, f, x, a, eps, F=None):
    """A x = P_L (T + Q - eps) P_L x for a compressed vector x on L(f) (Eq. precond)."""
    F = F or _filters.load()
    L, lo, shape = _box_of(geo, f)
    N = geo.desc.N
    c = _H.uncompress(N, L, np.asarray(x, np.float64), lo, shape)
    kin = _H.kinetic3d(c, geo.desc.h, F)                       # block lo - 14
    q, qlo = confine3d(c, lo, geo.desc.pos[geo.sf_atom[f]], a, geo.desc.h, F)
    inner = (slice(None),) + tuple(slice(HALF, HALF + s) for s in shape)
    tot = kin[inner] + q[inner] - eps * c
    return _H.compress(N, L, tot, lo)


def precondition(geo, f, g, a, eps, iters, F=None):
    """Conjugate gradients on A g_prec = -g from g_prec = 0, ``iters`` iterations.

    Returns (g_prec, residual 2-norms after each iteration)."""
    F = F or _filters.load()
    b = -np.asarray(g, np.float64)
    x = np.zeros_like(b)
    r = b.copy()
    p = r.copy()
    rr = float(np.dot(r, r))
    res = []
    for _ in range(iters):
        Ap = precond_operator(geo, f, p, a, eps, F)
        alpha = rr / float(np.dot(p, Ap))
        x = x + alpha * p
        r = r - alpha * Ap
        rr_new = float(np.dot(r, r))
        res.append(math.sqrt(rr_new))
        if rr_new == 0.0:
            break
        p = r + (rr_new / rr) * p
        rr = rr_new
    return x, res
