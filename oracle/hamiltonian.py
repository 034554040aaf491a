"""Localized Hamiltonian application H phi = L' (T + W^T M^T diag(V) M W) L phi (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Paper: Sec. II.A (H_KS = -1/2 nabla^2 + V), Sec. II.B Eq. phi (expansion in one scaling
function and seven wavelets per fine point; tensor products phi(x-i1) phi(y-i2)
phi(z-i3)), Sec. III.B (H phi = L' H L phi, applied only on the localization
regions).  The paper delegates the convolutions to the BigDFT literature; the reading
taken here (every step a plain separable 1D pass over a dense box, FP64):

  1. uncompress phi on L into dense type arrays c_t, t = bx + 2 by + 4 bz
     (b_d = 1: wavelet along dimension d; t = 0 is the scaling part s);
  2. synthesis W, one level, per dimension: c'_k = sum_i h_{k-2i} s_i + g_{k-2i} d_i,
     giving scaling coefficients at spacing h/2;
  3. magic filter M per dimension: u_j = sum_k w_{j-k} c'_k, values at x_j = j h/2;
  4. v_j = V(x_j) u_j on the locreg slice of the global V (E_pot = sum_j V_j u_j^2);
  5. M^T then W^T (analysis) back to the two-level coefficients;
  6. kinetic T = -1/(2h^2) sum_d (1D Galerkin blocks T_XY along d) (x) delta (x) delta;
  7. H phi = potential part + kinetic part, gathered on the members of L'.

Free boundary: intermediate arrays are unbounded (zero outside); V must cover fine
indices [-14, 2N+14] per dimension.
"""
from __future__ import annotations

import numpy as np

from . import filters as _filters
from .geometry import gcoords


# ------------------------------------------------------------------ 1D passes

def _along(a, axis):
    return np.moveaxis(a, axis, -1)


def upsample(a_s, a_d, start, fs, fd, f_lo, axis):
    """c'_k = sum_i fs[k-2i] s_i + fd[k-2i] d_i along ``axis``.

    ``start`` = global coarse index of element 0; returns (out, global fine start)."""
    s = _along(a_s, axis)
    d = _along(a_d, axis)
    n = s.shape[-1]
    L = len(fs)
    out = np.zeros(s.shape[:-1] + (2 * (n - 1) + L,))
    for t in range(L):
        out[..., t:t + 2 * (n - 1) + 1:2] += fs[t] * s + fd[t] * d
    return np.moveaxis(out, -1, axis), 2 * start + f_lo


def downsample(a, start, f, f_lo, axis):
    """s_i = sum_k f[k-2i] a_k along ``axis`` (transpose of one branch of upsample)."""
    x = _along(a, axis)
    n = x.shape[-1]
    L = len(f)
    f_hi = f_lo + L - 1
    i_lo = -((-(start - f_hi)) // 2)             # ceil((start - f_hi) / 2)
    i_hi = (start + n - 1 - f_lo) // 2
    nout = i_hi - i_lo + 1
    k0 = 2 * i_lo + f_lo                          # first fine index touched
    pad_lo = start - k0
    padded = np.zeros(x.shape[:-1] + (2 * (nout - 1) + L,))
    padded[..., pad_lo:pad_lo + n] = x
    out = np.zeros(x.shape[:-1] + (nout,))
    for t in range(L):
        out += f[t] * padded[..., t:t + 2 * (nout - 1) + 1:2]
    return np.moveaxis(out, -1, axis), i_lo


def convolve(a, start, w, w_lo, axis):
    """u_j = sum_k w[j-k] a_k (magic filter); returns (out, global start)."""
    x = _along(a, axis)
    n = x.shape[-1]
    L = len(w)
    out = np.zeros(x.shape[:-1] + (n + L - 1,))
    for t in range(L):
        out[..., t:t + n] += w[t] * x
    return np.moveaxis(out, -1, axis), start + w_lo


def convolve_t(a, start, w, w_lo, axis):
    """c_k = sum_j w[j-k] a_j (transposed magic filter); returns (out, global start)."""
    x = _along(a, axis)
    n = x.shape[-1]
    L = len(w)
    w_hi = w_lo + L - 1
    out = np.zeros(x.shape[:-1] + (n + L - 1,))
    for t in range(L):
        # l = w_lo + t; k = j - l  ->  k_local = j_local + (w_hi - l)
        o = w_hi - (w_lo + t)
        out[..., o:o + n] += w[t] * x
    return np.moveaxis(out, -1, axis), start - w_hi


def correlate(a, T, T_half, axis):
    """out_i = sum_l T(l) a_{i+l}, l = -T_half..T_half; out starts T_half before a."""
    x = _along(a, axis)
    n = x.shape[-1]
    out = np.zeros(x.shape[:-1] + (n + 2 * T_half,))
    for t in range(2 * T_half + 1):
        l = t - T_half
        out[..., T_half - l:T_half - l + n] += T[t] * x
    return np.moveaxis(out, -1, axis)


# ------------------------------------------------------------------ compression

def uncompress(N, loc, phi, lo, shape):
    """Dense type arrays c[t, x, y, z] on the block starting at ``lo`` (A9 layout)."""
    c = np.zeros((8,) + tuple(shape))
    nc = len(loc.coarse.g)
    nf = len(loc.fine.g)
    i1, i2, i3 = gcoords(N, loc.coarse.g)
    c[0, i1 - lo[0], i2 - lo[1], i3 - lo[2]] = phi[:nc]
    j1, j2, j3 = gcoords(N, loc.fine.g)
    for t in range(1, 8):
        c[t, j1 - lo[0], j2 - lo[1], j3 - lo[2]] = phi[nc + (t - 1) * nf: nc + t * nf]
    return c


def compress(N, loc, c, lo):
    """Inverse of uncompress on the members of ``loc`` (values outside are dropped)."""
    nc = len(loc.coarse.g)
    nf = len(loc.fine.g)
    out = np.zeros(nc + 7 * nf)
    i1, i2, i3 = gcoords(N, loc.coarse.g)
    out[:nc] = c[0, i1 - lo[0], i2 - lo[1], i3 - lo[2]]
    j1, j2, j3 = gcoords(N, loc.fine.g)
    for t in range(1, 8):
        out[nc + (t - 1) * nf: nc + t * nf] = c[t, j1 - lo[0], j2 - lo[1], j3 - lo[2]]
    return out


# ------------------------------------------------------------------ operators

def synthesis3d(c, lo, F):
    """W: 8 type arrays on the coarse block -> scaling coefficients at h/2 (x, y, z)."""
    a = {t: c[t] for t in range(8)}
    start = list(lo)
    for axis in range(3):
        nxt = {}
        for t in a:
            if (t >> axis) & 1:
                continue
            s, d = a[t], a[t | (1 << axis)]
            out, st = upsample(s, d, start[axis], F.h, F.g, F.h_lo, axis)
            nxt[t] = out
        start[axis] = st
        a = nxt
    return a[0], start


def analysis3d(cf, start, F):
    """W^T: scaling coefficients at h/2 -> 8 type arrays on a coarse block."""
    a = {0: cf}
    start = list(start)
    for axis in (2, 1, 0):
        nxt = {}
        for t, arr in a.items():
            s, i_lo = downsample(arr, start[axis], F.h, F.h_lo, axis)
            d, _ = downsample(arr, start[axis], F.g, F.h_lo, axis)
            nxt[t] = s
            nxt[t | (1 << axis)] = d
        start[axis] = i_lo
        a = nxt
    shape = a[0].shape
    c = np.zeros((8,) + shape)
    for t in range(8):
        c[t] = a[t]
    return c, start


def magic3d(cf, start, F):
    u = cf
    st = list(start)
    for axis in range(3):
        u, st[axis] = convolve(u, st[axis], F.magic, F.magic_lo, axis)
    return u, st


def magic3d_t(v, start, F):
    c = v
    st = list(start)
    for axis in (2, 1, 0):
        c, st[axis] = convolve_t(c, st[axis], F.magic, F.magic_lo, axis)
    return c, st


def kinetic3d(c, h, F):
    """T c with T = -1/(2h^2) sum_d T_{b_d b'_d} along d (identity on the other dims).

    Input on a coarse block; output on the block widened by 14 on every side."""
    half = -F.kin_lo
    shape = tuple(s + 2 * half for s in c.shape[1:])
    out = np.zeros((8,) + shape)
    name = "hg"
    for b in range(8):
        for axis in range(3):
            bit = (b >> axis) & 1
            for bp in (0, 1):
                src = (b & ~(1 << axis)) | (bp << axis)
                T = F.kin[name[bit] + name[bp]]
                r = correlate(c[src], T, half, axis)
                sl = [slice(half, half + n) for n in c.shape[1:]]
                sl[axis] = slice(0, r.shape[axis])
                out[(b,) + tuple(sl)] += r
    return out * (-1.0 / (2.0 * h * h))


def _place(dst, dst_lo, src, src_lo):
    """dst[...] += src on the overlap of the two blocks (leading type axis kept)."""
    sl_d, sl_s = [slice(None)], [slice(None)]
    for d in range(3):
        a0 = max(dst_lo[d], src_lo[d])
        a1 = min(dst_lo[d] + dst.shape[d + 1], src_lo[d] + src.shape[d + 1])
        if a1 <= a0:
            return
        sl_d.append(slice(a0 - dst_lo[d], a1 - dst_lo[d]))
        sl_s.append(slice(a0 - src_lo[d], a1 - src_lo[d]))
    dst[tuple(sl_d)] += src[tuple(sl_s)]


def v_slice(V, V_lo, start, shape):
    """V on the fine block [start, start+shape), returned indexed [x, y, z].

    The global array is stored [jz, jy, jx] (x fastest) from fine index ``V_lo``."""
    sl = tuple(slice(start[d] - V_lo[d], start[d] - V_lo[d] + shape[d]) for d in range(3))
    for d in range(3):
        if sl[d].start < 0 or sl[d].stop > V.shape[2 - d]:
            raise ValueError("V does not cover the real-space block of the locreg")
    return np.asarray(V[sl[2], sl[1], sl[0]]).transpose(2, 1, 0)


def apply_hamiltonian(geo, f, phi_f, V, V_lo, F=None, parts=False):
    """H phi_f on L'(f) (compressed), E_kin = <phi|T phi>, E_pot = <phi|V phi>.

    ``V`` is indexed V[jz - V_lo[2], jy - V_lo[1], jx - V_lo[0]] over fine indices j."""
    F = F or _filters.load()
    desc = geo.desc
    N = desc.N
    a = geo.sf_atom[f]
    L, Lp = geo.L[a], geo.Lp[a]
    lo = L.lo
    shape = tuple(L.hi - L.lo + 1)
    c = uncompress(N, L, np.asarray(phi_f, np.float64), lo, shape)

    # potential: W^T M^T V M W
    cf, st = synthesis3d(c, lo, F)
    u, ust = magic3d(cf, st, F)
    vv = v_slice(V, V_lo, ust, u.shape)
    e_pot = float(np.sum(vv * u * u))
    v = vv * u
    cb, bst = magic3d_t(v, ust, F)
    pot, plo = analysis3d(cb, bst, F)

    # kinetic on the two-level coefficients
    kin = kinetic3d(c, desc.h, F)
    half = -F.kin_lo
    klo = [lo[d] - half for d in range(3)]
    e_kin = float(np.sum(c * kin[(slice(None),) + tuple(slice(half, half + n) for n in shape)]))

    # sum on a common block covering L'
    blo = [min(plo[d], klo[d], Lp.lo[d]) for d in range(3)]
    bhi = [max(plo[d] + pot.shape[d + 1], klo[d] + kin.shape[d + 1], Lp.hi[d] + 1) for d in range(3)]
    tot_pot = np.zeros((8,) + tuple(bhi[d] - blo[d] for d in range(3)))
    tot_kin = np.zeros_like(tot_pot)
    _place(tot_pot, blo, pot, plo)
    _place(tot_kin, blo, kin, klo)
    if parts:
        return (compress(N, Lp, tot_pot, blo), compress(N, Lp, tot_kin, blo), e_kin, e_pot)
    hphi = compress(N, Lp, tot_pot + tot_kin, blo)
    return hphi, e_kin, e_pot


def hphi_abs_bound(geo, f, phi_f, V, V_lo, F=None):
    """Absolute-term bound of every element of H phi_f on L'(f): the steps of
    ``apply_hamiltonian`` taken with |phi|, |V| and every filter tap (h, g, magic,
    kinetic blocks) replaced by its absolute value, the kinetic and potential parts
    added in absolute value.  Each element is the sum of the magnitudes of the terms
    whose sum is that element, so any order of evaluation rounds it by at most a
    multiple of the unit roundoff times this bound."""
    import dataclasses
    F = F or _filters.load()
    Fa = dataclasses.replace(F, h=np.abs(F.h), g=np.abs(F.g), magic=np.abs(F.magic),
                             kin={k: np.abs(v) for k, v in F.kin.items()})
    pot, kin, _, _ = apply_hamiltonian(geo, f, np.abs(np.asarray(phi_f, np.float64)), np.abs(V), V_lo, Fa,
                                       parts=True)
    return np.abs(pot) + np.abs(kin)
