"""ctypes binding of ``liblsw.so`` (declared in include/lsw.h): argument marshalling only.

The functions below carry the C names and forward to the library; every step of the
Hamiltonian application and of the H/S build runs in the library's sm_103a kernels.
There is no Python or CPU fallback: if the library is missing, loading fails loudly.

``System`` is a convenience wrapper that keeps the handles, reads the layout, keys
and pattern into numpy arrays and takes torch tensors (their device pointers).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

(LSW_OK, LSW_ERR_ARG, LSW_ERR_OOM, LSW_ERR_CUDA, LSW_ERR_TIMEOUT, LSW_ERR_STATE, LSW_ERR_UNSUPPORTED,
 LSW_ERR_IO) = range(8)
LSW_HOST_ONLY = -1
LSW_FP64, LSW_FP32, LSW_FP32_BF16X = 0, 1, 2
LSW_REGION_L, LSW_REGION_LP = 0, 1
LSW_PART_COARSE, LSW_PART_FINE = 0, 1
LSW_FINE_UNION, LSW_FINE_OWN = 0, 1
LSW_PAIR_CUTOFF, LSW_PAIR_SUM_OF_RADII = 0, 1
FILTERS = {"h": 0, "g": 1, "moments": 2, "magic": 3, "kin_r": 4, "kin_hh": 5, "kin_hg": 6,
           "kin_gh": 7, "kin_gg": 8, "fwd_h": 9, "fwd_g": 10, "movl_0": 11, "movl_1": 12,
           "movl_2": 13, "movl_3": 14, "movl_4": 15}

_STATUS = {1: "LSW_ERR_ARG", 2: "LSW_ERR_OOM", 3: "LSW_ERR_CUDA", 4: "LSW_ERR_TIMEOUT",
           5: "LSW_ERR_STATE", 6: "LSW_ERR_UNSUPPORTED", 7: "LSW_ERR_IO"}


class LswError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (_STATUS.get(status, str(status)), msg))
        self.status = status


class lsw_system_desc(C.Structure):
    _fields_ = [("N", C.c_int32 * 3), ("h", C.c_double), ("n_atoms", C.c_int32),
                ("pos", C.POINTER(C.c_double)), ("r_loc", C.POINTER(C.c_double)),
                ("r_fine", C.POINTER(C.c_double)), ("n_sf", C.POINTER(C.c_int32)),
                ("lprime_margin", C.c_double), ("pair_cutoff", C.c_double),
                ("pair_mode", C.c_int32), ("fine_mode", C.c_int32), ("precision", C.c_int32)]


_lib = None
_P = C.c_void_p
_I64P = C.POINTER(C.c_int64)
_I32P = C.POINTER(C.c_int32)
_DP = C.POINTER(C.c_double)

_SIGS = {
    "lsw_last_error": (C.c_char_p, []),
    "lsw_ctx_create": (C.c_int, [C.c_int, _P, C.POINTER(_P)]),
    "lsw_ctx_destroy": (C.c_int, [_P]),
    "lsw_filter_table": (C.c_int, [_P, C.c_int32, _I32P, _I32P, _DP]),
    "lsw_system_create": (C.c_int, [_P, C.POINTER(lsw_system_desc), C.POINTER(_P)]),
    "lsw_system_destroy": (C.c_int, [_P]),
    "lsw_system_layout": (C.c_int, [_P, _I64P, _I64P, _I64P, C.POINTER(_I64P), C.POINTER(_I64P),
                                    C.POINTER(_I32P)]),
    "lsw_system_keys": (C.c_int, [_P, C.c_int32, C.c_int32, C.c_int32, _I64P, C.POINTER(_I64P)]),
    "lsw_pattern": (C.c_int, [_P, _I64P, C.POINTER(_I64P), C.POINTER(_I32P)]),
    "lsw_set_potential": (C.c_int, [_P, _P, _I64P, _I64P]),
    "lsw_apply_hamiltonian": (C.c_int, [_P, _P, _P, _P, _P]),
    "lsw_build_matrices": (C.c_int, [_P, _P, _P, _P, _P]),
    "lsw_build_density": (C.c_int, [_P, _P, _P, _P, _I64P, _I64P]),
    "lsw_apply_hamiltonian_noalloc": (C.c_int, [_P, _P, _P, _P, _P]),
    "lsw_combine": (C.c_int, [_P, _P, _P, _P]),
    "lsw_lowdin_taylor": (C.c_int, [_P, _P, _P, _P]),
    "lsw_add_confinement": (C.c_int, [_P, _P, _P, _P, _P]),
    "lsw_confinement_row": (C.c_int, [_P, C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_int64, _DP]),
    "lsw_precondition": (C.c_int, [_P, _P, _P, _P, _P, C.c_int32, _P]),
    "lsw_foe": (C.c_int, [_P, _P, _P, C.c_double, C.c_double, C.c_double, C.c_int32, C.c_double, C.c_double,
                          C.c_int32, _P, _P, _DP, _DP, _DP]),
    "lsw_reformat": (C.c_int, [_P, _P, _I32P, _P, _P]),
    "lsw_workspace_bytes": (C.c_int, [_P, _I64P]),
    "lsw_sync": (C.c_int, [_P, C.c_double]),
    "lsw_step_host": (C.c_int, [_P, _P, _P, _P, _P, _P, _P]),
    "lsw_set_option": (C.c_int, [_P, C.c_char_p, C.c_int64]),
    "lsw_profile": (C.c_int, [_P, C.c_int32]),
    "lsw_system_set_stream": (C.c_int, [_P, _P]),
    "lsw_profile_read": (C.c_int, [_P, C.c_int32, _I32P, _DP, _I64P]),
    "lsw_save": (C.c_int, [_P, _P, C.c_char_p]),
    "lsw_measure_peaks": (C.c_int, [_P, _DP, _DP, _DP]),
    "lsw_load": (C.c_int, [_P, C.c_char_p, C.POINTER(_P), _P]),
    "lsw_load_phi": (C.c_int, [_P, C.c_char_p, _P]),
}

TRACE_KINDS = ["memset", "uncompress", "fwd_xy", "z_stage", "bwd_xy", "kinetic", "hs_pack", "hs_tiles",
               "dens_realspace", "dens_products"]


def lib():
    """Load liblsw.so (built in-tree by ``paper_1401_7441_gb300.build``)."""
    global _lib
    if _lib is None:
        if not os.path.exists(_build.LIB):
            raise RuntimeError("liblsw.so is not built (run paper_1401_7441_gb300.build.build())")
        L = C.CDLL(_build.LIB)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def last_error() -> str:
    return lib().lsw_last_error().decode()


def check(status):
    if status != LSW_OK:
        raise LswError(status, last_error())


def _ptr(x):
    """Device/host pointer of a torch tensor, an int address, a numpy array or None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    return x.data_ptr()


# ---------------------------------------------------------------- same names as the C ABI

def lsw_ctx_create(device: int, stream=None):
    out = _P()
    check(lib().lsw_ctx_create(device, stream, C.byref(out)))
    return out


def lsw_ctx_destroy(ctx):
    check(lib().lsw_ctx_destroy(ctx))


def lsw_filter_table(ctx, which):
    first = C.c_int32()
    count = C.c_int32()
    vals = (C.c_double * 64)()
    w = FILTERS[which] if isinstance(which, str) else int(which)
    check(lib().lsw_filter_table(ctx, w, C.byref(first), C.byref(count), vals))
    return first.value, np.array(vals[:count.value])


def lsw_system_create(ctx, desc: lsw_system_desc):
    out = _P()
    check(lib().lsw_system_create(ctx, C.byref(desc), C.byref(out)))
    return out


def lsw_system_destroy(sys):
    check(lib().lsw_system_destroy(sys))


def lsw_system_layout(sys):
    n, tl, tp = C.c_int64(), C.c_int64(), C.c_int64()
    oL, oP, sa = _I64P(), _I64P(), _I32P()
    check(lib().lsw_system_layout(sys, C.byref(n), C.byref(tl), C.byref(tp), C.byref(oL), C.byref(oP),
                                  C.byref(sa)))
    nf = n.value
    return (nf, tl.value, tp.value, np.ctypeslib.as_array(oL, (nf + 1,)).copy(),
            np.ctypeslib.as_array(oP, (nf + 1,)).copy(), np.ctypeslib.as_array(sa, (nf,)).copy())


def lsw_system_keys(sys, atom, region, part):
    n = C.c_int64()
    k = _I64P()
    check(lib().lsw_system_keys(sys, atom, region, part, C.byref(n), C.byref(k)))
    if n.value == 0:
        return np.zeros((0, 3), np.int64)
    return np.ctypeslib.as_array(k, (n.value * 3,)).reshape(-1, 3).copy()


def lsw_pattern(sys):
    nnz = C.c_int64()
    rp, col = _I64P(), _I32P()
    check(lib().lsw_pattern(sys, C.byref(nnz), C.byref(rp), C.byref(col)))
    nf = lsw_system_layout(sys)[0]
    return (np.ctypeslib.as_array(rp, (nf + 1,)).copy(),
            np.ctypeslib.as_array(col, (nnz.value,)).copy() if nnz.value else np.zeros(0, np.int32))


def lsw_set_potential(sys, V, fine_lo, fine_dims):
    lo = (C.c_int64 * 3)(*fine_lo)
    dims = (C.c_int64 * 3)(*fine_dims)
    check(lib().lsw_set_potential(sys, _ptr(V), lo, dims))


def lsw_apply_hamiltonian(sys, phi, hphi, e_kin=None, e_pot=None):
    check(lib().lsw_apply_hamiltonian(sys, _ptr(phi), _ptr(hphi), _ptr(e_kin), _ptr(e_pot)))


def lsw_combine(sys, M, phi_in, phi_out):
    """(M Phi)_a = L(a) sum_b M_ab phi_b for M on the pattern (FP64 device values)."""
    check(lib().lsw_combine(sys, _ptr(M), _ptr(phi_in), _ptr(phi_out)))


def lsw_lowdin_taylor(sys, S, phi_in, phi_out):
    """phi'_a = L(a) sum_b (3 delta_ab - S_ab) / 2 phi_b (first-order Taylor Loewdin step)."""
    check(lib().lsw_lowdin_taylor(sys, _ptr(S), _ptr(phi_in), _ptr(phi_out)))


def lsw_foe(sys, H, S, e_min, e_max, n_el, n_pl, de, Kp, K, tol=1e-10, max_bisect=200):
    """Fermi operator expansion on the pattern; returns (mu, E_BS, Tr K')."""
    mu, ebs, tr = C.c_double(), C.c_double(), C.c_double()
    check(lib().lsw_foe(sys, _ptr(H), _ptr(S), e_min, e_max, n_el, n_pl, de, tol, max_bisect, _ptr(Kp), _ptr(K),
                        C.byref(mu), C.byref(ebs), C.byref(tr)))
    return mu.value, ebs.value, tr.value


def lsw_add_confinement(sys, a, phi, hphi, e_conf=None):
    """hphi += L' a Q L phi (quartic confinement of each function's atom); e_conf = <phi|aQ|phi>."""
    check(lib().lsw_add_confinement(sys, _ptr(a), _ptr(phi), _ptr(hphi), _ptr(e_conf)))


def lsw_confinement_row(sys, atom, dim, m, b, bp, i):
    """Entries <chi^b_i|(x_dim - R_dim)^m|chi^b'_{i+l}>, l = -14..14 (host)."""
    out = np.zeros(29)
    check(lib().lsw_confinement_row(sys, atom, dim, m, b, bp, int(i), out.ctypes.data_as(_DP)))
    return out


def lsw_precondition(sys, a, eps, g, gprec, iters, res=None):
    """CG on L (-1/2 nabla^2 + a (r - R)^4 - eps) L gprec = -g, ``iters`` iterations per function."""
    check(lib().lsw_precondition(sys, _ptr(a), _ptr(eps), _ptr(g), _ptr(gprec), int(iters), _ptr(res)))


def lsw_apply_hamiltonian_noalloc(sys, phi, hphi, e_kin=None, e_pot=None):
    """H phi without any device allocation (workspace in the library's fixed 32 MiB
    device array); for callers that must not allocate.  See include/lsw.h."""
    check(lib().lsw_apply_hamiltonian_noalloc(sys, _ptr(phi), _ptr(hphi), _ptr(e_kin), _ptr(e_pot)))


def lsw_build_matrices(sys, phi, hphi, H, S):
    check(lib().lsw_build_matrices(sys, _ptr(phi), _ptr(hphi), _ptr(H), _ptr(S)))


def lsw_build_density(sys, phi, K, rho, fine_lo, fine_dims):
    """rho_j = sum_ab K_ab u_a(j) u_b(j) on the fine grid block (FP64, [z][y][x])."""
    lo = (C.c_int64 * 3)(*fine_lo)
    dims = (C.c_int64 * 3)(*fine_dims)
    check(lib().lsw_build_density(sys, _ptr(phi), _ptr(K), _ptr(rho), lo, dims))


def lsw_reformat(dst, src, shift, phi_src, phi_dst):
    """Move compressed support functions onto shifted atoms (shift: [n_atoms, 3] ints)."""
    sh = np.ascontiguousarray(np.asarray(shift, dtype=np.int32).reshape(-1))
    check(lib().lsw_reformat(dst, src, sh.ctypes.data_as(_I32P), _ptr(phi_src), _ptr(phi_dst)))


def lsw_workspace_bytes(sys):
    b = C.c_int64()
    check(lib().lsw_workspace_bytes(sys, C.byref(b)))
    return b.value


def lsw_sync(sys, timeout_s=60.0):
    check(lib().lsw_sync(sys, timeout_s))


def lsw_step_host(sys, phi_host, hphi_host, H_host, S_host, e_kin_host=None, e_pot_host=None):
    check(lib().lsw_step_host(sys, _ptr(phi_host), _ptr(hphi_host), _ptr(H_host), _ptr(S_host),
                              _ptr(e_kin_host), _ptr(e_pot_host)))


def lsw_set_option(sys, name, value):
    check(lib().lsw_set_option(sys, name.encode(), int(value)))


def lsw_system_set_stream(sys, stream):
    check(lib().lsw_system_set_stream(sys, stream))


def lsw_profile(sys, enable):
    check(lib().lsw_profile(sys, int(enable)))


def lsw_profile_read(sys):
    """{kind: (milliseconds, launches)} since the last read."""
    n = C.c_int32()
    ms = (C.c_double * 32)()
    cnt = (C.c_int64 * 32)()
    check(lib().lsw_profile_read(sys, 32, C.byref(n), ms, cnt))
    return {TRACE_KINDS[k]: (ms[k], cnt[k]) for k in range(min(n.value, len(TRACE_KINDS)))}


# ---------------------------------------------------------------- convenience wrapper

def make_desc(N, h, pos, r_loc, r_fine, nsf, pair_cutoff, pair_mode=0, lprime_margin=8.0,
              fine_mode=0, precision=LSW_FP64):
    """lsw_system_desc plus the numpy arrays it points to (kept alive by the caller)."""
    keep = [np.ascontiguousarray(pos, np.float64).reshape(-1), np.ascontiguousarray(r_loc, np.float64),
            np.ascontiguousarray(r_fine, np.float64), np.ascontiguousarray(nsf, np.int32)]
    d = lsw_system_desc()
    d.N = (C.c_int32 * 3)(*[int(x) for x in N])
    d.h = float(h)
    d.n_atoms = len(keep[1])
    d.pos = keep[0].ctypes.data_as(_DP)
    d.r_loc = keep[1].ctypes.data_as(_DP)
    d.r_fine = keep[2].ctypes.data_as(_DP)
    d.n_sf = keep[3].ctypes.data_as(_I32P)
    d.lprime_margin = float(lprime_margin)
    d.pair_cutoff = float(pair_cutoff)
    d.pair_mode = int(pair_mode)
    d.fine_mode = int(fine_mode)
    d.precision = int(precision)
    return d, keep


class System:
    """Owns one lsw_system (and its context unless one is given)."""

    def __init__(self, N, h, pos, r_loc, r_fine, nsf, pair_cutoff, pair_mode=0, lprime_margin=8.0,
                 fine_mode=0, precision=LSW_FP64, device=0, stream=None, ctx=None):
        self._own_ctx = ctx is None
        self.ctx = ctx if ctx is not None else lsw_ctx_create(device, stream)
        desc, keep = make_desc(N, h, pos, r_loc, r_fine, nsf, pair_cutoff, pair_mode, lprime_margin,
                               fine_mode, precision)
        try:
            self.sys = lsw_system_create(self.ctx, desc)
        except Exception:
            if self._own_ctx:
                lsw_ctx_destroy(self.ctx)
            raise
        self.precision = precision
        (self.n_sf, self.total_L, self.total_Lp, self.off_L, self.off_Lp,
         self.sf_atom) = lsw_system_layout(self.sys)
        self.row_ptr, self.col = lsw_pattern(self.sys)

    def keys(self, atom, region=LSW_REGION_L, part=LSW_PART_COARSE):
        return lsw_system_keys(self.sys, atom, region, part)

    def close(self):
        if getattr(self, "sys", None) is not None:
            lsw_system_destroy(self.sys)
            self.sys = None
        if getattr(self, "_own_ctx", False) and getattr(self, "ctx", None) is not None:
            lsw_ctx_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def lsw_save(sys, phi, path):
    check(lib().lsw_save(sys, _ptr(phi), os.fsencode(path)))


def lsw_load(ctx, path, phi=None):
    out = _P()
    check(lib().lsw_load(ctx, os.fsencode(path), C.byref(out), _ptr(phi)))
    return out


def lsw_load_phi(sys, path, phi):
    check(lib().lsw_load_phi(sys, os.fsencode(path), _ptr(phi)))


def lsw_measure_peaks(ctx):
    """(fp32 TFLOP/s, fp64 TFLOP/s, copy GB/s) measured on the context's GPU."""
    a, b, c = C.c_double(), C.c_double(), C.c_double()
    check(lib().lsw_measure_peaks(ctx, C.byref(a), C.byref(b), C.byref(c)))
    return a.value, b.value, c.value
