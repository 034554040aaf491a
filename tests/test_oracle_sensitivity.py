"""The oracle's pins catch plausible mistakes: each case plants one mistake in the
oracle (on the CPU, through monkeypatch) and checks that a pin that passes on the
correct oracle now fails.  A pin set that let such a mistake through would not pin
the oracle to the paper."""
import dataclasses

import numpy as np
import pytest

from oracle import hamiltonian as Hm
from tests import test_oracle_filters as TF
from tests import test_oracle_operator as TO


def _fails(fn, *args):
    with pytest.raises(AssertionError):
        fn(*args)


def test_magic_filter_window_shifted_by_one_tap(monkeypatch):
    # the alternative tap window l = -8..7 with the same values (reading R4's other case)
    bad = dataclasses.replace(TO.FT, magic_lo=TO.FT.magic_lo - 1)
    monkeypatch.setattr(TO, "FT", bad)
    _fails(TO.test_gaussian_potential_closed_form)


def test_kinetic_blocks_transposed(monkeypatch):
    # T_hg and T_gh exchanged (a transposed operand in the two-level kinetic operator)
    kin = dict(TF.FT.kin)
    kin["hg"], kin["gh"] = kin["gh"], kin["hg"]
    monkeypatch.setattr(TF, "FT", dataclasses.replace(TF.FT, kin=kin))
    _fails(TF.test_kinetic_blocks_two_routes)


def test_kinetic_block_sign_flipped(monkeypatch):
    # a wrong sign on the wavelet-wavelet block
    kin = dict(TO.FT.kin)
    kin["gg"] = -kin["gg"]
    monkeypatch.setattr(TF, "FT", dataclasses.replace(TF.FT, kin=kin))
    _fails(TF.test_kinetic_blocks_two_routes)


def test_kinetic_connection_coefficients_index_shifted(monkeypatch):
    # r_l read one index off (l -> l + 1) in the scaling-scaling block
    kin = dict(TO.FT.kin)
    kin["hh"] = np.roll(kin["hh"], 1)
    monkeypatch.setattr(TO, "FT", dataclasses.replace(TO.FT, kin=kin))
    _fails(TO.test_gaussian_kinetic_energy)


def test_potential_slice_off_by_one(monkeypatch):
    # V taken one fine point off along x: the dense brute force indexes V on its own
    real = Hm.v_slice

    def shifted(V, V_lo, start, shape):
        return real(V, [V_lo[0] + 1, V_lo[1], V_lo[2]], start, shape)

    monkeypatch.setattr(Hm, "v_slice", shifted)
    _fails(TO.test_separable_oracle_equals_dense_matrices, 5, 6, 1.2, 0.6)


def test_high_pass_sign_in_synthesis_only(monkeypatch):
    # g negated in the synthesis but not in the analysis: analysis o synthesis != I
    real = Hm.synthesis3d
    bad = dataclasses.replace(TO.FT, g=-TO.FT.g)

    def wrong(c, lo, F):
        return real(c, lo, bad)

    monkeypatch.setattr(Hm, "synthesis3d", wrong)
    _fails(TO.test_analysis_inverts_synthesis_and_keeps_norm)


# ------------------------------------------------------------------ density (Eq. density)

from oracle import density as Dn
from tests import test_oracle_density as TD


def test_density_block_of_one_function_shifted(monkeypatch):
    # the real-space block of function 1 placed one fine point off along x
    real = Dn.realspace

    def shifted(geo, f, phi_f, F):
        u, st = real(geo, f, phi_f, F)
        return u, [st[0] + 1, st[1], st[2]] if f == 1 else st

    monkeypatch.setattr(Dn, "realspace", shifted)
    _fails(TD.test_density_equals_dense_matrices, 5, 6, 1.2, 0.6)


def test_density_lower_triangle_dropped(monkeypatch):
    # only the entries a <= b of the kernel summed (a symmetry folded without the factor 2)
    real = Dn.pattern_entries

    def upper(row_ptr, col, K):
        return [(a, b, k) for a, b, k in real(row_ptr, col, K) if a <= b]

    monkeypatch.setattr(Dn, "pattern_entries", upper)
    _fails(TD.test_density_trace_identity_with_potential_matrix)


def test_density_square_instead_of_pair_product(monkeypatch):
    # u_a^2 in place of u_a u_b
    real = Dn.accumulate

    def squares(fields, entries, lo, dims):
        return real(fields, [(a, a, k) for a, b, k in entries], lo, dims)

    monkeypatch.setattr(Dn, "accumulate", squares)
    _fails(TD.test_density_of_two_gaussians_closed_form)


def test_density_magic_filter_reversed(monkeypatch):
    # the magic filter applied as a correlation (taps reversed) in the real-space values
    real = Dn.realspace_block

    def reversed_w(c, lo, F):
        return real(c, lo, dataclasses.replace(F, magic=F.magic[::-1].copy()))

    monkeypatch.setattr(Dn, "realspace_block", reversed_w)
    _fails(TD.test_density_of_two_gaussians_closed_form)


# ------------------------------------------------------------------ confinement (Eq. precond)

from oracle import confinement as Cf
from tests import test_oracle_confinement as TC


def test_confinement_moment_overlaps_index_shifted(monkeypatch):
    # F^p(l) read one index off
    bad = dataclasses.replace(TC.FT, movl=np.roll(TC.FT.movl, 1, axis=1))
    monkeypatch.setattr(TC, "FT", bad)
    Cf._BLOCKS.clear()
    try:
        _fails(TC.test_quartic_block_gaussian_moments_1d, 2)
    finally:
        Cf._BLOCKS.clear()


def test_confinement_scaling_wavelet_coupling_dropped(monkeypatch):
    # the 1D operator applied type by type, without the scaling <-> wavelet blocks
    real = Cf._apply_1d

    def diagonal_only(arr, axis, blocks):
        z = {k: (v if k[0] == k[1] else np.zeros_like(v)) for k, v in blocks.items()}
        return real(arr, axis, z)

    monkeypatch.setattr(Cf, "_apply_1d", diagonal_only)
    _fails(TC.test_confinement_assembly_against_kronecker_products)


def test_confinement_wavelet_filter_in_place_of_scaling(monkeypatch):
    # the wavelet-wavelet block built with h in place of g (an operand swapped in the 1D blocks)
    real = Cf.quartic_block_1d

    def swapped(m, b, bp, i_idx, j_idx, c, h, F):
        return real(m, 0 if (b, bp) == (1, 1) else b, 0 if (b, bp) == (1, 1) else bp, i_idx, j_idx, c, h, F)

    monkeypatch.setattr(Cf, "quartic_block_1d", swapped)
    _fails(TC.test_quartic_blocks_by_cascade_quadrature)


def test_confinement_cross_terms_dropped(monkeypatch):
    # (r - R)^4 taken as sum_d X_d^4 only (the 2 X_d^2 X_e^2 terms lost)
    real = Cf._blocks

    def no_square(d_lo, n, c, h, F):
        b = real(d_lo, n, c, h, F)
        return {2: {k: np.zeros_like(v) for k, v in b[2].items()}, 4: b[4]}

    monkeypatch.setattr(Cf, "_blocks", no_square)
    _fails(TC.test_confinement_gaussian_closed_form_3d)


def test_precond_kinetic_sign_flipped(monkeypatch):
    # +1/2 nabla^2 in place of -1/2 nabla^2 in the preconditioning operator
    real = Hm.kinetic3d
    monkeypatch.setattr(Hm, "kinetic3d", lambda c, h, F: -real(c, h, F))
    _fails(TC.test_precond_operator_against_explicit_matrices)


# ------------------------------------------------------------------ sparse combinations (Loewdin)

from oracle import combine as Cb
from tests import test_oracle_combine as TB


def test_combine_matrix_transposed(monkeypatch):
    # M_beta,alpha used in row alpha (the transposed operand)
    real = Cb.combine

    def transposed(geo, M, phi, rows=None):
        rp, col = geo.row_ptr, geo.col
        pos = {(a, int(col[k])): k for a in range(len(rp) - 1) for k in range(rp[a], rp[a + 1])}
        Mt = np.array([M[pos[(int(col[k]), a)]] for a in range(len(rp) - 1) for k in range(rp[a], rp[a + 1])])
        return real(geo, Mt, phi, rows)

    monkeypatch.setattr(Cb, "combine", transposed)
    _fails(TB.test_combination_is_the_adjoint_of_the_scalar_products, 5, 3, 1.3)


def test_combine_placed_at_the_wrong_origin(monkeypatch):
    # phi_beta placed at L(alpha)'s origin instead of its own
    real_place = Cb._H._place

    def misplaced(dst, dst_lo, src, src_lo):
        return real_place(dst, dst_lo, src, dst_lo)

    monkeypatch.setattr(Cb._H, "_place", misplaced)
    _fails(TB.test_combination_is_the_adjoint_of_the_scalar_products, 5, 3, 1.3)


def test_taylor_step_with_the_wrong_sign(monkeypatch):
    # (3I + S)/2 in place of (3I - S)/2
    real = Cb.combine

    def plus(geo, M, phi, rows=None):
        rp, col = geo.row_ptr, geo.col
        diag = np.array([float(int(col[k]) == a) for a in range(len(rp) - 1) for k in range(rp[a], rp[a + 1])])
        return real(geo, 3.0 * diag - M, phi, rows)       # (3I - S)/2 -> (3I + S)/2 when M = (3I - S)/2

    monkeypatch.setattr(Cb, "combine", plus)
    _fails(TB.test_taylor_loewdin_error_is_second_order)


# ------------------------------------------------------------------ Fermi operator expansion

from oracle import foe as Fo
from tests import test_oracle_foe as TF2


def test_foe_recursion_without_the_factor_two(monkeypatch):
    # t^{j+1} = H t^j - t^{j-1} (the Chebyshev recursion's factor 2 dropped)
    def bad(Ht, c, pattern=None):
        n = len(Ht)
        K = np.zeros((n, n))
        for l in range(n):
            t_prev = np.zeros(n)
            t_prev[l] = 1.0
            k = 0.5 * c[0] * t_prev
            t = Ht @ t_prev
            k = k + c[1] * t
            for j in range(2, len(c)):
                t_prev, t = t, Ht @ t - t_prev
                k = k + c[j] * t
            K[:, l] = k
        return K

    monkeypatch.setattr(Fo, "kernel_prime", bad)
    _fails(TF2.test_kernel_equals_exact_diagonalization)


def test_foe_zeroth_coefficient_not_halved(monkeypatch):
    real = Fo.chebyshev_value

    monkeypatch.setattr(Fo, "chebyshev_value", lambda c, x: real(c, x) + 0.5 * c[0])
    _fails(TF2.test_chebyshev_interpolation_and_evaluation)


def test_foe_kernel_not_transformed_back(monkeypatch):
    # K = K' (the S^-1/2 ... S^-1/2 back-transform forgotten)
    real_foe = Fo.foe

    def no_back(H, S, n_el, n_pl, de, **kw):
        r = real_foe(H, S, n_el, n_pl, de, **kw)
        r["K"] = r["Kp"]
        return r

    monkeypatch.setattr(Fo, "foe", no_back)
    _fails(TF2.test_kernel_equals_exact_diagonalization)


# ------------------------------------------------------------------ gradient (Eq. gradient)

from oracle import gradient as Gr
from tests import test_oracle_gradient as TG


def _patched_gradient(half=0.5, sym=True):
    def energy_gradient(geo, phi, hphi, K, S, sinv="exact"):
        n = len(geo.sf_atom)
        Phi = np.stack([Gr.to_box(geo, geo.L[geo.sf_atom[f]], phi[f]) for f in range(n)])
        HPhi = np.stack([Gr.to_box(geo, geo.Lp[geo.sf_atom[f]], hphi[f]) for f in range(n)])
        D = np.tensordot(np.asarray(K), HPhi, axes=([1], [0]))
        Chi = np.tensordot(np.asarray(S), D, axes=([1], [0]))
        Lam = np.array([[float(np.sum(Phi[a] * Chi[b])) for b in range(n)] for a in range(n)])
        M = half * np.linalg.inv(S) @ ((Lam + Lam.T) if sym else 2.0 * Lam)
        G = Chi - np.tensordot(M, Phi, axes=([1], [0]))
        return {f: Gr.from_box(geo, geo.L[geo.sf_atom[f]], G[f]) for f in range(n)}
    return energy_gradient


def test_gradient_without_the_half(monkeypatch):
    monkeypatch.setattr(Gr, "energy_gradient", _patched_gradient(half=1.0))
    _fails(TG.test_gradient_is_tangent_to_the_orthonormality_constraint)


def test_gradient_with_unsymmetrized_multipliers(monkeypatch):
    # 2 Lambda in place of Lambda + Lambda^T
    monkeypatch.setattr(Gr, "energy_gradient", _patched_gradient(sym=False))
    _fails(TG.test_gradient_is_the_derivative_along_tangent_directions, 3)
