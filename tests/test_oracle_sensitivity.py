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
