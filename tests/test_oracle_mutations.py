"""Plant plausible mistakes in the oracle (CPU only) and check that a pin fails.

Each mutant replaces one oracle function for the duration of one pin test; the
pin must then raise.  This shows the pins constrain the oracle rather than
restating it."""
import numpy as np
import pytest

import oracle.dpd as D
import oracle.motion as MD

import test_oracle_dpd as TD
import test_oracle_motion as TM


def fir_off_by_one(h, hist, z):
    y, nh = ORIG["fir"](h, hist, z)
    return np.concatenate([[0], y[:-1]]), nh


def fir_forgets_history(h, hist, z):
    return ORIG["fir"](h, np.zeros_like(hist), z)


def fir_conj_taps(h, hist, z):
    return ORIG["fir"](np.conj(h), hist, z)


def psi_wrong_power(x, order):
    return ORIG["psi"](x, order + 2 if order > 1 else order)


def erode_border_zero(b):
    H, W = b.shape
    p = np.zeros((H + 2, W + 2), np.uint8)
    p[1:-1, 1:-1] = b
    out = b.copy()
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            out = np.minimum(out, p[1 + dy:H + 1 + dy, 1 + dx:W + 1 + dx])
    return out


def threshold_ge(d, t=25):
    return (d >= t).astype(np.uint8)


def tiles_transposed(counts, tile=16):
    return ORIG["tile_records"](counts.T.copy(), tile)


ORIG = {"fir": D.fir, "psi": D.psi, "tile_records": MD.tile_records}

CASES = [
    (D, "fir", fir_off_by_one, lambda: TD.test_single_branch_is_closed_form_fir_p2()),
    (D, "fir", fir_forgets_history, lambda: TD.test_random_masks_restatement_p4(64, 10, 1)),
    (D, "fir", fir_conj_taps, lambda: TD.test_all_branches_active_p3()),
    (D, "psi", psi_wrong_power, lambda: TD.test_all_branches_active_p3()),
    (MD, "erode3x3", erode_border_zero, lambda: TM.test_morphology_matches_scipy_p10()),
    (MD, "threshold", threshold_ge, lambda: TM.test_threshold_is_strict()),
    (MD, "tile_records", tiles_transposed, lambda: TM.test_translated_rectangle_closed_form_p9()),
]


@pytest.mark.parametrize("mod,name,mutant,pin", CASES, ids=[c[2].__name__ for c in CASES])
def test_pin_catches_mutant(monkeypatch, mod, name, mutant, pin):
    monkeypatch.setattr(mod, name, mutant)
    with pytest.raises(AssertionError):
        pin()
