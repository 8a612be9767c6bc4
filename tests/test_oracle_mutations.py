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


# ------------------------------------------- amplifier model and Adam fit ----
import oracle.fit as OF  # noqa: E402
import oracle.pa as PA  # noqa: E402

import test_oracle_pa_fit_pins as TP  # noqa: E402


def pm_sign_flipped(r, alpha_p, beta_p):
    return -ORIG_PA["saleh_pm"](r, alpha_p, beta_p)


def pm_without_beta(r, alpha_p, beta_p):
    return alpha_p * r * r


def am_linear_beta(r, alpha_a, beta_a):
    return alpha_a * r / (1.0 + beta_a * r)


def pa_memory_first(x, saleh=TP.SALEH, memory=(1.0, 0.1, -0.05)):
    x = np.asarray(x, np.complex128)
    s = np.zeros_like(x)
    for i, c in enumerate(memory):
        s[i:] += c * x[:len(x) - i]
    return ORIG_PA["pa"](s, saleh, (1.0,))


def pa_phase_from_output(x, saleh=TP.SALEH, memory=(1.0, 0.1, -0.05)):
    x = np.asarray(x, np.complex128)
    aa, ba, ap, bp = saleh
    r = np.abs(x)
    a = ORIG_PA["saleh_am"](r, aa, ba)
    v = a * np.exp(1j * (np.angle(x) + ORIG_PA["saleh_pm"](a, ap, bp)))
    y = np.zeros_like(v)
    for i, c in enumerate(memory):
        y[i:] += c * v[:len(v) - i]
    return y


def _adam_variant(no_bias_correction=False, eps_inside=False, joint_moment=False):
    def adam_fit(u, target, h0, orders, steps, lr, betas=(0.9, 0.999), eps=1e-8):
        h = np.array(h0, np.complex128)
        m = np.zeros(h.shape + (2,))
        v = np.zeros(h.shape + (2,))
        losses = []
        N = len(u)
        for t in range(1, steps + 1):
            out = D.dpd_stream(u, h, orders)
            r = out - target
            losses.append(float(np.mean(r.real ** 2 + r.imag ** 2)))
            _, gh = D.dpd_stream_backward(u, h, orders, 2.0 * r / N)
            gr = np.stack([gh.real, gh.imag], axis=-1)
            m = betas[0] * m + (1 - betas[0]) * gr
            g2 = np.abs(gh)[..., None] ** 2 * np.ones(2) if joint_moment else gr * gr
            v = betas[1] * v + (1 - betas[1]) * g2
            mh = m if no_bias_correction else m / (1 - betas[0] ** t)
            vh = v if no_bias_correction else v / (1 - betas[1] ** t)
            den = np.sqrt(vh + eps) if eps_inside else np.sqrt(vh) + eps
            step = lr * mh / den
            h = h - (step[..., 0] + 1j * step[..., 1])
        return h, np.array(losses)
    return adam_fit


ORIG_PA = {"saleh_pm": PA.saleh_pm, "saleh_am": PA.saleh_am, "pa": PA.pa}

PA_CASES = [
    (PA, "saleh_pm", pm_sign_flipped, lambda: TP.test_am_pm_phases_add_to_saturation_phase(0.5)),
    (PA, "saleh_pm", pm_without_beta, lambda: TP.test_am_pm_phases_add_to_saturation_phase(2.0)),
    (PA, "saleh_am", am_linear_beta, lambda: TP.test_am_am_symmetry_under_r_to_one_over_beta_r(0.5)),
    (PA, "pa", pa_memory_first, lambda: TP.test_memory_taps_follow_the_nonlinearity()),
    (PA, "pa", pa_phase_from_output, lambda: TP.test_am_pm_phases_add_to_saturation_phase(0.5)),
    (OF, "adam_fit", _adam_variant(no_bias_correction=True), lambda: TP.test_adam_one_tap_hand_expanded()),
    (OF, "adam_fit", _adam_variant(eps_inside=True), lambda: TP.test_adam_matches_torch_optim_two_branches()),
    (OF, "adam_fit", _adam_variant(joint_moment=True), lambda: TP.test_adam_one_tap_hand_expanded()),
]


@pytest.mark.parametrize("mod,name,mutant,pin", PA_CASES,
                         ids=["pm_sign_flipped", "pm_without_beta", "am_linear_beta", "pa_memory_first",
                              "pa_phase_from_output", "adam_no_bias_correction", "adam_eps_inside_sqrt",
                              "adam_joint_second_moment"])
def test_pa_fit_pin_catches_mutant(monkeypatch, mod, name, mutant, pin):
    monkeypatch.setattr(mod, name, mutant)
    with pytest.raises(AssertionError):
        pin()


def test_adam_variant_without_mistake_passes_the_pins(monkeypatch):
    """The mutant factory itself, with no mistake planted, passes both Adam pins."""
    monkeypatch.setattr(OF, "adam_fit", _adam_variant())
    TP.test_adam_one_tap_hand_expanded()
    TP.test_adam_matches_torch_optim_two_branches()
