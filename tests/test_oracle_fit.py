"""The oracle's indirect-learning fit (parity unpinned: the paper gives no fit
outcome); these check its composition, not its result."""
import numpy as np

import synth
from oracle import dpd as D
from oracle import fit as OF
from oracle import pa as PA


def test_one_iteration_is_the_plain_fit():
    """P_0 is the identity, so the first iteration drives the amplifier with x
    itself and trains exactly the plain fit."""
    w = synth.dpd_fit(n=2048)
    h1, curves, nmse = OF.ila_fit_iterative(w.x, iterations=1, steps=15)
    h0, losses = OF.ila_fit(w.x, steps=15)
    np.testing.assert_array_equal(h1, h0)
    np.testing.assert_array_equal(curves[0], losses)
    x = w.x.astype(np.complex128)
    e = PA.pa(D.dpd_stream(x, h0, (1, 3, 5, 7))) / PA.small_signal_gain() - x
    assert abs(nmse[0] - 10 * np.log10(np.sum(np.abs(e) ** 2) / np.sum(np.abs(x) ** 2))) < 1e-12


def test_plain_fit_lowers_the_loss():
    w = synth.dpd_fit(n=4096)
    _, losses = OF.ila_fit(w.x, steps=30)
    assert losses[-1] < losses[0]
