"""Synthetic power amplifier for the predistorter fit (oracle; test infrastructure).

Memoryless Saleh model followed by a short memory FIR:

    A(r)   = alpha_a r / (1 + beta_a r^2)        (AM/AM)
    Phi(r) = alpha_p r^2 / (1 + beta_p r^2)      (AM/PM)
    v[n]   = A(|x[n]|) exp(j (arg x[n] + Phi(|x[n]|)))
    y[n]   = sum_i c_i v[n - i]                  (zeros before the first sample)

The fit normalises by the small-signal gain G = alpha_a * sum_i c_i.

Pins (tests): A(r) = A(1/(beta_a r)) and Phi(r) + Phi(1/(beta_p r)) =
alpha_p / beta_p at large and small amplitudes, the small-signal limits, the
AM/AM peak at r = 1/sqrt(beta_a), the sign of the phase shift, and the
memory taps acting after the nonlinearity (numpy.convolve of the memoryless
output).
"""
from __future__ import annotations

import numpy as np


def saleh_am(r, alpha_a, beta_a):
    return alpha_a * r / (1.0 + beta_a * r * r)


def saleh_pm(r, alpha_p, beta_p):
    return alpha_p * r * r / (1.0 + beta_p * r * r)


def pa(x, saleh=(2.1587, 1.1517, 4.0033, 9.1040), memory=(1.0, 0.1, -0.05)):
    x = np.asarray(x, np.complex128)
    aa, ba, ap, bp = saleh
    r = np.abs(x)
    v = saleh_am(r, aa, ba) * np.exp(1j * (np.angle(x) + saleh_pm(r, ap, bp)))
    y = np.zeros_like(v)
    for i, c in enumerate(memory):
        y[i:] += c * v[:len(v) - i]
    return y


def small_signal_gain(saleh=(2.1587, 1.1517, 4.0033, 9.1040), memory=(1.0, 0.1, -0.05)):
    return saleh[0] * float(np.sum(memory))
