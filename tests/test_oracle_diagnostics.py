"""Oracle pins for the diagnostics: the temporal power trace and the energy
spectrum of the fields (Sec. 6 power formula, resolved in tau or Omega).

For a Gaussian beam-pulse A = a0 exp(-r^2/w0^2) exp(-(1 + iC) tau^2/tau0^2)
(window >= 10 widths, well sampled, so grid sums equal the integrals to
rounding):
  P(tau)  = 1/2 c eps0 n a0^2 (pi w0^2 / 2) exp(-2 tau^2 / tau0^2)
  S(Omega_m) = 1/2 c eps0 n a0^2 (pi w0^2 / 2) |A~(Omega_m)|^2 dOmega / (2 pi),
  |A~(Omega)|^2 = pi tau0^2 / sqrt(1 + C^2) exp(-Omega^2 tau0^2 / (2 (1 + C^2))),
with dOmega = 2 pi / (nt dt); both sum to the energy (Parseval)."""
import math

import numpy as np
import pytest

import oracle
from paper_2609_08384_gb300 import workloads as wl

C0, EPS0 = wl.C0, wl.EPS0


def _beam_pulse(g, a0, w0, tau0, chirp=0.0, delay=0.0):
    x, y, t = g.axes()
    r2 = x[None, None, :] ** 2 + y[None, :, None] ** 2
    tt = (t - delay)[:, None, None]
    return (a0 * np.exp(-r2 / w0**2) * np.exp(-(1 + 1j * chirp) * tt**2 / tau0**2)).astype(np.complex128)


def _setup(chirp=0.0, delay=0.0):
    g = wl.Grid(64, 48, 256, 4e-6, 6e-6, 10e-15)
    fields = [wl.FieldParams(wl.LAM_SH, wl.N_SH), wl.FieldParams(wl.LAM_F, wl.N_F)]
    a = _beam_pulse(g, 3e7, 30e-6, 150e-15, chirp, delay)
    b = _beam_pulse(g, 1e7, 25e-6, 100e-15, -chirp, delay)
    return g, fields, [a, b], oracle.make_problem(g, fields, wl.D_EFF)


def test_power_trace_gaussian_closed_form_and_energy():
    g, fields, arrs, prob = _setup()
    p = oracle.power_trace(prob, arrs)
    e, _ = oracle.energy(prob, arrs)
    _, _, t = g.axes()
    for f, (a0, w0, tau0) in enumerate([(3e7, 30e-6, 150e-15), (1e7, 25e-6, 100e-15)]):
        ref = 0.5 * C0 * EPS0 * fields[f].n * a0**2 * (math.pi * w0**2 / 2) * np.exp(-2 * t**2 / tau0**2)
        assert np.max(np.abs(p[f] - ref)) < 1e-10 * ref.max()
        assert p[f].sum() * g.dt == pytest.approx(e[f], rel=1e-12)


@pytest.mark.parametrize("chirp", [0.0, 2.5])
def test_spectrum_gaussian_closed_form_and_parseval(chirp):
    g, fields, arrs, prob = _setup(chirp)
    s = oracle.spectrum(prob, arrs)
    e, _ = oracle.energy(prob, arrs)
    om = np.array([oracle.angular_freq(m, g.nt, g.dt) for m in range(g.nt)])
    d_om = 2 * math.pi / (g.nt * g.dt)
    for f, (a0, w0, tau0, c) in enumerate([(3e7, 30e-6, 150e-15, chirp), (1e7, 25e-6, 100e-15, -chirp)]):
        spec = math.pi * tau0**2 / math.sqrt(1 + c * c) * np.exp(-om**2 * tau0**2 / (2 * (1 + c * c)))
        ref = 0.5 * C0 * EPS0 * fields[f].n * a0**2 * (math.pi * w0**2 / 2) * spec * d_om / (2 * math.pi)
        assert np.max(np.abs(s[f] - ref)) < 1e-9 * ref.max()
        assert s[f].sum() == pytest.approx(e[f], rel=1e-12)


def test_spectrum_is_shift_invariant_and_power_trace_shifts():
    """A delay by an integer number of samples shifts the power trace by the
    same number of bins and leaves the spectrum unchanged."""
    g, fields, arrs, prob = _setup(1.0)
    g2, _, arrs2, _ = _setup(1.0, delay=17 * 10e-15)
    p, p2 = oracle.power_trace(prob, arrs), oracle.power_trace(prob, arrs2)
    s, s2 = oracle.spectrum(prob, arrs), oracle.spectrum(prob, arrs2)
    for f in range(2):
        assert np.allclose(np.roll(p[f], 17), p2[f], rtol=0, atol=1e-12 * p[f].max())
        assert np.allclose(s[f], s2[f], rtol=0, atol=1e-11 * s[f].max())
