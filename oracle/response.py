"""Tapered frequency response |H^alpha| (Eq. Halpha, Sec. 7.1) and the amplitude
spectrum of the modulated Gaussian incident pulse.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

The probe series J_n = J(t_n), t_n = n dt (n = 1..N), is tapered by a cosine window on
its last fraction (reading R15: w_n = 1 for n <= n_flat = N - floor(taper N), else
(1 + cos(pi (n - n_flat) / (N - n_flat))) / 2), transformed by the plain sum
    j(f) = dt sum_n w_n J_n exp(-2 pi i f t_n),
and divided by eps0 (eps_r - 1) |e^i(f)| (eps0 = 1).
"""
import numpy as np


def taper_weights(n_steps, taper):
    n_flat = n_steps - int(np.floor(taper * n_steps))
    n = np.arange(1, n_steps + 1)
    w = np.ones(n_steps)
    if n_steps > n_flat:
        tail = n > n_flat
        w[tail] = 0.5 * (1.0 + np.cos(np.pi * (n[tail] - n_flat) / (n_steps - n_flat)))
    return w


def tapered_dft(J, dt, taper, freqs):
    """j(f) for J [N][...]: returns [n_freq][...] complex."""
    N = J.shape[0]
    w = taper_weights(N, taper)
    t = dt * np.arange(1, N + 1)
    out = []
    for f in np.asarray(freqs, float):
        ph = np.exp(-2j * np.pi * f * t)
        out.append(dt * np.tensordot(w * ph, J, axes=(0, 0)))
    return np.array(out)


def incident_amplitude(f, f_c, sigma_t):
    """|e^i(f)| of sin(2 pi f_c t) exp(-t^2 / (2 sigma_t^2)) (Fourier transform of a
    Gaussian shifted by +-f_c)."""
    f = np.asarray(f, float)
    g = 2.0 * np.pi ** 2 * sigma_t ** 2
    return sigma_t * np.sqrt(2.0 * np.pi) / 2.0 * np.abs(np.exp(-g * (f - f_c) ** 2)
                                                        - np.exp(-g * (f + f_c) ** 2))


def frequency_response(J, dt, taper, eps_probe, f_c, sigma_t, freqs):
    """|H^alpha| [n_freq][n_probe][3] from J [N][n_probe][3] (Eq. Halpha)."""
    jf = tapered_dft(J, dt, taper, freqs)
    ei = incident_amplitude(freqs, f_c, sigma_t)
    e = np.asarray(eps_probe, float)
    return np.abs(jf) / ((e - 1.0)[None, :, None] * ei[:, None, None])
