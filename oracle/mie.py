"""Mie series for plane-wave scattering by the unit sphere (oracle; test infrastructure).

Not in the paper; the textbook closed form used to pin the method.  With the e^{-i omega t}
convention of Sec. 1 (outgoing h_n^(1)), incident direction d and theta = angle(x^, d):

    sound-soft:  u_inf = (i/kappa) sum_n (2n+1) [j_n(kappa)/h_n(kappa)] P_n(cos theta)
    sound-hard:  u_inf = (i/kappa) sum_n (2n+1) [j_n'(kappa)/h_n'(kappa)] P_n(cos theta)

h_n = j_n + i y_n; truncation n <= kappa + 4 kappa^(1/3) + 10 (plus 10 more terms).
"""
from __future__ import annotations

import numpy as np
from scipy.special import eval_legendre, spherical_jn, spherical_yn


def mie_far_field(kappa, xhat, d=(0.0, 0.0, 1.0), hard=False):
    xhat = np.atleast_2d(np.asarray(xhat, float))
    d = np.asarray(d, float) / np.linalg.norm(d)
    c = np.clip(xhat @ d, -1.0, 1.0)
    nmax = int(kappa + 4 * kappa ** (1 / 3) + 20)
    out = np.zeros(c.shape, dtype=complex)
    for n in range(nmax + 1):
        if hard:
            j = spherical_jn(n, kappa, derivative=True)
            h = j + 1j * spherical_yn(n, kappa, derivative=True)
        else:
            j = spherical_jn(n, kappa)
            h = j + 1j * spherical_yn(n, kappa)
        out += (2 * n + 1) * (j / h) * eval_legendre(n, c)
    return 1j / kappa * out


def mie_scattered_field(kappa, x, d=(0.0, 0.0, 1.0), hard=False):
    """Scattered field u_s at points x (n, 3) outside the unit sphere, for the plane wave of direction d:
    with theta = angle(x, d) and r = |x|,
        sound-soft:  u_s = -sum_n (2n+1) i^n [j_n(kappa) / h_n(kappa)] h_n(kappa r) P_n(cos theta)
        sound-hard:  u_s = -sum_n (2n+1) i^n [j_n'(kappa) / h_n'(kappa)] h_n(kappa r) P_n(cos theta)
    (the expansion of the incident wave in spherical waves, u_inc = sum (2n+1) i^n j_n(kappa r) P_n)."""
    x = np.atleast_2d(np.asarray(x, float))
    d = np.asarray(d, float) / np.linalg.norm(d)
    r = np.linalg.norm(x, axis=1)
    c = np.clip((x @ d) / r, -1.0, 1.0)
    nmax = int(kappa * r.max() + 4 * (kappa * r.max()) ** (1 / 3) + 20)
    out = np.zeros(r.shape, dtype=complex)
    for n in range(nmax + 1):
        if hard:
            a = spherical_jn(n, kappa, derivative=True) / (spherical_jn(n, kappa, derivative=True)
                                                           + 1j * spherical_yn(n, kappa, derivative=True))
        else:
            a = spherical_jn(n, kappa) / (spherical_jn(n, kappa) + 1j * spherical_yn(n, kappa))
        hn = spherical_jn(n, kappa * r) + 1j * spherical_yn(n, kappa * r)
        out -= (2 * n + 1) * (1j ** n) * a * hn * eval_legendre(n, c)
    return out
