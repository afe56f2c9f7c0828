"""Far-field pattern of a computed boundary density (oracle; test infrastructure).

Sec. 1 defines u_inf by u_s(x) = exp(i kappa |x|)/|x| (u_inf(x^) + O(1/|x|)).  From the
representations of Sec. 2 (with the sign of the single layer term that Green's formula gives under
outward normals: u_s = -SL(du/dn) for sound-soft, u_s = DL(u) for sound-hard) and the asymptotics
G(x, y) ~ exp(i kappa |x|)/(4 pi |x|) exp(-i kappa x^.y):

    sound-soft:  u_inf(x^) = -1/(4 pi) int exp(-i kappa x^.y) t(y) dsigma_y
    sound-hard:  u_inf(x^) = -i kappa/(4 pi) int (x^.n_y) exp(-i kappa x^.y) u(y) dsigma_y

evaluated with the 4x4 Gauss rule on every element.
"""
from __future__ import annotations

import numpy as np

from .assemble import ElementRules


def density_at_points(space, coeff, rules: ElementRules):
    """Values of the discrete function with global coefficients coeff (N,) or (N, R) at all Gauss
    points: (npts,) or (npts, R)."""
    cX = np.asarray(coeff)[space.x2g]
    loc = cX[space.l2x[rules.pts.e]]                 # (npts, nloc[, R])
    if loc.ndim == 2:
        return np.einsum("pk,pk->p", rules.pts.phi, loc)
    return np.einsum("pk,pkr->pr", rules.pts.phi, loc)


def far_field(space, kappa, coeff, xhat, hard: bool, rules: ElementRules | None = None):
    """u_inf at unit directions xhat (n_dir, 3) for density coefficients (N,) -> (n_dir,)."""
    rules = rules or ElementRules(space)
    pts = rules.pts
    wq = np.tile(rules.w, space.mesh.E)
    dens = density_at_points(space, coeff, rules)
    xhat = np.atleast_2d(xhat)
    ph = np.exp(-1j * kappa * (xhat @ pts.x.T))        # (n_dir, npts)
    if hard:
        return (-1j * kappa / (4 * np.pi)) * (ph * (xhat @ pts.n.T)) @ (wq * dens)
    return (-1.0 / (4 * np.pi)) * ph @ (wq * pts.a * dens)


def potential(space, kappa, coeff, points, hard: bool, rules: ElementRules | None = None):
    """The scattered field at points outside the scatterer (the representations of Sec. 2, Sec. 5.3's
    potential evaluation), summed directly over the 4x4 Gauss points of every element:
        sound-soft:  u_s(x) = -SL(t)(x) = -int G(x, y) t(y) dsigma_y
        sound-hard:  u_s(x) =  DL(u)(x) =  int dG/dn_y(x, y) u(y) dsigma_y,
    dG/dn_y = G'(r)/r (y - x).n_y, G'(r)/r = G (i kappa r - 1)/r^2; coeff (N,) -> (n_points,)."""
    rules = rules or ElementRules(space)
    pts = rules.pts
    wq = np.tile(rules.w, space.mesh.E)
    dens = density_at_points(space, coeff, rules)
    X = np.atleast_2d(np.asarray(points, float))
    out = np.zeros(X.shape[0], dtype=complex)
    for i, x in enumerate(X):
        v = pts.x - x                                   # y - x
        r = np.linalg.norm(v, axis=1)
        G = np.exp(1j * kappa * r) / (4 * np.pi * r)
        if hard:
            dGn = G * (1j * kappa * r - 1.0) / r ** 2 * np.sum(v * pts.n, axis=1)   # a dG/dn_y
            out[i] = np.sum(wq * dGn * dens)
        else:
            out[i] = -np.sum(wq * pts.a * G * dens)
    return out
