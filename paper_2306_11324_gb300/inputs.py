"""Seeded synthetic inputs: scatterer geometries, directions and random vectors.

This module is shared by the CUDA path's tests and benchmark and by the CPU oracle. It builds input
data only (NURBS control nets, unit directions, seeded random vectors); none of the boundary element
arithmetic (basis evaluation, quadrature, kernels, assembly, solves) lives here.

Geometry conventions (Sec. 3.2, patch maps F_j : [0,1]^2 -> Gamma_j given as NURBS):
  * a patch is ``NurbsPatch(p1, p2, knots1, knots2, ctrl, weights)`` with ``ctrl`` of shape
    (k1, k2, 3) and ``weights`` of shape (k1, k2); index j1 runs along the first parameter s;
  * patches of one scatterer meet conformingly: a shared edge has the same parametrisation from both
    sides, up to reversal, as Sec. 3.2 requires for the continuous space;
  * d_s F x d_t F points out of the enclosed volume.
"""
from __future__ import annotations

import dataclasses
from math import comb

import numpy as np


@dataclasses.dataclass
class NurbsPatch:
    p1: int
    p2: int
    knots1: np.ndarray
    knots2: np.ndarray
    ctrl: np.ndarray      # (k1, k2, 3)
    weights: np.ndarray   # (k1, k2)

    @property
    def k1(self) -> int:
        return self.ctrl.shape[0]

    @property
    def k2(self) -> int:
        return self.ctrl.shape[1]


# --------------------------------------------------------------------------------------------
# Exact unit sphere as six rational tensor-product patches in cube topology.
#
# A conforming cube layout of biquadratic rational patches on the sphere does not exist (the
# bilinear quaternion lift of such patches would be a global section of the Hopf fibration), so the
# lowest degree exact construction is used: degree (4,4).  Each face is the inverse stereographic
# image of a planar rational biquadratic patch whose four edges are the circular arcs that the
# stereographic projection makes of the cube's great-circle edges; the other five faces are rotated
# copies of the +z face.  The face is symmetric under its eight square symmetries, so rotated
# copies meet with identical edge parametrisations.
# --------------------------------------------------------------------------------------------

_CUBE_FRAMES = (
    # (normal, u, v) with u x v = normal; face corner (i, j) sits at (normal + (2i-1)u + (2j-1)v)/sqrt3
    ((1, 0, 0), (0, 1, 0), (0, 0, 1)),
    ((-1, 0, 0), (0, 0, 1), (0, 1, 0)),
    ((0, 1, 0), (0, 0, 1), (1, 0, 0)),
    ((0, -1, 0), (1, 0, 0), (0, 0, 1)),
    ((0, 0, 1), (1, 0, 0), (0, 1, 0)),
    ((0, 0, -1), (0, 1, 0), (1, 0, 0)),
)


def _bernstein_product(f: np.ndarray, g: np.ndarray) -> np.ndarray:
    """Bernstein coefficients of the product of two tensor Bernstein polynomials."""
    p, q = f.shape[0] - 1, g.shape[0] - 1
    h = np.zeros((p + q + 1, p + q + 1))
    for i in range(p + 1):
        for j in range(p + 1):
            for k in range(q + 1):
                for l in range(q + 1):
                    c = (comb(p, i) * comb(q, k) / comb(p + q, i + k)) * \
                        (comb(p, j) * comb(q, l) / comb(p + q, j + l))
                    h[i + k, j + l] += f[i, j] * g[k, l] * c
    return h


def _sphere_face_homogeneous(center_weight: float = 1.5) -> np.ndarray:
    """Homogeneous Bernstein net (5, 5, 4) = (wX, wY, wZ, w) of the +z face of the unit sphere."""
    s3 = np.sqrt(3.0)
    rho = 1.0 / (s3 + 1.0)                 # stereographic image of the corner (1,1,1)/sqrt3
    a1 = rho + rho * rho / (rho + 1.0)     # tangent intersection of the edge arc
    w1 = (rho + 1.0) / np.sqrt(2.0)        # cosine of the arc's half angle
    net = {
        (0, 0): (-rho, -rho, 1.0), (2, 0): (rho, -rho, 1.0),
        (0, 2): (-rho, rho, 1.0), (2, 2): (rho, rho, 1.0),
        (1, 0): (0.0, -a1, w1), (1, 2): (0.0, a1, w1),
        (0, 1): (-a1, 0.0, w1), (2, 1): (a1, 0.0, w1),
        (1, 1): (0.0, 0.0, center_weight),
    }
    A = np.zeros((3, 3)); B = np.zeros((3, 3)); W = np.zeros((3, 3))
    for (i, j), (x, y, w) in net.items():
        A[i, j], B[i, j], W[i, j] = x * w, y * w, w
    # inverse stereographic projection from the south pole: (a,b) -> (2a, 2b, 1-a^2-b^2)/(1+a^2+b^2)
    AA, BB, WW = _bernstein_product(A, A), _bernstein_product(B, B), _bernstein_product(W, W)
    X = 2.0 * _bernstein_product(A, W)
    Y = 2.0 * _bernstein_product(B, W)
    Z = WW - AA - BB
    H = WW + AA + BB
    return np.stack([X, Y, Z, H], axis=-1)


def unit_sphere_patches() -> list[NurbsPatch]:
    """Unit sphere as 6 exact rational Bezier patches of degree (4,4), cube topology."""
    H = _sphere_face_homogeneous()
    knots = np.array([0.0] * 5 + [1.0] * 5)
    patches = []
    for n, u, v in _CUBE_FRAMES:
        R = np.stack([np.array(u, float), np.array(v, float), np.array(n, float)], axis=1)
        w = H[..., 3].copy()
        ctrl = (H[..., :3] / w[..., None]) @ R.T
        patches.append(NurbsPatch(4, 4, knots.copy(), knots.copy(), ctrl, w))
    return patches


# --------------------------------------------------------------------------------------------
# Refinement of a control net by knot insertion (input preparation for the deformed sphere).
# --------------------------------------------------------------------------------------------

def _insert_knot_curve(knots: np.ndarray, p: int, P: np.ndarray, x: float):
    """Insert knot x once into a curve with homogeneous control points P (k, d); Boehm's rule."""
    k = P.shape[0]
    s = int(np.searchsorted(knots, x, side="right")) - 1
    Q = np.zeros((k + 1, P.shape[1]))
    for i in range(k + 1):
        if i <= s - p:
            Q[i] = P[i]
        elif i > s:
            Q[i] = P[i - 1]
        else:
            a = (x - knots[i]) / (knots[i + p] - knots[i])
            Q[i] = a * P[i] + (1.0 - a) * P[i - 1]
    return np.insert(knots, s + 1, x), Q


def refine_patch(patch: NurbsPatch, spans: int) -> NurbsPatch:
    """Insert the knots j/spans (j=1..spans-1) once in both directions; the surface is unchanged."""
    Hw = np.concatenate([patch.ctrl * patch.weights[..., None], patch.weights[..., None]], axis=-1)
    new = [j / spans for j in range(1, spans)]
    k1 = patch.knots1.copy()
    rows = []
    for j2 in range(Hw.shape[1]):
        kk, P = patch.knots1.copy(), Hw[:, j2, :]
        for x in new:
            kk, P = _insert_knot_curve(kk, patch.p1, P, x)
        rows.append(P)
        k1 = kk
    Hw = np.stack(rows, axis=1)
    k2 = patch.knots2.copy()
    cols = []
    for j1 in range(Hw.shape[0]):
        kk, P = patch.knots2.copy(), Hw[j1, :, :]
        for x in new:
            kk, P = _insert_knot_curve(kk, patch.p2, P, x)
        cols.append(P)
        k2 = kk
    Hw = np.stack(cols, axis=0)
    w = Hw[..., 3]
    return NurbsPatch(patch.p1, patch.p2, k1, k2, Hw[..., :3] / w[..., None], w.copy())


def fibonacci_directions(n: int) -> np.ndarray:
    """n unit vectors on a Fibonacci sphere: z_i = 1-(2i+1)/n, phi_i = i*pi*(3-sqrt5)."""
    i = np.arange(n, dtype=np.float64)
    z = 1.0 - (2.0 * i + 1.0) / n
    phi = i * np.pi * (3.0 - np.sqrt(5.0))
    r = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    return np.stack([r * np.cos(phi), r * np.sin(phi), z], axis=1)


def smooth_random_field(seed: int, n_waves: int = 8, freq_sigma: float = 2.0):
    """A seeded smooth scalar field on the unit sphere with max |f| = 1 (sampled on 4096 points).

    f(u) = sum_j a_j cos(omega_j . u + phase_j), a_j ~ N(0,1), omega_j ~ N(0, freq_sigma^2 I),
    phase_j ~ U[0, 2pi).
    """
    rng = np.random.default_rng(seed)
    a = rng.standard_normal(n_waves)
    om = rng.standard_normal((n_waves, 3)) * freq_sigma
    ph = rng.uniform(0.0, 2.0 * np.pi, n_waves)

    def raw(u):
        return np.cos(u @ om.T + ph) @ a

    scale = np.abs(raw(fibonacci_directions(4096))).max()
    return lambda u: raw(np.asarray(u, float)) / scale


def deformed_sphere_patches(amplitude: float = 0.15, seed: int = 1, spans: int = 4) -> list[NurbsPatch]:
    """Unit sphere patches refined to `spans` knot spans per direction (degree 4, so spans+4 control
    points), control points displaced radially: P <- P (1 + amplitude f(P/|P|)), f from
    `smooth_random_field(seed)`.  Shared interface control points move identically, so the surface
    stays watertight and conforming."""
    f = smooth_random_field(seed)
    out = []
    for pt in unit_sphere_patches():
        r = refine_patch(pt, spans)
        P = r.ctrl.reshape(-1, 3)
        u = P / np.linalg.norm(P, axis=1, keepdims=True)
        P = P * (1.0 + amplitude * f(u))[:, None]
        out.append(NurbsPatch(r.p1, r.p2, r.knots1, r.knots2, P.reshape(r.ctrl.shape), r.weights.copy()))
    return out


def flat_patch(corners) -> NurbsPatch:
    """Bilinear patch with corners F(0,0), F(1,0), F(0,1), F(1,1) (each a 3-vector)."""
    c00, c10, c01, c11 = (np.asarray(c, float) for c in corners)
    ctrl = np.array([[c00, c01], [c10, c11]])
    return NurbsPatch(1, 1, np.array([0.0, 0, 1, 1]), np.array([0.0, 0, 1, 1]), ctrl, np.ones((2, 2)))


def random_complex(n: int, seed: int = 1234, cols: int | None = None) -> np.ndarray:
    """(N(0,1) + i N(0,1))/sqrt2 entries, shape (n,) or (n, cols), from default_rng(seed)."""
    rng = np.random.default_rng(seed)
    shape = (n,) if cols is None else (n, cols)
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / np.sqrt(2.0)


def patches_to_arrays(patches: list[NurbsPatch]):
    """Flatten patches into the arrays the C ABI takes (degrees, sizes, knots, ctrl, weights)."""
    deg = np.array([[p.p1, p.p2] for p in patches], dtype=np.int32)
    cnt = np.array([[p.k1, p.k2] for p in patches], dtype=np.int32)
    knots = np.concatenate([np.concatenate([p.knots1, p.knots2]) for p in patches]).astype(np.float64)
    ctrl = np.concatenate([p.ctrl.reshape(-1, 3) for p in patches]).astype(np.float64)
    w = np.concatenate([p.weights.reshape(-1) for p in patches]).astype(np.float64)
    return deg, cnt, knots, ctrl, w


def torus_patches(R: float = 2.0, r: float = 0.5) -> list[NurbsPatch]:
    """The torus with major radius R and minor radius r as 16 exact rational biquadratic patches:
    a surface of revolution whose profile (the minor circle) and sweep (the major circle) are each
    four rational quadratic quarter-circle arcs (control points on the arc ends and at the corner of
    their tangents, middle weight 1/sqrt(2)); patch (i, j) covers the quarter i of the major circle
    and the quarter j of the minor circle, so neighbouring patches share edge parametrisations.  The
    parameter s runs along the major circle and t along the minor one, which makes d_s F x d_t F
    point out of the enclosed volume."""
    h = 1.0 / np.sqrt(2.0)
    w3 = np.array([1.0, h, 1.0])

    def arc(k):   # unit-circle quarter arc k (angles k pi/2 .. (k+1) pi/2): 2-D control points
        a0, a1 = k * np.pi / 2, (k + 1) * np.pi / 2
        p0 = np.array([np.cos(a0), np.sin(a0)])
        p2 = np.array([np.cos(a1), np.sin(a1)])
        return np.stack([p0, p0 + p2, p2])   # the corner of the two tangents is p0 + p2 for a quarter arc

    knots = np.array([0.0, 0.0, 0.0, 1.0, 1.0, 1.0])
    patches = []
    for i in range(4):          # major circle (sweep), parameter t
        C = arc(i)
        for j in range(4):      # minor circle (profile), parameter s
            Dm = arc(j)
            ctrl = np.zeros((3, 3, 3))
            wts = np.zeros((3, 3))
            for a in range(3):      # s index (profile)
                for b in range(3):  # t index (sweep)
                    rho = R + r * Dm[a, 0]     # distance of the profile control point from the axis
                    ctrl[a, b] = [rho * C[b, 0], rho * C[b, 1], r * Dm[a, 1]]
                    wts[a, b] = w3[a] * w3[b]
            # first parameter along the sweep: d_s F x d_t F then points outward
            patches.append(NurbsPatch(2, 2, knots.copy(), knots.copy(), ctrl.transpose(1, 0, 2).copy(),
                                      wts.T.copy()))
    return patches


def polyhedral_torus_patches(R: float = 2.0, r: float = 0.5, n_major: int = 4, n_minor: int = 4):
    """A closed genus-1 surface of n_major x n_minor flat bilinear patches whose corners lie on the
    torus with radii (R, r); used where a closed surface with Euler characteristic 0 is needed."""
    def pt(i, j):
        a = 2 * np.pi * (i % n_major) / n_major
        b = 2 * np.pi * (j % n_minor) / n_minor
        return np.array([(R + r * np.cos(b)) * np.cos(a), (R + r * np.cos(b)) * np.sin(a), r * np.sin(b)])
    return [flat_patch((pt(i, j), pt(i + 1, j), pt(i, j + 1), pt(i + 1, j + 1)))
            for i in range(n_major) for j in range(n_minor)]
