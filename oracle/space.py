"""Meshes and spline spaces on NURBS patches (oracle; test infrastructure).

Sec. 3.3: every patch parameter square is refined uniformly to level m, giving 2^m x 2^m elements of
side h = 2^-m; the ansatz functions are tensor B-splines of degree p on the p-open knot vector
Xi_{p,m} = [0,...,0, 1/2^m, ..., (2^m-1)/2^m, 1,...,1] (p+1 repeated end knots), pulled back by the
patch maps.  S^2_{p,m} takes them patchwise (dimension n (2^m+p)^2); S^0_{p,m} glues them to a
globally continuous space.

Indexing.  Element e = (j, ix, iy) has index j 4^m + ix 2^m + iy and local coordinates (u, v) in
[0,1]^2 with patch parameters (s, t) = ((ix+u) h, (iy+v) h).  The patch-wise coefficient space
("X space", equal to S^2) orders the functions of patch j as j n_b^2 + i1 n_b + i2, n_b = 2^m + p.
Local function k = a (p+1) + b of element e is the B-spline (ix+a, iy+b) of its patch.

Gluing for S^0 (Sec. 3.3 requires the patch maps to coincide on interfaces).  A B-spline is anchored
at the image of its Greville point; functions of different patches whose anchors coincide are the
same continuous function, because the conforming parametrisations make their traces equal.
"""
from __future__ import annotations

import numpy as np
from scipy.spatial import cKDTree

from . import bspline


def knot_vector(p: int, m: int) -> np.ndarray:
    """Xi_{p,m} of Sec. 3.3."""
    inner = [j / 2 ** m for j in range(1, 2 ** m)]
    return np.array([0.0] * (p + 1) + inner + [1.0] * (p + 1))


class Mesh:
    """Uniform level-m refinement of every patch parameter square."""

    def __init__(self, patches, m: int):
        self.patches = patches
        self.m = m
        self.n1 = 2 ** m
        self.h = 1.0 / self.n1
        self.n_patches = len(patches)
        self.E = self.n_patches * self.n1 * self.n1
        e = np.arange(self.E)
        self.patch_of = e // (self.n1 * self.n1)
        self.ix = (e // self.n1) % self.n1
        self.iy = e % self.n1
        cu = np.array([0.0, 1.0, 0.0, 1.0])
        cv = np.array([0.0, 0.0, 1.0, 1.0])
        self.corners = np.zeros((self.E, 4, 3))
        for c in range(4):
            x, _, _ = self.geometry(e, np.full(self.E, cu[c]), np.full(self.E, cv[c]))
            self.corners[:, c] = x
        self.scale = np.abs(self.corners).max()

    def params(self, e, u, v):
        return (self.ix[e] + u) * self.h, (self.iy[e] + v) * self.h

    def geometry(self, e, u, v):
        """F, d_s F, d_t F at local points (u, v) of elements e (all arrays of equal length)."""
        e = np.asarray(e)
        s, t = self.params(e, np.asarray(u, float), np.asarray(v, float))
        x = np.zeros((e.shape[0], 3)); fs = np.zeros_like(x); ft = np.zeros_like(x)
        for j in np.unique(self.patch_of[e]):
            sel = self.patch_of[e] == j
            x[sel], fs[sel], ft[sel] = bspline.nurbs_eval(self.patches[j], s[sel], t[sel])
        return x, fs, ft

    def touching(self):
        """Pairs (e, f, kind) of distinct elements with a common corner; kind 2 = common edge,
        kind 1 = common vertex (physical coincidence within 1e-10 of the geometry's size)."""
        pts = self.corners.reshape(-1, 3)
        tree = cKDTree(pts)
        pairs = tree.query_pairs(1e-10 * self.scale, output_type="ndarray")
        shared = {}
        for a, b in pairs:
            e, f = a // 4, b // 4
            if e != f:
                key = (min(e, f), max(e, f))
                shared.setdefault(key, set()).add((a % 4, b % 4) if e < f else (b % 4, a % 4))
        out = []
        for (e, f), s in shared.items():
            n_common = len({c for c, _ in s})
            out.append((e, f, 2 if n_common >= 2 else 1))
            out.append((f, e, 2 if n_common >= 2 else 1))
        return out


class Space:
    """S^2_{p,m} (continuous=False) or S^0_{p,m} (continuous=True) on a mesh."""

    def __init__(self, mesh: Mesh, p: int, continuous: bool = False):
        if continuous and p < 1:
            raise ValueError("the continuous space needs p >= 1")
        self.mesh = mesh
        self.p = p
        self.continuous = continuous
        self.knots = knot_vector(p, mesh.m)
        self.nb = mesh.n1 + p
        self.nloc = (p + 1) ** 2
        self.NX = mesh.n_patches * self.nb * self.nb
        a = np.arange(p + 1)
        l2x = np.zeros((mesh.E, self.nloc), dtype=np.int64)
        for ka in range(p + 1):
            for kb in range(p + 1):
                l2x[:, ka * (p + 1) + kb] = (mesh.patch_of * self.nb * self.nb
                                             + (mesh.ix + ka) * self.nb + (mesh.iy + kb))
        self.l2x = l2x
        if continuous:
            self.x2g, self.N = self._glue()
        else:
            self.x2g, self.N = np.arange(self.NX), self.NX
        del a

    def greville(self) -> np.ndarray:
        p, kn = self.p, self.knots
        return np.array([kn[i + 1:i + p + 1].mean() for i in range(self.nb)])

    def _glue(self):
        g = self.greville()
        anchors = np.zeros((self.NX, 3))
        i1, i2 = np.meshgrid(np.arange(self.nb), np.arange(self.nb), indexing="ij")
        for j, patch in enumerate(self.mesh.patches):
            x, _, _ = bspline.nurbs_eval(patch, g[i1.ravel()], g[i2.ravel()])
            anchors[j * self.nb * self.nb:(j + 1) * self.nb * self.nb] = x
        tree = cKDTree(anchors)
        parent = np.arange(self.NX)

        def find(i):
            while parent[i] != i:
                parent[i] = parent[parent[i]]
                i = parent[i]
            return i

        for a, b in tree.query_pairs(1e-9 * self.mesh.scale, output_type="ndarray"):
            ra, rb = find(a), find(b)
            if ra != rb:
                parent[max(ra, rb)] = min(ra, rb)
        roots = np.array([find(i) for i in range(self.NX)])
        uniq, x2g = np.unique(roots, return_inverse=True)
        return x2g, len(uniq)

    def prolongation(self) -> np.ndarray:
        """The 0/1 matrix P (NX x N) with x_X = P x_global."""
        P = np.zeros((self.NX, self.N))
        P[np.arange(self.NX), self.x2g] = 1.0
        return P

    def eval(self, e, u, v):
        """Local basis values and their d/ds, d/dt derivatives at local points of elements e:
        three arrays (n, (p+1)^2), column k = a (p+1) + b."""
        e = np.asarray(e)
        mesh, p = self.mesh, self.p
        s, t = mesh.params(e, np.asarray(u, float), np.asarray(v, float))
        # element ix lies in knot span mu = ix + p of Xi_{p,m}; its functions are ix .. ix+p
        bs, dbs = bspline.local_basis_and_derivative(self.knots, p, s, mesh.ix[e] + p)
        bt, dbt = bspline.local_basis_and_derivative(self.knots, p, t, mesh.iy[e] + p)
        val = (bs[:, :, None] * bt[:, None, :]).reshape(-1, self.nloc)
        ds = (dbs[:, :, None] * bt[:, None, :]).reshape(-1, self.nloc)
        dt = (bs[:, :, None] * dbt[:, None, :]).reshape(-1, self.nloc)
        return val, ds, dt
