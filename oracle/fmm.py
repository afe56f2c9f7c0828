"""Cluster tree, admissibility and the interpolated-kernel Galerkin matrix (oracle; test
infrastructure).

Sec. 4.4 compresses the Galerkin matrix with a black-box (interpolation) fast multipole method on the
reference domain: clusters are squares of the patch parameter domains, admissible cluster pairs get a
degenerate (tensor interpolation) approximation of the pull-back kernel, the rest is split
hierarchically.  The paper names the admissibility parameter (eta = 1.6) and the number of
interpolation points per direction (9) but defines neither; the readings used here:

  * clusters: the square (j, l, cx, cy) = [cx, cx+1] x [cy, cy+1] / 2^l of patch j, levels 0..L, the
    leaf level L = m - b (b >= 0, element leaves for b = 0);
  * bounding ball: centre F_j(midpoint), radius the largest distance from it to F_j on the uniform
    9 x 9 grid of the square (corners and edges included);
  * admissible (tau, sigma) iff max(2 r_tau, 2 r_sigma) <= eta_adm (|c_tau - c_sigma| - r_tau -
    r_sigma), and, when a cap is set, kappa max(2 r_tau, 2 r_sigma) <= cap;
  * block partition: start from all pairs of patch roots at level 0; per level an admissible pair is
    kept as a far block, an inadmissible pair at the leaf level is a near block, any other pair is
    replaced by its 4 x 4 child pairs;
  * interpolation: Chebyshev points of the first kind, q per direction, s_a = mid + half cos((2a+1)
    pi/(2q)); tensor Lagrange basis L_a;
  * interpolated kernel on a far block: k~(x^, y^) = sum_{a,b} L_a(x^) k(x^_a, y^_b) L_b(y^), where k
    is the pull-back kernel of V, K or K' (it contains the surface measures) and, for W, the kernel G
    alone (the curl and normal factors of Maue's formula stay at the quadrature points).

"Mode B" is the Galerkin matrix with k~ in place of k on the element pairs of far blocks and the exact
rules on all other pairs, every element pair integrated with the same rules as the exact matrix; the
fast multipole matrix-vector product reproduces it up to rounding.

Level-adaptive interpolation (not in the paper, whose wavenumbers stay below 2.5 on objects of size <= 5
and which uses one q everywhere).  For kappa diam >> 1 a fixed q either loses accuracy on coarse levels
or, with a kappa cap, pushes every block down to fine levels.  Reading used here: with the
textbook bound for Chebyshev interpolation of exp(i omega t) on [-1, 1] with q points,
    eps(q, omega) = omega^q / (2^(q-1) q!),
the finest-level pair (q0 = cheb_q, cap0 = kappa_cap) fixes the accuracy eps_ref = eps(q0, cap0 / 2)
(omega = kappa diam / 2: the phase of the kernel changes by at most kappa diam across a cluster); on
level l with largest cluster diameter D_l = max 2 r the level takes the smallest q in [q0, q_max] with
eps(q, kappa D_l / 2) <= eps_ref (q_max if none does), and its cap is the kappa diam at which that q
reaches eps_ref: cap_l = 2 (eps_ref 2^(q-1) q!)^(1/q) (cap0 itself where q = q0).  A far block on level
l uses q_l points per direction; mode B is defined with these per-level q.
"""
from __future__ import annotations

import math

import numpy as np

from .bspline import nurbs_eval
from .assemble import (ElementRules, PointData, kernel_arrays, mass_blocks, regular_row_blocks,
                       singular_blocks)


def cheb_nodes(q: int, lo: float, hi: float) -> np.ndarray:
    a = np.arange(q)
    return 0.5 * (lo + hi) + 0.5 * (hi - lo) * np.cos((2 * a + 1) * np.pi / (2 * q))


def lagrange(nodes: np.ndarray, s: np.ndarray) -> np.ndarray:
    """L_a(s) for all nodes a: array (len(s), q)."""
    s = np.asarray(s, float)
    q = nodes.shape[0]
    out = np.ones((s.shape[0], q))
    for a in range(q):
        for b in range(q):
            if b != a:
                out[:, a] *= (s - nodes[b]) / (nodes[a] - nodes[b])
    return out


def cheb_error_bound(q: int, omega: float) -> float:
    """Bound on the max error of q-point Chebyshev interpolation of exp(i omega t) on [-1, 1]:
    max|f^(q)| / (2^(q-1) q!) with |f^(q)| = omega^q."""
    return omega ** q / (2.0 ** (q - 1) * math.factorial(q))


def level_q_and_caps(kappa, diam, q0, cap0, q_max):
    """Per-level interpolation points and kappa caps (see the module header): diam[l] is the largest
    cluster diameter bound 2 r on level l."""
    if q_max is None or q_max <= q0 or not np.isfinite(cap0):
        return [q0] * len(diam), [cap0] * len(diam)
    eps_ref = cheb_error_bound(q0, cap0 / 2)
    qs, caps = [], []
    for D in diam:
        q = next((qq for qq in range(q0, q_max + 1) if cheb_error_bound(qq, kappa * D / 2) <= eps_ref), q_max)
        qs.append(q)
        caps.append(cap0 if q == q0 else 2.0 * (eps_ref * 2.0 ** (q - 1) * math.factorial(q)) ** (1.0 / q))
    return qs, caps


class ClusterTree:
    def __init__(self, mesh, leaf_level: int, eta_adm: float, q: int, kappa: float = 0.0,
                 kappa_cap: float = np.inf, q_max: int | None = None):
        if not 0 <= leaf_level <= mesh.m:
            raise ValueError("leaf level must lie in 0..m")
        self.mesh, self.L, self.eta, self.q = mesh, leaf_level, eta_adm, q
        self.kappa, self.cap = kappa, kappa_cap
        n = mesh.n_patches
        self.center, self.radius = [], []
        g = np.linspace(0.0, 1.0, 9)
        gs, gt = np.meshgrid(g, g, indexing="ij")
        for l in range(leaf_level + 1):
            nl = 2 ** l
            c = np.zeros((n * nl * nl, 3)); r = np.zeros(n * nl * nl)
            for j in range(n):
                cx, cy = np.meshgrid(np.arange(nl), np.arange(nl), indexing="ij")
                cx, cy = cx.ravel(), cy.ravel()
                mid, _, _ = nurbs_eval(mesh.patches[j], (cx + 0.5) / nl, (cy + 0.5) / nl)
                S = ((cx[:, None] + gs.ravel()[None, :]) / nl).ravel()
                T = ((cy[:, None] + gt.ravel()[None, :]) / nl).ravel()
                P, _, _ = nurbs_eval(mesh.patches[j], S, T)
                P = P.reshape(nl * nl, -1, 3)
                sl = slice(j * nl * nl, (j + 1) * nl * nl)
                c[sl] = mid
                r[sl] = np.linalg.norm(P - mid[:, None, :], axis=2).max(axis=1)
            self.center.append(c); self.radius.append(r)
        self.ql, self.caps = level_q_and_caps(kappa, [2 * r.max() for r in self.radius], q, kappa_cap, q_max)
        self.far = [[] for _ in range(leaf_level + 1)]
        self.near = []
        cand = [(t, s) for t in range(n) for s in range(n)]
        for l in range(leaf_level + 1):
            nxt = []
            for t, s in cand:
                if self.admissible(l, t, s):
                    self.far[l].append((t, s))
                elif l == leaf_level:
                    self.near.append((t, s))
                else:
                    ct, cs = self.children(l, t), self.children(l, s)
                    nxt.extend((a, b) for a in ct for b in cs)
            cand = nxt

    def admissible(self, l, t, s) -> bool:
        ct, cs = self.center[l][t], self.center[l][s]
        rt, rs = self.radius[l][t], self.radius[l][s]
        diam = max(2 * rt, 2 * rs)
        dist = np.linalg.norm(ct - cs) - rt - rs
        if dist <= 0 or diam > self.eta * dist:
            return False
        return self.kappa * diam <= self.caps[l]

    @staticmethod
    def decode(l, t):
        nl = 2 ** l
        return t // (nl * nl), (t // nl) % nl, t % nl

    def children(self, l, t):
        j, cx, cy = self.decode(l, t)
        nl = 2 ** (l + 1)
        return [j * nl * nl + (2 * cx + a) * nl + (2 * cy + b) for a in (0, 1) for b in (0, 1)]

    def cluster_of(self, l, e):
        mesh = self.mesh
        sh = mesh.m - l
        nl = 2 ** l
        return mesh.patch_of[e] * nl * nl + (mesh.ix[e] >> sh) * nl + (mesh.iy[e] >> sh)

    def elements(self, l, t):
        mesh = self.mesh
        j, cx, cy = self.decode(l, t)
        k = 2 ** (mesh.m - l)
        ix, iy = np.meshgrid(np.arange(cx * k, (cx + 1) * k), np.arange(cy * k, (cy + 1) * k),
                             indexing="ij")
        return j * mesh.n1 * mesh.n1 + ix.ravel() * mesh.n1 + iy.ravel()

    def nodes(self, l, t):
        """Chebyshev nodes of cluster t at level l (q = q_l per direction): patch index and parameters
        (s, t) (q*q,), node index a = a1 q + a2."""
        j, cx, cy = self.decode(l, t)
        nl = 2 ** l
        q = self.ql[l]
        n1 = cheb_nodes(q, cx / nl, (cx + 1) / nl)
        n2 = cheb_nodes(q, cy / nl, (cy + 1) / nl)
        return j, np.repeat(n1, q), np.tile(n2, q), n1, n2

    def cover_check(self):
        """Every ordered element pair lies in exactly one far block or one near block."""
        mesh = self.mesh
        cnt = np.zeros((mesh.E, mesh.E), dtype=np.int32)
        for l, pairs in enumerate(self.far):
            for t, s in pairs:
                cnt[np.ix_(self.elements(l, t), self.elements(l, s))] += 1
        for t, s in self.near:
            cnt[np.ix_(self.elements(self.L, t), self.elements(self.L, s))] += 1
        return cnt


class InterpolatedKernel:
    """Kernel samples at node pairs and Lagrange evaluations for far blocks (cached)."""

    def __init__(self, tree: ClusterTree, kappa: float, rules: ElementRules):
        self.tree, self.kappa, self.rules = tree, kappa, rules
        self._nodes = {}
        self._S = {}

    def node_data(self, l, t):
        key = (l, t)
        if key not in self._nodes:
            j, s, tt, n1, n2 = self.tree.nodes(l, t)
            x, fs, ft = nurbs_eval(self.tree.mesh.patches[j], s, tt)
            n = np.cross(fs, ft)
            self._nodes[key] = (x, n, np.linalg.norm(n, axis=1), n1, n2)
        return self._nodes[key]

    def samples(self, op, l, t, s):
        key = (op, l, t, s)
        if key not in self._S:
            xt, nt, at, _, _ = self.node_data(l, t)
            xs, ns, as_, _, _ = self.node_data(l, s)
            kop = "G" if op == "W" else op
            self._S[key] = kernel_arrays(kop, self.kappa, xt[:, None, :], nt[:, None, :],
                                         at[:, None], xs[None, :, :], ns[None, :, :], as_[None, :])
        return self._S[key]

    def lagrange_at_gauss(self, l, t, elems):
        """(len(elems), nq, q*q) tensor Lagrange values of cluster t at the Gauss points."""
        _, _, _, n1, n2 = self.node_data(l, t)
        pts = self.rules.pts
        q = self.tree.ql[l]
        idx = (np.asarray(elems)[:, None] * self.rules.nq + np.arange(self.rules.nq)[None, :]).ravel()
        s, tt = self.tree.mesh.params(pts.e[idx], *self._local_uv(idx))
        L1 = lagrange(n1, s)
        L2 = lagrange(n2, tt)
        return (L1[:, :, None] * L2[:, None, :]).reshape(len(elems), self.rules.nq, q * q)

    def _local_uv(self, idx):
        from .quadrature import tensor_rule
        u, v, _ = tensor_rule(int(round(np.sqrt(self.rules.nq))))
        return u[idx % self.rules.nq], v[idx % self.rules.nq]

    def far_blocks(self, op, e):
        """[(f_indices, blocks)] of all far blocks that contain test element e."""
        tree = self.tree
        out = []
        for l in range(tree.L + 1):
            t = tree.cluster_of(l, e)
            for tt, s in tree.far[l]:
                if tt != t:
                    continue
                fs = tree.elements(l, s)
                Lx = self.lagrange_at_gauss(l, t, [e])[0]          # (nq, Q)
                Ly = self.lagrange_at_gauss(l, s, fs)              # (F, nq, Q)
                S = self.samples(op, l, t, s)
                kt = np.einsum("qa,ab,frb->qfr", Lx, S, Ly)
                out.append((fs, regular_row_blocks(op, self.kappa, self.rules, e, fs, ktilde=kt)))
        return out


def modeB_operators(space, kappa, ops, tree: ClusterTree, rules: ElementRules | None = None):
    """Dense X-space mode-B matrices {op: (NX, NX)}."""
    from .assemble import dense_operators
    rules = rules or ElementRules(space)
    ik = InterpolatedKernel(tree, kappa, rules)
    return dense_operators(space, kappa, ops, rules, far=lambda e, op: ik.far_blocks(op, e))


def cfie_rows(space, kappa, eta, hard: bool, x, rows, tree: ClusterTree | None = None,
              rules: ElementRules | None = None):
    """Selected entries (A x)[rows] of the global CFIE operator (mode B if a tree is given, else the
    exact matrix), computed element row by element row without forming A.  x is (N,) or (N, R); the
    result is (len(rows),) or (len(rows), R)."""
    mesh = space.mesh
    rules = rules or ElementRules(space)
    ops = ["K", "W"] if hard else ["Kp", "V"]
    coef = {"K": -1.0, "W": -1j * eta} if hard else {"Kp": 1.0, "V": -1j * eta}
    x = np.asarray(x, complex)
    single = x.ndim == 1
    xX = (x[:, None] if single else x)[space.x2g]                # (NX, R)
    rows = np.asarray(rows)
    want = np.nonzero(np.isin(space.x2g, rows))[0]             # X indices of the wanted rows
    elems = sorted({e for X in want for e in np.nonzero((space.l2x == X).any(axis=1))[0]})
    touch = {}
    for e, f, k in mesh.touching():
        touch.setdefault(e, []).append((f, k))
    ik = InterpolatedKernel(tree, kappa, rules) if tree is not None else None
    Mb = mass_blocks(rules)
    yX = {}
    for e in elems:
        acc = 0.5 * Mb[e] @ xX[space.l2x[e]]
        done = np.zeros(mesh.E, dtype=bool)
        for op in ops:
            if ik is not None:
                for fs, blocks in ik.far_blocks(op, e):
                    acc = acc + coef[op] * np.einsum("fkl,flr->kr", blocks, xX[space.l2x[fs]])
                    done[fs] = True
        pairs = [(e, e, 0)] + [(e, f, k) for f, k in touch.get(e, []) if not done[f]]
        sb = singular_blocks(ops, kappa, space, pairs)
        for i, (_, f, _) in enumerate(pairs):
            for op in ops:
                acc = acc + coef[op] * sb[op][i] @ xX[space.l2x[f]]
            done[f] = True
        reg = np.nonzero(~done)[0]
        for op in ops:
            blocks = regular_row_blocks(op, kappa, rules, e, reg)
            acc = acc + coef[op] * np.einsum("fkl,flr->kr", blocks, xX[space.l2x[reg]])
        for k, X in enumerate(space.l2x[e]):
            yX[X] = yX.get(X, 0.0) + acc[k]
    out = np.zeros((len(rows), xX.shape[1]), dtype=complex)
    for i, r in enumerate(rows):
        out[i] = sum(yX[X] for X in np.nonzero(space.x2g == r)[0])
    return out[:, 0] if single else out
