"""Galerkin matrices and right-hand sides of the CFIE systems (oracle; test infrastructure).

Operators (Sec. 2): with G(x,y) = exp(i kappa r) / (4 pi r), r = |x - y|,
  V:  kernel G;   K: dG/dn_y;   K' (K*): dG/dn_x;
  W:  Maue's regularisation (Sec. 4.3): <W u, v> = int int G [curl u(y) . curl v(x)
      - kappa^2 (n_x . n_y) u(y) v(x)], the sign that makes W = -d/dn_x of the double layer.
Pull-back (Sec. 4.2): with n~ = d_s F x d_t F and a = |n~| the entry of operator A between the test
function psi_i (variable x) and the trial function psi_j (variable y) is

    A_ij = sum over element pairs  int int k(x^, y^) psi_i(x^) psi_j(y^) dy^ dx^

with the pull-back kernels a_x a_y G (V), a_y G'(r)/r (x-y).n~_x (K'), a_x G'(r)/r (y-x).n~_y (K),
G'(r) = G (i kappa r - 1)/r, and for W (Sec. 4.3, curl formula with 1/a_j read for the patch of x)
    G [c_i(x^) . c_j(y^) - kappa^2 (n~_x . n~_y) psi_i psi_j],   c = d_s psi d_t F - d_t psi d_s F,
in which the surface measures cancel.  M_ij = int psi_i psi_j a.

Systems (Sec. 4.1):  sound-soft  (1/2 M + K' - i eta V) t = u,  u_i = <du_inc/dn - i eta u_inc, psi_i>;
                     sound-hard  (1/2 M - K - i eta W) g = v,  v_i = <u_inc - i eta du_inc/dn, psi_i>;
on S^2 resp. S^0, u_inc = exp(i kappa d.x).  Quadrature rules: see ``quadrature``.
"""
from __future__ import annotations

import numpy as np

from . import quadrature as Q

NG = 4          # Gauss points per direction on regular pairs, right-hand sides and far field
NS = 5          # Gauss points per transformed variable on touching pairs


class PointData:
    """Geometry and basis data at a batch of points (elements e, local coordinates u, v)."""

    def __init__(self, space, e, u, v):
        mesh = space.mesh
        self.e = np.asarray(e)
        self.x, fs, ft = mesh.geometry(self.e, u, v)
        self.fs, self.ft = fs, ft
        self.n = np.cross(fs, ft)                       # n~ = d_s F x d_t F
        self.a = np.linalg.norm(self.n, axis=1)
        self.phi, dps, dpt = space.eval(self.e, u, v)
        # c_k = d_s psi_k d_t F - d_t psi_k d_s F : (npts, nloc, 3)
        self.curl = dps[:, :, None] * ft[:, None, :] - dpt[:, :, None] * fs[:, None, :]


def kernel_arrays(op: str, kappa: float, x, nx, ax, y, ny, ay):
    """Pull-back kernel of op in {'V', 'K', 'Kp', 'G'} for broadcastable point arrays
    (x, nx: (..., 3); ax: (...)) and (y, ny, ay)."""
    d = x - y
    r = np.linalg.norm(d, axis=-1)
    G = np.exp(1j * kappa * r) / (4.0 * np.pi * r)
    if op == "G":
        return G
    if op == "V":
        return ax * ay * G
    dG_r = G * (1j * kappa * r - 1.0) / (r * r)         # G'(r) / r
    if op == "Kp":
        return ay * dG_r * np.sum(d * nx, axis=-1)
    if op == "K":
        return ax * dG_r * np.sum(-d * ny, axis=-1)
    raise ValueError(op)


def kernel(op: str, kappa: float, X: "PointData", Y: "PointData", ix, iy):
    """Pull-back kernel of op at the point pairs (X[ix], Y[iy])."""
    return kernel_arrays(op, kappa, X.x[ix], X.n[ix], X.a[ix], Y.x[iy], Y.n[iy], Y.a[iy])


def pair_block(op, kappa, X: PointData, Y: PointData, ix, iy, w, ktilde=None):
    """Block B[k, l] = sum_points w k(x, y) psi_k(x) psi_l(y) for one element pair, where the
    points are X[ix], Y[iy] with weights w.  ``ktilde`` replaces the exact kernel values (it is the
    interpolated kernel on admissible blocks; for W it replaces G)."""
    if op == "W":
        kappa2 = kappa * kappa
        Gv = kernel("G", kappa, X, Y, ix, iy) if ktilde is None else ktilde
        cc = np.einsum("pkd,pld->pkl", X.curl[ix], Y.curl[iy])
        nn = np.sum(X.n[ix] * Y.n[iy], axis=-1)
        pp = X.phi[ix][:, :, None] * Y.phi[iy][:, None, :]
        return np.einsum("p,pkl->kl", w * Gv, cc - kappa2 * nn[:, None, None] * pp)
    kv = kernel(op, kappa, X, Y, ix, iy) if ktilde is None else ktilde
    return np.einsum("p,pk,pl->kl", w * kv, X.phi[ix], Y.phi[iy])


class ElementRules:
    """Tensor Gauss data of every element (for regular pairs, mass matrix, RHS, far field)."""

    def __init__(self, space, n=NG):
        mesh = space.mesh
        u, v, w = Q.tensor_rule(n)
        self.nq = u.shape[0]
        E = mesh.E
        e = np.repeat(np.arange(E), self.nq)
        self.pts = PointData(space, e, np.tile(u, E), np.tile(v, E))
        self.w = w * mesh.h * mesh.h                    # d x^ = h^2 du dv
        self.space = space

    def sl(self, e):
        """Point indices of element e."""
        return np.arange(e * self.nq, (e + 1) * self.nq)


def regular_block(op, kappa, rules: ElementRules, e, f):
    return regular_row_blocks(op, kappa, rules, e, np.array([f]))[0]


def regular_row_blocks(op, kappa, rules: ElementRules, e, fs, ktilde=None):
    """Blocks (len(fs), nloc, nloc) of test element e against trial elements fs with the tensor
    Gauss rule on both elements.  ``ktilde`` (nq, len(fs), nq), if given, replaces the exact kernel
    values (for W it replaces G)."""
    P, nq = rules.pts, rules.nq
    fs = np.asarray(fs)
    qe = rules.sl(e)
    qf = (fs[:, None] * nq + np.arange(nq)[None, :])            # (F, nq)
    we = rules.w * 1.0
    wf = np.broadcast_to(rules.w, qf.shape)
    if op == "W":
        Gv = kernel_arrays("G", kappa, P.x[qe][:, None, None, :], None, None,
                           P.x[qf][None, :, :, :], None, None) if ktilde is None else ktilde
        Gw = Gv * wf[None, :, :] * we[:, None, None]            # (q, F, r)
        T1 = np.einsum("qfr,frld->qfld", Gw, P.curl[qf])
        B = np.einsum("qkd,qfld->fkl", P.curl[qe], T1)
        T2 = np.einsum("qfr,frd,frl->qfld", Gw, P.n[qf], P.phi[qf])
        B -= kappa * kappa * np.einsum("qd,qk,qfld->fkl", P.n[qe], P.phi[qe], T2)
        return B
    if ktilde is None:
        kv = kernel_arrays(op, kappa, P.x[qe][:, None, None, :], P.n[qe][:, None, None, :],
                           P.a[qe][:, None, None], P.x[qf][None], P.n[qf][None], P.a[qf][None])
    else:
        kv = ktilde
    kw = kv * wf[None, :, :] * we[:, None, None]
    return np.einsum("qk,qfr,frl->fkl", P.phi[qe], kw, P.phi[qf])


def _canonical_transforms(mesh, e, f, kind):
    """First (T_e, T_f) in the fixed D4 order that puts the shared edge (kind 2) at local u = 0 with
    matching v, or the shared vertex (kind 1) at the local origin, for both elements."""
    tol = 1e-10 * mesh.scale

    def corner(el, T, u, v):
        uu, vv = T(u, v)
        c = int(round(uu)) + 2 * int(round(vv))
        return mesh.corners[el, c]

    for Te in Q.D4:
        for Tf in Q.D4:
            if np.linalg.norm(corner(e, Te, 0, 0) - corner(f, Tf, 0, 0)) > tol:
                continue
            if kind == 2 and np.linalg.norm(corner(e, Te, 0, 1) - corner(f, Tf, 0, 1)) > tol:
                continue
            return Te, Tf
    raise RuntimeError("touching pair without a canonical position")


def singular_block(op, kappa, space, e, f, kind, n=NS):
    """Block of a touching pair: kind 0 identical, 2 common edge, 1 common vertex."""
    return singular_blocks([op], kappa, space, [(e, f, kind)], n)[op][0]


def singular_blocks(ops, kappa, space, pairs, n=NS, chunk=32):
    """Blocks of touching pairs [(e, f, kind)] for every op in ops: {op: (len(pairs), nloc, nloc)}.
    The pairs are only batched for speed; each block is the same sum as ``pair_block`` of one pair."""
    mesh = space.mesh
    rules = {0: Q.rule_identical(n), 2: Q.rule_edge(n), 1: Q.rule_vertex(n)}
    out = {op: np.zeros((len(pairs), space.nloc, space.nloc), dtype=complex) for op in ops}
    for c0 in range(0, len(pairs), chunk):
        batch = pairs[c0:c0 + chunk]
        E_, UE, VE, F_, UF, VF, W_, ID = [], [], [], [], [], [], [], []
        for b, (e, f, kind) in enumerate(batch):
            x1, x2, y1, y2, w = rules[kind]
            Te, Tf = (Q.D4[0], Q.D4[0]) if kind == 0 else _canonical_transforms(mesh, e, f, kind)
            ue, ve = Te(x1, x2)
            uf, vf = Tf(y1, y2)
            E_.append(np.full(w.shape[0], e)); F_.append(np.full(w.shape[0], f))
            UE.append(ue); VE.append(ve); UF.append(uf); VF.append(vf)
            W_.append(w * mesh.h ** 4); ID.append(np.full(w.shape[0], b))
        X = PointData(space, np.concatenate(E_), np.concatenate(UE), np.concatenate(VE))
        Y = PointData(space, np.concatenate(F_), np.concatenate(UF), np.concatenate(VF))
        W = np.concatenate(W_)
        ID = np.concatenate(ID)
        for b in range(len(batch)):
            idx = np.nonzero(ID == b)[0]
            for op in ops:
                out[op][c0 + b] = pair_block(op, kappa, X, Y, idx, idx, W[idx])
    return out


def mass_blocks(rules: ElementRules):
    sp = rules.space
    out = np.zeros((sp.mesh.E, sp.nloc, sp.nloc))
    for e in range(sp.mesh.E):
        s = rules.sl(e)
        out[e] = np.einsum("q,qk,ql->kl", rules.w * rules.pts.a[s], rules.pts.phi[s], rules.pts.phi[s])
    return out


def _scatter(A, space, e, f, B):
    A[np.ix_(space.l2x[e], space.l2x[f])] += B


def dense_operator(space, kappa: float, op: str, rules: ElementRules | None = None, far=None):
    """Dense X-space matrix (NX x NX) of op in {'V','K','Kp','W','M'}; see ``dense_operators``."""
    return dense_operators(space, kappa, [op], rules, far)[op]


def dense_operators(space, kappa: float, ops, rules: ElementRules | None = None, far=None):
    """Dense X-space matrices {op: (NX, NX)} for ops in {'V','K','Kp','W','M'}.

    ``far`` (optional) is a callable far(e, op) -> list of (f_indices, blocks) giving, for test
    element e, trial elements whose blocks replace the exact rules (the interpolated-kernel matrix
    of the fast multipole method); all other pairs use the exact rules.
    """
    mesh = space.mesh
    rules = rules or ElementRules(space)
    out = {op: np.zeros((space.NX, space.NX), dtype=complex) for op in ops}
    if "M" in ops:
        for e, B in enumerate(mass_blocks(rules)):
            _scatter(out["M"], space, e, e, B)
    kops = [op for op in ops if op != "M"]
    if not kops:
        return out
    touch = [(e, e, 0) for e in range(mesh.E)] + mesh.touching()
    far_sets = {}
    if far is not None:
        for e in range(mesh.E):
            far_sets[e] = {op: far(e, op) for op in kops}
    sing_pairs = [t for t in touch
                  if not (far is not None and any(t[1] in fs for fs, _ in far_sets[t[0]][kops[0]]))]
    sblocks = singular_blocks(kops, kappa, space, sing_pairs)
    sing_of = {}
    for i, (e, f, _) in enumerate(sing_pairs):
        sing_of.setdefault(e, []).append((f, i))
    for e in range(mesh.E):
        done = np.zeros(mesh.E, dtype=bool)
        for op in kops:
            if far is not None:
                for fs, blocks in far_sets[e][op]:
                    for f, B in zip(fs, blocks):
                        _scatter(out[op], space, e, f, B)
                    done[fs] = True
            for f, i in sing_of.get(e, []):
                _scatter(out[op], space, e, f, sblocks[op][i])
                done[f] = True
        reg = np.nonzero(~done)[0]
        if reg.size:
            cols = space.l2x[reg].ravel()
            for op in kops:
                blocks = regular_row_blocks(op, kappa, rules, e, reg)
                np.add.at(out[op], (space.l2x[e][:, None], cols[None, :]),
                          blocks.transpose(1, 0, 2).reshape(space.nloc, -1))
    return out


def cfie_matrix(space, kappa, eta, hard: bool, ops=None):
    """Global CFIE matrix: sound-soft 1/2 M + K' - i eta V on S^2; sound-hard P^T (1/2 M - K -
    i eta W) P on S^0.  ``ops`` may supply precomputed X-space matrices by name."""
    names = ["M", "K", "W"] if hard else ["M", "Kp", "V"]
    ops = dict(ops or {})
    missing = [nm for nm in names if nm not in ops]
    if missing:
        ops.update(dense_operators(space, kappa, missing))
    get = ops.__getitem__
    M = get("M")
    if hard:
        AX = 0.5 * M - get("K") - 1j * eta * get("W")
    else:
        AX = 0.5 * M + get("Kp") - 1j * eta * get("V")
    P = space.prolongation()
    return P.T @ AX @ P


def rhs_point_sources(space, kappa, eta, z, hard: bool, rules: ElementRules | None = None):
    """Load vectors (N, R) of the CFIE systems (Sec. 4.1) for the incident fields u_inc = G(., z_r) of
    point sources at the rows of z (R, 3): sound-soft <du_inc/dn - i eta u_inc, psi_i>, sound-hard
    <u_inc - i eta du_inc/dn, psi_i>, with du_inc/dn = G'(r)/r (x - z).n, 4x4 Gauss per element."""
    rules = rules or ElementRules(space)
    Z = np.atleast_2d(np.asarray(z, float))
    pts = rules.pts
    wq = np.tile(rules.w, space.mesh.E)
    out = np.zeros((space.N, Z.shape[0]), dtype=complex)
    for r, zr in enumerate(Z):
        v = pts.x - zr
        dist = np.linalg.norm(v, axis=1)
        G = np.exp(1j * kappa * dist) / (4.0 * np.pi * dist)
        dn = G * (1j * kappa * dist - 1.0) / dist ** 2 * np.sum(v * pts.n, axis=1)   # a du_inc/dn
        f = (G * pts.a - 1j * eta * dn) if hard else (dn - 1j * eta * pts.a * G)
        vals = (wq * f)[:, None] * pts.phi
        bX = np.zeros(space.NX, dtype=complex)
        np.add.at(bX, space.l2x[pts.e], vals)
        np.add.at(out[:, r], space.x2g, bX)
    return out


def rhs(space, kappa, eta, d, hard: bool, rules: ElementRules | None = None):
    """Load vector(s) for incident directions d (3,) or (R, 3): (N,) or (N, R).

    sound-soft: <du_inc/dn - i eta u_inc, psi_i>;  sound-hard: <u_inc - i eta du_inc/dn, psi_i>,
    u_inc = exp(i kappa d.x), du_inc/dn = i kappa (d.n) u_inc, 4x4 Gauss per element."""
    rules = rules or ElementRules(space)
    D = np.atleast_2d(np.asarray(d, float))
    pts = rules.pts
    wq = np.tile(rules.w, space.mesh.E)
    out = np.zeros((space.N, D.shape[0]), dtype=complex)
    for r, dr in enumerate(D):
        uinc = np.exp(1j * kappa * (pts.x @ dr))
        dn = 1j * kappa * (pts.n @ dr) * uinc                 # a du_inc/dn
        f = (uinc * pts.a - 1j * eta * dn) if hard else (dn - 1j * eta * pts.a * uinc)
        vals = (wq * f)[:, None] * pts.phi                     # (npts, nloc)
        bX = np.zeros(space.NX, dtype=complex)
        np.add.at(bX, space.l2x[pts.e], vals)
        np.add.at(out[:, r], space.x2g, bX)
    return out[:, 0] if np.ndim(d) == 1 else out
