"""Three-level multigrid on top of the inexact-deflation subspace, FP64 oracle.

TEST INFRASTRUCTURE ONLY, like ``qxd_oracle``: only ``tests/`` may import it.

The paper's GPU solves use multigrid GCR and its CPU solves openQxD's deflated SAP-GCR (Sec. 5.1);
the paper names the methods and gives no detail.  This module writes out a textbook aggregation
multigrid with three levels whose first coarse level is the deflation subspace of
``dfl_oracle``.  Readings, where the paper is silent:

  * Level 0: the fine operator D, smoothed by the Schwarz alternating procedure (``sap_oracle``).
  * Level 1: the little Dirac operator A1 = P1^+ D P1 of a block-local deflation subspace
    (``dfl_oracle.Deflation``).  A level-1 vector has one entry per (block b, basis vector k),
    index b ns1 + k, blocks numbered lexicographically by block coordinates (direction 3 fastest).
  * Level 2: aggregates of a_0 x a_1 x a_2 x a_3 level-1 blocks (numbered the same way by
    aggregate coordinates).  ns2 level-1 vectors, restricted to every aggregate and
    orthonormalised there in vector order (modified Gram-Schmidt), give the basis of P2;
    A2 = P2^+ A1 P2.
  * Level-1 smoother S1(f): nu minimal-residual steps on A1 from zero.
  * Coarsest solve G2(f): n2 steps of GCR on A2 from zero (restart every m steps).
  * Two-grid cycle at level 1: T1(f): y = S1(f); y += P2 G2(P2^+ (f - A1 y)); y += S1(f - A1 y).
  * Level-1 solve K1(f): n1 steps of flexible GCR on A1 from zero with T1 as the preconditioner
    (a K-cycle).
  * Fine preconditioner: z = M_pre(r) (SAP, ncy_pre cycles; none for ncy_pre = 0);
    z += P1 K1(P1^+ (r - D z)); z += M_SAP(r - D z).  It runs inside flexible GCR.
  * GCR steps (coarse levels): z = M r (M = 1 without a preconditioner), w = A z; classical
    Gram-Schmidt of w against the cycle's earlier normalised w_j (the same combination applied
    to z); w and z divided by ||w||; alpha = <w, r>; x += alpha z, r -= alpha w.  A step whose w
    vanishes leaves x and r unchanged.
  * Subspace of level 2: ns2 start vectors (drawn by the caller), each improved by n_it
    normalised approximate inverse iterations v <- G1(v) / ||G1(v)||, with G1 = k steps of
    unpreconditioned GCR on A1 from zero.
"""
from __future__ import annotations

import itertools

import numpy as np

from oracle import sap_oracle as S


def _vdot(a, b):
    return complex(np.vdot(a, b))


def gcr(apply_A, f, nsteps, m=16, precond=None):
    """nsteps steps of (flexible) GCR on A x = f from x = 0; returns x."""
    x = np.zeros_like(f)
    r = f.copy()
    W, Z = [], []
    for it in range(nsteps):
        if it % m == 0:
            W, Z = [], []
        z = precond(r) if precond is not None else r.copy()
        w = apply_A(z)
        betas = [_vdot(wj, w) for wj in W]  # classical Gram-Schmidt: all from the same w
        for b, wj, zj in zip(betas, W, Z):
            w = w - b * wj
            z = z - b * zj
        nn = float(np.real(_vdot(w, w)))
        s = 1.0 / np.sqrt(nn) if nn > 0 else 0.0
        w, z = s * w, s * z
        a = _vdot(w, r)
        x = x + a * z
        r = r - a * w
        W.append(w)
        Z.append(z)
    return x


def mr(apply_A, f, nu):
    """nu minimal-residual steps on A y = f from y = 0: alpha = <A rho, rho> / <A rho, A rho>."""
    y = np.zeros_like(f)
    rho = f.copy()
    for _ in range(nu):
        q = apply_A(rho)
        qq = float(np.real(_vdot(q, q)))
        if qq == 0:
            break
        a = _vdot(q, rho) / qq
        y = y + a * rho
        rho = rho - a * q
    return y


def block_grid(L, b):
    return tuple(int(Lm) // int(bm) for Lm, bm in zip(L, b))


class Aggregation:
    """The level-2 space: aggregates of level-1 blocks, their orthonormal bases and A2."""

    def __init__(self, A1, grid1, ns1, agg, vectors):
        self.A1 = np.asarray(A1)
        self.grid1 = tuple(int(v) for v in grid1)
        self.agg = tuple(int(v) for v in agg)
        self.ns1 = int(ns1)
        self.ns2 = len(vectors)
        for n, a in zip(self.grid1, self.agg):
            if a < 1 or n % a:
                raise ValueError("aggregate extents must divide the level-1 block grid")
        self.grid2 = tuple(n // a for n, a in zip(self.grid1, self.agg))
        blocks = list(itertools.product(*(range(n) for n in self.grid1)))  # lexicographic, dir 3 fastest
        aggs = list(itertools.product(*(range(n) for n in self.grid2)))
        gidx = {g: i for i, g in enumerate(aggs)}
        self.of_block = np.array([gidx[tuple(k // a for k, a in zip(kb, self.agg))] for kb in blocks])
        self.nb2 = len(aggs)
        # level-1 entries of every aggregate, in level-1 order
        self.entries = []
        for g in range(self.nb2):
            bs = np.flatnonzero(self.of_block == g)
            self.entries.append((bs[:, None] * self.ns1 + np.arange(self.ns1)[None, :]).reshape(-1))
        self.basis = []
        for e in self.entries:
            q = []
            for v in vectors:
                w = np.asarray(v, dtype=np.complex128)[e].copy()
                n0 = np.linalg.norm(w)
                for u in q:
                    w = w - _vdot(u, w) * u
                nrm = np.linalg.norm(w)
                if not nrm > 1e-12 * n0:
                    raise ValueError("level-2 vectors are linearly dependent on an aggregate")
                q.append(w / nrm)
            self.basis.append(np.array(q))
        self.n1 = self.A1.shape[0]
        self.n2 = self.nb2 * self.ns2
        P = np.zeros((self.n1, self.n2), dtype=np.complex128)
        for g, e in enumerate(self.entries):
            P[e, g * self.ns2:(g + 1) * self.ns2] = self.basis[g].T
        self.P = P
        self.A2 = np.conj(P.T) @ self.A1 @ P

    def prolong(self, c):
        return self.P @ c

    def restrict(self, v):
        return np.conj(self.P.T) @ v

    def apply_A1(self, v):
        return self.A1 @ v

    def apply_A2(self, c):
        return self.A2 @ c


class Multigrid:
    """The three-level preconditioner: SAP on level 0, the deflation space as level 1 (dfl),
    the aggregation as level 2 (agg)."""

    def __init__(self, dfl, agg, sap_blocks, nu=2, n1=4, n2=8, m=16, ncy_pre=0, ncy=1, nmr=4):
        self.dfl, self.agg, self.sap_blocks = dfl, agg, sap_blocks
        self.nu, self.n1, self.n2, self.m = nu, n1, n2, m
        self.ncy_pre, self.ncy, self.nmr = ncy_pre, ncy, nmr

    def coarsest(self, f2):
        """G2: n2 GCR steps on A2."""
        return gcr(self.agg.apply_A2, f2, self.n2, self.m)

    def two_grid(self, f):
        """T1(f) at level 1."""
        A1 = self.agg.apply_A1
        y = mr(A1, f, self.nu)
        y = y + self.agg.prolong(self.coarsest(self.agg.restrict(f - A1(y))))
        return y + mr(A1, f - A1(y), self.nu)

    def level1(self, f):
        """K1(f): n1 flexible GCR steps on A1 preconditioned by T1."""
        return gcr(self.agg.apply_A1, f, self.n1, self.m, precond=self.two_grid)

    def precond(self, r):
        """The fine preconditioner z = M_MG r."""
        op = self.dfl.op
        z = np.zeros_like(r)
        if self.ncy_pre > 0:
            z = S.sap(op, self.sap_blocks, r, ncy=self.ncy_pre, nmr=self.nmr)
        z = z + self.dfl.prolong(self.level1(self.dfl.restrict(r - op.D(z))))
        return z + S.sap(op, self.sap_blocks, r - op.D(z), ncy=self.ncy, nmr=self.nmr)


def generate_level2(A1, start, n_it, k=8, m=16):
    """Level-2 vectors: the start vectors (level-1 vectors drawn by the caller) after n_it
    normalised inverse iterations v <- G1(v) / ||G1(v)||, G1 = k GCR steps on A1."""
    out = []
    for v in start:
        v = np.asarray(v, dtype=np.complex128)
        v = v / np.linalg.norm(v)
        for _ in range(n_it):
            v = gcr(lambda u: A1 @ u, v, k, m)
            v = v / np.linalg.norm(v)
        out.append(v)
    return out


def solve(mg, eta, tol=1e-12, maxiter=500, restart=16):
    """Flexible GCR on D psi = eta with the multigrid preconditioner; (psi, steps, rel)."""
    return S.fgcr(mg.dfl.op.D, eta, mg.precond, tol, maxiter, restart=restart)
