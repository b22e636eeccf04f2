"""Inexact deflation with block-local subspaces, the other half of DFL_SAP_GCR, FP64 oracle.

TEST INFRASTRUCTURE ONLY, like ``qxd_oracle``: only ``tests/`` may import it.

The paper's CPU solves use openQxD's deflated, SAP-preconditioned GCR (Sec. 5.1), and its GPU
runs use multigrid, which builds its coarse space the same way.  The paper gives no detail.
This module writes out the textbook two-level method with a block-local deflation subspace
(inexact deflation).  Readings, where the paper is silent:

  * Subspace generation: Ns random start vectors (drawn by the caller and passed in), each
    improved by n_it steps of approximate inverse iteration v <- M v / ||M v||, with M the SAP
    preconditioner (ncy cycles, nmr MR steps from zero).  Approximate low modes of D result.
  * Block basis: deflation blocks as SAP blocks (colours unused).  On every block, the Ns
    vectors restricted to it are orthonormalised (Gram-Schmidt, in vector order) over all
    12 |Lambda| components.  That gives n_blocks * Ns basis vectors with disjoint block supports.
  * Prolongation P: coarse vector c (n_blocks, Ns) -> sum c_{Lambda,k} psi_{Lambda,k}; P^+ P = 1.
  * Little Dirac operator A = P^+ D P, dense here.  It couples only blocks that share a face,
    since D is nearest-neighbour.
  * Two-level preconditioner: z = P A^{-1} P^+ r (coarse correction), then
    z += M_SAP (r - D z) (smoothing).  It runs inside flexible GCR (``sap_oracle.fgcr``).
"""
from __future__ import annotations

import numpy as np

from oracle import qxd_oracle as O
from oracle import sap_oracle as S


class Deflation:
    """A block-local deflation subspace and its little Dirac operator."""

    def __init__(self, op, blocks, vectors):
        self.op = op
        self.masks = [m for m, _ in blocks]
        self.ns = len(vectors)
        self.shape = vectors[0].shape
        # block-local orthonormal bases: basis[b] has shape (Ns, |Lambda_b| * 12)
        self.sites = [np.flatnonzero(m) for m in self.masks]
        self.basis = []
        for s in self.sites:
            vs = [v[s].reshape(-1) for v in vectors]
            q = []
            for v in vs:
                w = v.astype(np.complex128).copy()
                for u in q:
                    w = w - np.vdot(u, w) * u
                nrm = np.linalg.norm(w)
                if nrm == 0:
                    raise ValueError("deflation vectors are linearly dependent on a block")
                q.append(w / nrm)
            self.basis.append(np.array(q))
        self.n = len(self.masks) * self.ns
        # little Dirac operator A[(b, k), (b', k')] = <psi_{b,k}, D psi_{b',k'}>
        self.A = np.empty((self.n, self.n), dtype=np.complex128)
        for j in range(self.n):
            e = np.zeros(self.n, dtype=np.complex128)
            e[j] = 1.0
            self.A[:, j] = self.restrict(op.D(self.prolong(e)))

    def prolong(self, c):
        """P c: the fine field sum_{b,k} c_{b,k} psi_{b,k}."""
        out = np.zeros(self.shape, dtype=np.complex128)
        c = np.asarray(c).reshape(len(self.masks), self.ns)
        for b, s in enumerate(self.sites):
            out[s] = (c[b] @ self.basis[b]).reshape(-1, 4, 3)
        return out

    def restrict(self, v):
        """P^+ v: the coarse vector <psi_{b,k}, v>."""
        return np.concatenate([np.conj(self.basis[b]) @ v[s].reshape(-1) for b, s in enumerate(self.sites)])

    def coarse_solve(self, r):
        """P A^{-1} P^+ r."""
        return self.prolong(np.linalg.solve(self.A, self.restrict(r)))


def generate_subspace(op, sap_blocks, start, n_it, ncy=1, nmr=4):
    """Approximate low modes: the given start vectors (random fields, drawn by the caller) after
    n_it normalised SAP inverse iterations v <- M v / ||M v||."""
    vs = []
    for v in start:
        v = v / O.norm(v)
        for _ in range(n_it):
            v = S.sap(op, sap_blocks, v, ncy=ncy, nmr=nmr)
            v = v / O.norm(v)
        vs.append(v)
    return vs


def two_level(dfl, sap_blocks, r, ncy=1, nmr=4):
    """z = P A^{-1} P^+ r, then z += M_SAP (r - D z)."""
    z = dfl.coarse_solve(r)
    return z + S.sap(dfl.op, sap_blocks, r - dfl.op.D(z), ncy=ncy, nmr=nmr)
