"""Schwarz alternating procedure (SAP) preconditioner and flexible GCR, FP64 oracle.

TEST INFRASTRUCTURE ONLY, like ``qxd_oracle``: only ``tests/`` may import it; the product
library never does, and the two share no code.

The paper's CPU solves use a heavily preconditioned GCR whose preconditioner is the Schwarz
alternating procedure (openQxD's DFL_SAP_GCR, Sec. 5.1).  The paper only names the method.
This module writes out the textbook procedure, a multiplicative Schwarz method on
non-overlapping blocks.  The readings below fill what the paper leaves open:

  * Blocks: extents b_mu that divide L_mu.  The block grid n_mu = L_mu / b_mu is 1 or even in
    every direction, so blocks of one colour never touch, periodic wrap included.  With C*, a
    hop across the y or z boundary also moves x by L1 (Sec. 4.2), so L1 must be an even number
    of x blocks as well.  The colour of a block is the parity of the sum of its block
    coordinates.
  * Block operator D_Lambda: the matrix of D restricted to the sites of the block, rows and
    columns both.  Hops that leave the block are dropped (Dirichlet boundary).  A block that
    spans a whole extent keeps its wrap-around links, since both ends lie in the block.
  * One SAP cycle: colour 0, then colour 1.  Every block of the colour gets
    e = (approximate) D_Lambda^{-1} r restricted to the block, then x += e and r -= D e.
  * The block solve is nmr minimal-residual steps from zero, or an exact dense solve (pins).
  * The preconditioner M applies ncy cycles starting from x = 0.

``fgcr`` is flexible GCR with restarts around any preconditioner, judged by its own recurrence
residual; callers judge the result by the true residual.
"""
from __future__ import annotations

import itertools

import numpy as np

from oracle import qxd_oracle as O


def sap_blocks(L, b, cstar_L1=None):
    """The blocks of extents b on a lattice of extents L: a list of (site mask, colour).

    cstar_L1: the physical L1 of a C* lattice (L is then the doubled lattice).  A hop across the
    y or z boundary moves x by L1, so L1 must be an even number of x blocks for blocks that meet
    there to have opposite colours."""
    L, b = tuple(int(v) for v in L), tuple(int(v) for v in b)
    if cstar_L1 is not None and int(cstar_L1) % (2 * b[1]):
        raise ValueError("with C*, the physical L1 must be an even number of x blocks")
    n = []
    for Lm, bm in zip(L, b):
        if bm <= 0 or Lm % bm:
            raise ValueError(f"block extent {bm} does not divide {Lm}")
        nm = Lm // bm
        if nm != 1 and nm % 2:
            raise ValueError("the block grid must be 1 or even in every direction")
        n.append(nm)
    x = O.coords_of(L)  # (V, 4) site coordinates, lexicographic order
    bc = x // np.array(b)
    out = []
    for k in itertools.product(*(range(nm) for nm in n)):
        mask = np.all(bc == np.array(k), axis=1)
        out.append((mask, int(sum(k)) % 2))
    return out


def block_apply(op, mask, v):
    """D_Lambda v: D on v restricted to the block, the result restricted to the block."""
    return op.block(v, mask, mask)


def mr_block(op, mask, r, nmr):
    """nmr minimal-residual steps for D_Lambda e = r_Lambda from e = 0."""
    e = np.zeros_like(r)
    rr = np.where(mask[:, None, None], r, 0)
    for _ in range(nmr):
        ar = block_apply(op, mask, rr)
        den = O.vdot(ar, ar)
        if den == 0:
            break
        alpha = O.vdot(ar, rr) / den  # minimises ||rr - alpha D_Lambda rr||
        e = e + alpha * rr
        rr = rr - alpha * ar
    return e


def exact_block(op, mask, r):
    """e = D_Lambda^{-1} r_Lambda by a dense solve on the block (small blocks only)."""
    sites = np.flatnonzero(mask)
    n = 12 * sites.size
    cols = np.empty((n, n), dtype=np.complex128)
    unit = np.zeros(r.shape, dtype=np.complex128)
    for j in range(n):
        s, c = divmod(j, 12)
        unit[sites[s]].flat[c] = 1.0
        cols[:, j] = block_apply(op, mask, unit)[sites].reshape(-1)
        unit[sites[s]].flat[c] = 0.0
    e = np.zeros_like(r)
    e[sites] = np.linalg.solve(cols, r[sites].reshape(-1)).reshape(-1, 4, 3)
    return e


def sap(op, blocks, eta, ncy, nmr=None):
    """M eta: ncy SAP cycles from x = 0 (block solves: nmr MR steps, or exact when nmr is None)."""
    x = np.zeros_like(eta)
    r = eta.copy()
    for _ in range(ncy):
        for colour in (0, 1):
            for mask, c in blocks:
                if c != colour:
                    continue
                e = exact_block(op, mask, r) if nmr is None else mr_block(op, mask, r, nmr)
                x = x + e
                r = r - op.D(e)
    return x


def fgcr(apply_D, eta, precond, tol, maxiter, restart=16, x0=None):
    """Flexible GCR(restart) for D x = eta with a right preconditioner that may change each step.

    Each step: z = M r, w = D z, orthogonalised against the cycle's earlier w (modified
    Gram-Schmidt, the same combination applied to z); x += alpha z, r -= alpha w with
    alpha = <w, r> / <w, w>.  Stops when ||r|| <= tol ||eta||.  Returns (x, steps, ||r|| / ||eta||).
    """
    x = np.zeros_like(eta) if x0 is None else x0.copy()
    r = eta - apply_D(x) if x0 is not None else eta.copy()
    bn = O.norm(eta)
    if bn == 0:
        return np.zeros_like(eta), 0, 0.0
    steps = 0
    rel = O.norm(r) / bn
    while rel > tol and steps < maxiter:
        ws, zs = [], []
        for _ in range(restart):
            z = precond(r)
            w = apply_D(z)
            for wj, zj in zip(ws, zs):
                beta = O.vdot(wj, w) / O.vdot(wj, wj)
                w = w - beta * wj
                z = z - beta * zj
            alpha = O.vdot(w, r) / O.vdot(w, w)
            x = x + alpha * z
            r = r - alpha * w
            ws.append(w)
            zs.append(z)
            steps += 1
            rel = O.norm(r) / bn
            if rel <= tol or steps >= maxiter:
                break
    return x, steps, rel
