"""Pins of the inexact-deflation oracle (the deflation half of DFL_SAP_GCR, Sec. 5.1), CPU only.

Each pin is a property of the construction that holds whatever the subspace is:
  * the block bases are orthonormal and block-local (P^+ P = 1);
  * the little Dirac operator equals the Galerkin product P^+ D P formed with the dense matrix
    of an independent edge-loop D, and couples only blocks that share a face;
  * the coarse solve returns every vector of the subspace exactly;
  * 1 - P A^{-1} P^+ D is a projector that annihilates the subspace;
  * the two-level preconditioned GCR reaches 1e-10 with the eo-CG oracle's solution.
"""
import numpy as np
import pytest

from oracle import dfl_oracle as F
from oracle import qxd_oracle as O
from oracle import sap_oracle as S
from paper_2502_02490_gb300 import synth
from tests import dense

PARAMS = dict(q=-1 / 3, m0=0.1, csw=1.9, csw_qed=1.0)


def setup(L, db, ns, seed=1300, n_it=2):
    lat = O.Lattice(L, antiperiodic=True)
    U, A = synth.gauge_field(L, seed, 0.3)
    op = O.Operator(lat, U, A, **PARAMS)
    sb = S.sap_blocks(L, (2, 2, 2, 2))
    vs = F.generate_subspace(op, sb, [synth.gaussian_spinor(L, 3000 + k) for k in range(ns)], n_it=n_it)
    return op, sb, F.Deflation(op, S.sap_blocks(L, db), vs), U, A


def pin_orthonormal(dfl, L):
    c = synth.gaussian_spinor((dfl.n, 1, 1, 1), 5).reshape(-1)[: dfl.n]
    ok = np.abs(dfl.restrict(dfl.prolong(c)) - c).max() < 1e-13 * np.abs(c).max()
    for b, m in enumerate(dfl.masks):  # basis vectors vanish outside their block
        e = np.zeros(dfl.n, complex)
        e[b * dfl.ns] = 1.0
        ok &= not np.any(dfl.prolong(e)[~m])
    return bool(ok)


def pin_galerkin(dfl, L, U, A):
    V = int(np.prod(L))
    H = dense.dense_hop(L, U * np.exp(1j * PARAMS["q"] * A)[..., None, None], True)
    Dm = dense.block_diag_sites(dfl.op.C) - 0.5 * H
    Pm = np.stack([dfl.prolong(np.eye(dfl.n)[j]).reshape(-1) for j in range(dfl.n)], axis=1)
    ref = np.conj(Pm.T) @ Dm @ Pm
    return np.abs(dfl.A - ref).max() < 1e-12 * np.abs(ref).max() and V * 12 == Pm.shape[0]


def pin_coarse_exact(dfl):
    c = synth.gaussian_spinor((dfl.n, 1, 1, 1), 6).reshape(-1)[: dfl.n]
    v = dfl.prolong(c)
    return np.abs(dfl.coarse_solve(dfl.op.D(v)) - v).max() < 1e-11 * np.abs(v).max()


def test_block_bases_are_orthonormal_and_block_local():
    L = (4, 4, 2, 2)
    op, sb, dfl, U, A = setup(L, (2, 2, 2, 2), 3)
    assert dfl.n == 4 * 3
    assert pin_orthonormal(dfl, L)


def test_little_operator_is_the_galerkin_product_of_the_dense_D():
    L = (4, 4, 2, 2)
    op, sb, dfl, U, A = setup(L, (2, 2, 2, 2), 3)
    assert pin_galerkin(dfl, L, U, A)


def test_little_operator_couples_only_face_neighbours():
    L = (4, 4, 4, 4)
    op, sb, dfl, U, A = setup(L, (2, 2, 2, 2), 2, n_it=1)
    x = O.coords_of(L)
    kb = [tuple(x[m][0] // 2) for m in dfl.masks]  # block coordinates
    ns = dfl.ns
    for b in range(len(kb)):
        for b2 in range(len(kb)):
            far = sum(k1 != k2 for k1, k2 in zip(kb[b], kb[b2])) >= 2
            blk = dfl.A[b * ns:(b + 1) * ns, b2 * ns:(b2 + 1) * ns]
            if far:
                assert not np.any(blk), (kb[b], kb[b2])
            elif b != b2:
                assert np.abs(blk).max() > 0  # a shared face couples them


def test_coarse_solve_returns_subspace_vectors_and_projects():
    L = (4, 4, 2, 2)
    op, sb, dfl, U, A = setup(L, (2, 2, 2, 2), 3)
    assert pin_coarse_exact(dfl)
    # E = 1 - P A^-1 P^+ D is a projector with E P = 0; P_L = 1 - D P A^-1 P^+ has P_L D P = 0
    y = synth.gaussian_spinor(L, 7)
    E = lambda v: v - dfl.coarse_solve(op.D(v))  # noqa: E731
    Ey = E(y)
    assert np.abs(E(Ey) - Ey).max() < 1e-11 * np.abs(Ey).max()
    c = synth.gaussian_spinor((dfl.n, 1, 1, 1), 8).reshape(-1)[: dfl.n]
    Pc = dfl.prolong(c)
    assert np.abs(E(Pc)).max() < 1e-11 * np.abs(Pc).max()
    DPc = op.D(Pc)
    PL = DPc - op.D(dfl.coarse_solve(DPc))
    assert np.abs(PL).max() < 1e-11 * np.abs(DPc).max()


def test_deflated_sap_gcr_reaches_the_tolerance():
    L = (4, 4, 4, 4)
    op, sb, dfl, U, A = setup(L, (2, 2, 2, 2), 4)
    eta = synth.gaussian_spinor(L, 9)
    x, steps, rel = S.fgcr(op.D, eta, lambda r: F.two_level(dfl, sb, r), tol=1e-10, maxiter=200)
    assert rel <= 1e-10 and O.true_rel_residual(op, x, eta) <= 2e-10
    ref, _ = O.solve_eo_cg(op, eta, tol=1e-12)
    assert O.norm(x - ref) <= 1e-8 * O.norm(ref)


# ---- planted mistakes -------------------------------------------------------------------------
def _restrict_no_conj(self, v):
    return np.concatenate([self.basis[b] @ v[s].reshape(-1) for b, s in enumerate(self.sites)])


class _NoProjection(F.Deflation):
    """Gram-Schmidt that only normalises (the projections dropped)."""

    def __init__(self, op, blocks, vectors):
        super().__init__(op, blocks, vectors)
        for b, s in enumerate(self.sites):
            q = np.array([v[s].reshape(-1) for v in vectors], dtype=complex)
            self.basis[b] = q / np.linalg.norm(q, axis=1, keepdims=True)


@pytest.mark.parametrize("mutant", ["restrict without conjugation", "Gram-Schmidt without projection",
                                    "little operator from D^+"])
def test_dfl_pins_catch_planted_mistake(mutant, monkeypatch):
    L = (4, 4, 2, 2)
    op, sb, dfl, U, A = setup(L, (2, 2, 2, 2), 3)
    vs = F.generate_subspace(op, sb, [synth.gaussian_spinor(L, 3000 + k) for k in range(3)], n_it=2)
    if mutant == "restrict without conjugation":
        monkeypatch.setattr(F.Deflation, "restrict", _restrict_no_conj)
        dfl = F.Deflation(op, S.sap_blocks(L, (2, 2, 2, 2)), vs)
    elif mutant == "Gram-Schmidt without projection":
        dfl = _NoProjection(op, S.sap_blocks(L, (2, 2, 2, 2)), vs)
    else:
        dfl.A = np.conj(dfl.A.T)  # <psi, D^+ psi'> = conj(<psi', D psi>)
    assert not (pin_orthonormal(dfl, L) and pin_galerkin(dfl, L, U, A) and pin_coarse_exact(dfl)), mutant
