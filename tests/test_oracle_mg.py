"""Pins of the three-level multigrid oracle (the multigrid GCR of Sec. 5.1), CPU only.

Each pin is a property that holds whatever the subspaces are, checked against something the
multigrid code does not compute itself:
  * the level-2 bases are orthonormal and aggregate-local (P2^+ P2 = 1);
  * A2 equals the Galerkin product (P1 P2)^+ D (P1 P2) with the dense matrix of an independent
    edge-loop D, and couples only aggregates that share a face;
  * k GCR steps minimise the residual over the Krylov space (a least-squares solve over an
    explicit Krylov basis), and an MR step leaves a residual orthogonal to A rho;
  * after an exact coarsest solve the level-1 residual is orthogonal to the level-2 space;
  * with a level-2 space that spans all of level 1 the two-grid cycle is A1^-1;
  * inverse iteration with an exact level-1 solve equals A1^-n v, normalised;
  * multigrid-preconditioned flexible GCR reaches 1e-12 with the eo-CG oracle's solution;
  * planted mistakes (an unconjugated restriction, A2 from A1^T, Gram-Schmidt without its
    projections) fail.
"""
import numpy as np
import pytest

from oracle import dfl_oracle as F
from oracle import mg_oracle as M
from oracle import qxd_oracle as O
from oracle import sap_oracle as S
from paper_2502_02490_gb300 import synth
from tests import dense

PARAMS = dict(q=-1 / 3, m0=0.1, csw=1.9, csw_qed=1.0)


def cvec(n, seed):
    return synth.gaussian_spinor((n, 1, 1, 1), seed).reshape(-1)[:n].astype(np.complex128)


def setup(L, db, ns1, agg, ns2, seed=1300):
    lat = O.Lattice(L, antiperiodic=True)
    U, A = synth.gauge_field(L, seed, 0.3)
    op = O.Operator(lat, U, A, **PARAMS)
    sb = S.sap_blocks(L, (2, 2, 2, 2))
    vs = F.generate_subspace(op, sb, [synth.gaussian_spinor(L, 3000 + k) for k in range(ns1)], n_it=2)
    dfl = F.Deflation(op, S.sap_blocks(L, db), vs)
    grid1 = M.block_grid(L, db)
    v2 = M.generate_level2(dfl.A, [cvec(dfl.n, 4000 + k) for k in range(ns2)], n_it=2)
    ag = M.Aggregation(dfl.A, grid1, ns1, agg, v2)
    return op, sb, dfl, ag, U, A


def dense_D(L, U, A, op):
    H = dense.dense_hop(L, U * np.exp(1j * PARAMS["q"] * A)[..., None, None], True)
    return dense.block_diag_sites(op.C) - 0.5 * H


def test_level2_bases_are_orthonormal_and_aggregate_local():
    op, sb, dfl, ag, U, A = setup((4, 4, 4, 2), (2, 2, 2, 2), 3, (1, 1, 2, 1), 3)
    assert ag.grid2 == (2, 2, 1, 1) and ag.n2 == 12
    assert np.abs(np.conj(ag.P.T) @ ag.P - np.eye(ag.n2)).max() < 1e-13
    for g in range(ag.nb2):
        col = ag.P[:, g * ag.ns2:(g + 1) * ag.ns2]
        outside = np.ones(ag.n1, bool)
        outside[ag.entries[g]] = False
        assert not np.any(col[outside])
        # the aggregate holds the blocks whose block coordinates divided by agg give its own
        assert len(ag.entries[g]) == 2 * ag.ns1


def pin_galerkin(dfl, ag, Dm):
    P1 = np.stack([dfl.prolong(np.eye(dfl.n)[j]).reshape(-1) for j in range(dfl.n)], axis=1)
    P = P1 @ ag.P
    ref = np.conj(P.T) @ Dm @ P
    return np.abs(ag.A2 - ref).max() < 1e-12 * np.abs(ref).max()


def test_A2_is_the_galerkin_product_of_the_dense_D():
    L = (4, 4, 4, 2)
    op, sb, dfl, ag, U, A = setup(L, (2, 2, 2, 2), 3, (1, 1, 2, 1), 3)
    assert pin_galerkin(dfl, ag, dense_D(L, U, A, op))


def test_A2_couples_only_face_neighbours():
    op, sb, dfl, ag, U, A = setup((4, 4, 4, 2), (2, 2, 2, 2), 3, (1, 1, 2, 1), 2)
    import itertools
    kg = list(itertools.product(*(range(n) for n in ag.grid2)))
    ns = ag.ns2
    for g, kg1 in enumerate(kg):
        for h, kg2 in enumerate(kg):
            blk = ag.A2[g * ns:(g + 1) * ns, h * ns:(h + 1) * ns]
            if sum(a != b for a, b in zip(kg1, kg2)) >= 2:
                assert not np.any(np.abs(blk) > 1e-14 * np.abs(ag.A2).max()), (kg1, kg2)
            else:
                assert np.abs(blk).max() > 0


def test_gcr_minimises_the_residual_over_the_krylov_space():
    rng = np.random.default_rng(5)
    n = 40
    Am = np.eye(n) * 3 + (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / np.sqrt(n)
    f = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    for k in (1, 3, 7):
        x = M.gcr(lambda v: Am @ v, f, k, m=16)
        K = np.stack([np.linalg.matrix_power(Am, j) @ f for j in range(k)], axis=1)
        c, *_ = np.linalg.lstsq(Am @ K, f, rcond=None)
        assert np.linalg.norm(x - K @ c) < 1e-10 * np.linalg.norm(x)
    # an MR step leaves rho orthogonal to A rho
    y = M.mr(lambda v: Am @ v, f, 1)
    rho1 = f - Am @ y
    assert abs(np.vdot(Am @ f, rho1)) < 1e-12 * np.linalg.norm(Am @ f) * np.linalg.norm(f)


def test_coarse_correction_is_galerkin_orthogonal_and_full_space_is_exact():
    op, sb, dfl, ag, U, A = setup((4, 4, 4, 2), (2, 2, 2, 2), 3, (1, 1, 2, 1), 3)
    mg = M.Multigrid(dfl, ag, sb, nu=2, n2=ag.n2, m=ag.n2)  # GCR exact in n2 steps
    f = cvec(ag.n1, 11)
    y = M.mr(ag.apply_A1, f, 2)
    y = y + ag.prolong(mg.coarsest(ag.restrict(f - ag.apply_A1(y))))
    assert np.linalg.norm(ag.restrict(f - ag.apply_A1(y))) < 1e-10 * np.linalg.norm(f)
    # a level-2 space spanning level 1 on every aggregate: T1 = A1^-1
    full = [np.eye(ag.n1)[:, j] + 0.1 * cvec(ag.n1, 20 + j) for j in range(2 * ag.ns1)]
    agf = M.Aggregation(dfl.A, ag.grid1, ag.ns1, ag.agg, full)
    mgf = M.Multigrid(dfl, agf, sb, nu=1, n2=agf.n2, m=agf.n2)
    ref = np.linalg.solve(dfl.A, f)
    assert np.linalg.norm(mgf.two_grid(f) - ref) < 1e-9 * np.linalg.norm(ref)


def test_inverse_iteration_with_an_exact_solve_is_a_power_of_the_inverse():
    op, sb, dfl, ag, U, A = setup((4, 4, 4, 2), (2, 2, 2, 2), 3, (1, 1, 2, 1), 2)
    v0 = cvec(dfl.n, 31)
    (v,) = M.generate_level2(dfl.A, [v0], n_it=3, k=dfl.n, m=dfl.n)
    ref = np.linalg.matrix_power(np.linalg.inv(dfl.A), 3) @ v0
    ref /= np.linalg.norm(ref)
    assert np.linalg.norm(v - ref) < 1e-8


def test_multigrid_gcr_reaches_1e12_with_the_eo_cg_solution():
    L = (4, 4, 4, 4)
    op, sb, dfl, ag, U, A = setup(L, (2, 2, 2, 2), 4, (1, 1, 2, 2), 3)
    mg = M.Multigrid(dfl, ag, sb, nu=2, n1=3, n2=6, ncy_pre=1, ncy=1)
    eta = synth.gaussian_spinor(L, 9)
    x, steps, rel = M.solve(mg, eta, tol=1e-12, maxiter=200)
    assert rel <= 1e-12 and O.true_rel_residual(op, x, eta) <= 2e-12
    ref, _ = O.solve_eo_cg(op, eta, tol=1e-13)
    assert O.norm(x - ref) <= 1e-9 * O.norm(ref)


# ---- planted mistakes -------------------------------------------------------------------------
class _RestrictNoConj(M.Aggregation):
    def restrict(self, v):
        return self.P.T @ v


class _A2FromTranspose(M.Aggregation):
    def __init__(self, *a, **k):
        super().__init__(*a, **k)
        self.A2 = np.conj(self.P.T) @ self.A1.T @ self.P


class _NoProjection(M.Aggregation):
    """Gram-Schmidt that only normalises (the projections dropped)."""

    def __init__(self, A1, grid1, ns1, agg, vectors):
        super().__init__(A1, grid1, ns1, agg, vectors)
        for g, e in enumerate(self.entries):
            q = np.array([np.asarray(v)[e] for v in vectors], dtype=complex)
            self.basis[g] = q / np.linalg.norm(q, axis=1, keepdims=True)
            self.P[e, g * self.ns2:(g + 1) * self.ns2] = self.basis[g].T
        self.A2 = np.conj(self.P.T) @ self.A1 @ self.P


@pytest.mark.parametrize("mutant", ["restrict without conjugation", "A2 from A1^T", "Gram-Schmidt without projection"])
def test_mg_pins_catch_planted_mistake(mutant):
    L = (4, 4, 4, 2)
    op, sb, dfl, ag, U, A = setup(L, (2, 2, 2, 2), 3, (1, 1, 2, 1), 3)
    v2 = [cvec(ag.n1, 4000 + k) for k in range(3)]
    cls = {"restrict without conjugation": _RestrictNoConj, "A2 from A1^T": _A2FromTranspose,
           "Gram-Schmidt without projection": _NoProjection}[mutant]
    bad = cls(dfl.A, ag.grid1, ag.ns1, ag.agg, v2)
    caught = not pin_galerkin(dfl, bad, dense_D(L, U, A, op))
    mg = M.Multigrid(dfl, bad, sb, nu=2, n2=bad.n2, m=bad.n2)
    f = cvec(bad.n1, 11)
    y = M.mr(bad.apply_A1, f, 2)
    y = y + bad.prolong(mg.coarsest(bad.restrict(f - bad.apply_A1(y))))
    caught |= not np.linalg.norm(np.conj(bad.P.T) @ (f - bad.apply_A1(y))) < 1e-10 * np.linalg.norm(f)
    caught |= not np.abs(np.conj(bad.P.T) @ bad.P - np.eye(bad.n2)).max() < 1e-13
    assert caught
