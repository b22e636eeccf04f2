"""Pins of the SAP / flexible-GCR oracle (the solver named in Sec. 5.1), all on the CPU.

Each pin comes from outside the procedure itself:
  * one block spanning the lattice with exact block solves is D^{-1};
  * with exact block solves one cycle has the error propagator of multiplicative Schwarz,
    (1 - P_1)(1 - P_0) with P_c = sum over blocks of colour c of R^T (R D R^T)^{-1} R D,
    written here with the dense matrix of D;
  * minimal-residual block solves converge to the exact block solve, and each step leaves a
    residual orthogonal to D_Lambda r (the textbook property of the minimal-residual step);
  * the preconditioner is gauge covariant;
  * SAP-preconditioned GCR reaches 1e-12 (the paper's stopping rule) with the solution of
    the even-odd CG oracle, in fewer steps than unpreconditioned GCR.
"""
import numpy as np
import pytest

from oracle import qxd_oracle as O
from oracle import sap_oracle as S
from paper_2502_02490_gb300 import synth
from tests import fields

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")

PARAMS = dict(q=-1 / 3, m0=0.3, csw=1.9, csw_qed=1.0)


def make_op(L, seed=1200, eps=0.3, **kw):
    lat = O.Lattice(L, antiperiodic=True)
    U, A = synth.gauge_field(L, seed, eps)
    return O.Operator(lat, U, A, **dict(PARAMS, **kw)), U, A


def dense_D(op, V):
    n = 12 * V
    M = np.empty((n, n), dtype=np.complex128)
    unit = np.zeros((V, 4, 3), dtype=np.complex128)
    for j in range(n):
        unit.flat[j] = 1.0
        M[:, j] = op.D(unit).reshape(-1)
        unit.flat[j] = 0.0
    return M


def test_blocks_tile_the_lattice_and_same_colours_never_touch():
    L, b = (4, 4, 2, 4), (2, 2, 2, 2)
    lat = O.Lattice(L)
    blocks = S.sap_blocks(L, b)
    assert len(blocks) == 8
    owner = np.full(lat.V, -1)
    for k, (mask, _) in enumerate(blocks):
        assert mask.sum() == 16 and np.all(owner[mask] == -1)
        owner[mask] = k
    assert np.all(owner >= 0)
    colour = np.array([c for _, c in blocks])
    for mu in range(4):
        a, bb = owner, owner[lat.fwd(mu)]
        cross = a != bb
        assert np.all(colour[a[cross]] != colour[bb[cross]]), mu  # neighbours across a face differ
    assert sorted(colour.tolist()) == [0] * 4 + [1] * 4
    with pytest.raises(ValueError):
        S.sap_blocks(L, (3, 2, 2, 2))  # does not divide
    with pytest.raises(ValueError):
        S.sap_blocks((6, 4, 4, 4), (2, 2, 2, 2))  # three blocks in t: same colours would touch


def test_cstar_blocks_keep_same_colours_apart():
    """With C* a hop across the y or z boundary moves x by the physical L1 (Sec. 4.2): blocks of
    one colour stay apart exactly when L1 is an even number of x blocks."""
    def touching_same_colour(L, b):
        lat = O.Lattice(L, cstar=True)
        blocks = S.sap_blocks(lat.dims, b)
        owner, colour = np.empty(lat.V, int), np.array([c for _, c in blocks])
        for k, (mask, _) in enumerate(blocks):
            owner[mask] = k
        return any(np.any((owner != owner[lat.fwd(mu)]) & (colour[owner] == colour[owner[lat.fwd(mu)]]))
                   for mu in range(4))

    assert not touching_same_colour((4, 4, 2, 4), (2, 2, 1, 2))  # L1 = 4: two x blocks
    assert touching_same_colour((4, 2, 2, 4), (2, 2, 1, 2))      # L1 = 2: one x block
    S.sap_blocks((4, 8, 2, 4), (2, 2, 1, 2), cstar_L1=4)
    with pytest.raises(ValueError):
        S.sap_blocks((4, 4, 2, 4), (2, 2, 1, 2), cstar_L1=2)


def test_one_block_with_exact_solves_is_the_inverse():
    L = (2, 2, 2, 2)
    op, _, _ = make_op(L)
    eta = synth.gaussian_spinor(L, 5)
    x = S.sap(op, S.sap_blocks(L, L), eta, ncy=1)
    Dm = dense_D(op, 16)
    ref = np.linalg.solve(Dm, eta.reshape(-1)).reshape(eta.shape)
    assert np.abs(x - ref).max() < 1e-12 * np.abs(ref).max()


def test_cycles_follow_the_multiplicative_schwarz_error_propagator():
    L, b = (4, 2, 2, 4), (2, 2, 2, 2)
    V = 64
    op, _, _ = make_op(L, seed=1201)
    Dm = dense_D(op, V)
    blocks = S.sap_blocks(L, b)
    n = 12 * V
    I = np.eye(n)

    def projector(colour):
        P = np.zeros((n, n), dtype=np.complex128)
        for mask, c in blocks:
            if c != colour:
                continue
            idx = np.flatnonzero(np.repeat(mask, 12))
            R = I[idx]
            P += R.T @ np.linalg.solve(R @ Dm @ R.T, R @ Dm)
        return P

    E = (I - projector(1)) @ (I - projector(0))
    eta = synth.gaussian_spinor(L, 6)
    for ncy in (1, 2):
        x = S.sap(op, blocks, eta, ncy=ncy)
        # x = M eta with 1 - M D = E^ncy, i.e. M = (1 - E^ncy) D^{-1}
        ref = (I - np.linalg.matrix_power(E, ncy)) @ np.linalg.solve(Dm, eta.reshape(-1))
        assert np.abs(x.reshape(-1) - ref).max() < 1e-11 * np.abs(ref).max(), ncy


def test_mr_block_solves_converge_to_the_exact_block_solve():
    L = (4, 2, 2, 2)
    op, _, _ = make_op(L, seed=1202, m0=0.5)
    mask = S.sap_blocks(L, (2, 2, 2, 2))[1][0]
    r = synth.gaussian_spinor(L, 7)
    exact = S.exact_block(op, mask, r)
    errs = [O.norm(S.mr_block(op, mask, r, k) - exact) / O.norm(exact) for k in (2, 8, 64)]
    assert errs[0] > errs[1] > errs[2] and errs[2] < 1e-8, errs
    assert np.all(S.mr_block(op, mask, r, 4)[~mask] == 0)  # the correction stays in the block
    # one MR step minimises ||r - alpha D r|| over complex alpha: the new residual is orthogonal to D r
    rb = np.where(mask[:, None, None], r, 0)
    ar = S.block_apply(op, mask, rb)
    r1 = rb - S.block_apply(op, mask, S.mr_block(op, mask, r, 1))
    assert abs(O.vdot(ar, r1)) <= 1e-13 * O.norm(ar) * O.norm(rb)


def test_sap_is_gauge_covariant():
    L, b = (4, 4, 2, 2), (2, 2, 2, 2)
    lat = O.Lattice(L)
    U, A = synth.gauge_field(L, 1203, 0.4)
    Om = synth.random_su3(lat.V, 81)
    al = synth.random_angles(lat.V, 82)
    U2, A2 = fields.gauge_transform(L, [lat.fwd(m) for m in range(4)], U, A, Om, al)
    op, op2 = O.Operator(lat, U, A, **PARAMS), O.Operator(lat, U2, A2, **PARAMS)

    def transform(v):
        return np.exp(1j * PARAMS["q"] * al)[:, None, None] * np.einsum("xab,xsb->xsa", Om, v)

    blocks = S.sap_blocks(L, b)
    eta = synth.gaussian_spinor(L, 8)
    lhs = S.sap(op2, blocks, transform(eta), ncy=2, nmr=4)
    rhs = transform(S.sap(op, blocks, eta, ncy=2, nmr=4))
    assert np.abs(lhs - rhs).max() < 1e-12 * np.abs(rhs).max()


def test_sap_gcr_reaches_the_papers_tolerance():
    L, b = (4, 4, 4, 4), (2, 2, 2, 2)
    op, _, _ = make_op(L, seed=1204, m0=0.1)
    blocks = S.sap_blocks(L, b)
    eta = synth.gaussian_spinor(L, 9)
    x, steps, rel = S.fgcr(op.D, eta, lambda r: S.sap(op, blocks, r, ncy=1, nmr=4), tol=1e-12, maxiter=200)
    assert rel <= 1e-12 and O.true_rel_residual(op, x, eta) <= 2e-12, (steps, rel)
    ref, _ = O.solve_eo_cg(op, eta, tol=1e-13)
    assert O.norm(x - ref) <= 1e-9 * O.norm(ref)
    _, plain, _ = S.fgcr(op.D, eta, lambda r: r, tol=1e-12, maxiter=2000)
    assert steps < plain, (steps, plain)
    # flexible GCR with a fixed identity preconditioner is GCR: a zero source gives zero at once
    z, k, _ = S.fgcr(op.D, np.zeros_like(eta), lambda r: r, tol=1e-12, maxiter=10)
    assert k == 0 and not np.any(z)


# ---- planted mistakes: each must be caught by one of the pins above ---------------------------
def _run(test, *args):
    try:
        test(*args)
        return True
    except AssertionError:
        return False


def _sap_colours_swapped(op, blocks, eta, ncy, nmr=None):
    x, r = np.zeros_like(eta), eta.copy()
    for _ in range(ncy):
        for colour in (1, 0):
            for mask, c in blocks:
                if c == colour:
                    e = S.exact_block(op, mask, r) if nmr is None else S.mr_block(op, mask, r, nmr)
                    x, r = x + e, r - op.D(e)
    return x


def _sap_stale_residual(op, blocks, eta, ncy, nmr=None):
    x, r = np.zeros_like(eta), eta.copy()
    for _ in range(ncy):
        for colour in (0, 1):
            upd = np.zeros_like(eta)
            for mask, c in blocks:
                if c == colour:
                    upd = upd + (S.exact_block(op, mask, r) if nmr is None else S.mr_block(op, mask, r, nmr))
            x = x + upd
        r = eta - op.D(x)  # residual refreshed once per cycle only: additive within the cycle
    return x


def _block_apply_leaks(op, mask, v):
    return op.D(np.where(mask[:, None, None], v, 0))  # hops leaving the block kept


def _mr_alpha_conjugated(op, mask, r, nmr):
    e = np.zeros_like(r)
    rr = np.where(mask[:, None, None], r, 0)
    for _ in range(nmr):
        ar = S.block_apply(op, mask, rr)
        alpha = O.vdot(rr, ar) / O.vdot(ar, ar)
        e, rr = e + alpha * rr, rr - alpha * ar
    return e


SAP_MUTANTS = {
    "colours in the wrong order": ("sap", _sap_colours_swapped),
    "residual not updated between colours": ("sap", _sap_stale_residual),
    "block operator keeps hops leaving the block": ("block_apply", _block_apply_leaks),
    "MR step length conjugated": ("mr_block", _mr_alpha_conjugated),
}
SAP_PINS = [test_cycles_follow_the_multiplicative_schwarz_error_propagator,
            test_mr_block_solves_converge_to_the_exact_block_solve]


@pytest.mark.parametrize("name", list(SAP_MUTANTS))
def test_sap_pins_catch_planted_mistake(name, monkeypatch):
    attr, fn = SAP_MUTANTS[name]
    monkeypatch.setattr(S, attr, fn)
    assert not all(_run(p) for p in SAP_PINS), f"no pin caught: {name}"
