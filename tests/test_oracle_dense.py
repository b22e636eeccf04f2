"""The oracle's D, Schur complement and eo-CG against dense brute force on tiny lattices."""
import numpy as np
import pytest

from oracle import qxd_oracle as O
from paper_2502_02490_gb300 import synth
from tests import dense

PARAMS = dict(q=-1 / 3, m0=-0.1, csw=1.9, csw_qed=1.0)


def build(L, cstar=False, anti=True, eps=0.3, seed=1000):
    lat = O.Lattice(L, antiperiodic=anti, cstar=cstar)
    U, A = synth.gauge_field(lat.dims, seed, eps)
    op = O.Operator(lat, U, A, **PARAMS)
    H = dense.dense_hop(lat.dims, O.hop_links(U, A, PARAMS["q"]), anti, L[1] if cstar else None)
    Dd = dense.block_diag_sites(op.C) - 0.5 * H
    return lat, op, Dd


@pytest.mark.parametrize("L,cstar,anti", [((2, 2, 2, 2), False, True), ((4, 4, 4, 4), False, True),
                                          ((2, 4, 2, 4), False, False), ((2, 2, 2, 2), True, True)])
def test_dense_equals_oracle(L, cstar, anti):
    lat, op, Dd = build(L, cstar, anti)
    psi = synth.gaussian_spinor(lat.dims, 9)
    got = op.D(psi).ravel()
    want = Dd @ psi.ravel()
    assert np.abs(got - want).max() < 1e-13 * np.abs(want).max()
    # gamma5-hermiticity of the dense matrix itself
    G5 = np.kron(np.eye(lat.V), np.kron(np.diag([1, 1, -1, -1]), np.eye(3)))
    assert np.abs(Dd.conj().T - G5 @ Dd @ G5).max() < 1e-13


def test_unit_vector_columns_2to4():
    lat, op, Dd = build((2, 2, 2, 2))
    for j in range(0, 12 * lat.V, 7):
        e = np.zeros(12 * lat.V, dtype=complex)
        e[j] = 1
        assert np.abs(op.D(e.reshape(-1, 4, 3)).ravel() - Dd[:, j]).max() < 1e-14


@pytest.mark.parametrize("L,cstar", [((4, 4, 4, 4), False), ((2, 2, 2, 2), True)])
def test_eo_cg_matches_dense_solve(L, cstar):
    lat, op, Dd = build(L, cstar)
    eta = synth.gaussian_spinor(lat.dims, 2000)
    psi, info = O.solve_eo_cg(op, eta, tol=1e-12)
    ref = np.linalg.solve(Dd, eta.ravel())
    kappa = np.linalg.cond(Dd)
    assert info["true_rel_residual"] <= 1e-12
    assert np.linalg.norm(psi.ravel() - ref) / np.linalg.norm(ref) <= kappa * 1e-12


def test_schur_determinant_identity():
    lat, op, Dd = build((2, 2, 2, 2), eps=0.5)
    even = np.where(lat.par == 0)[0]
    odd = np.where(lat.par == 1)[0]
    cols = []
    for x in even:
        for k in range(12):
            v = np.zeros((lat.V, 4, 3), dtype=complex)
            v[x].reshape(12)[k] = 1
            cols.append(op.Dhat(v)[even].ravel())
    Dhat = np.array(cols).T
    det_full = np.linalg.slogdet(Dd)
    det_oo = np.linalg.slogdet(op.C[odd])
    det_hat = np.linalg.slogdet(Dhat)
    log_full = np.log(det_full[0]) + det_full[1]
    log_parts = np.sum(np.log(det_oo[0]) + det_oo[1]) + np.log(det_hat[0]) + det_hat[1]
    d = log_full - log_parts
    assert abs(d.real) < 1e-10 and abs((d.imag + np.pi) % (2 * np.pi) - np.pi) < 1e-10


def test_schur_block_structure_against_dense():
    """Dhat = D_ee - D_eo D_oo^-1 D_oe computed from the dense blocks equals the oracle's Dhat."""
    lat, op, Dd = build((2, 4, 2, 2))
    idx = np.arange(12 * lat.V).reshape(lat.V, 12)
    e = idx[lat.par == 0].ravel()
    o = idx[lat.par == 1].ravel()
    Dh = Dd[np.ix_(e, e)] - Dd[np.ix_(e, o)] @ np.linalg.solve(Dd[np.ix_(o, o)], Dd[np.ix_(o, e)])
    psi = synth.gaussian_spinor(lat.dims, 4)
    psi[lat.par == 1] = 0
    got = op.Dhat(psi)[lat.par == 0].ravel()
    assert np.abs(got - Dh @ psi[lat.par == 0].ravel()).max() < 1e-13 * np.abs(got).max()


@pytest.mark.parametrize("L,cstar", [((2, 4, 2, 2), False), ((4, 2, 2, 4), False), ((2, 2, 2, 2), True)])
def test_sampled_site_schur_complement_against_dense(L, cstar):
    """Dhat_at_sites (and its gamma5 dagger) at sampled even sites equals the dense Schur
    complement D_ee - D_eo D_oo^-1 D_oe built from the edge-loop matrix; odd entries of the
    input field are ignored."""
    lat, op, Dd = build(L, cstar=cstar)
    U, A = synth.gauge_field(lat.dims, 1000, 0.3)  # the field build() used
    idx = np.arange(12 * lat.V).reshape(lat.V, 12)
    e = idx[lat.par == 0].ravel()
    o = idx[lat.par == 1].ravel()
    Dh = Dd[np.ix_(e, e)] - Dd[np.ix_(e, o)] @ np.linalg.solve(Dd[np.ix_(o, o)], Dd[np.ix_(o, e)])
    psi = synth.gaussian_spinor(lat.dims, 6)
    g5 = np.kron(np.eye(len(e) // 12), np.kron(np.diag([1, 1, -1, -1]), np.eye(3)))
    even_sites = np.flatnonzero(lat.par == 0)
    sites = even_sites[np.random.default_rng(1).choice(len(even_sites), 5, replace=False)]
    rank = np.searchsorted(even_sites, sites)
    for dagger, M in ((False, Dh), (True, g5 @ Dh @ g5)):
        ref = (M @ psi[lat.par == 0].ravel()).reshape(-1, 4, 3)[rank]
        got = O.Dhat_at_sites(lat, U, A, PARAMS["q"], PARAMS["m0"],
                              PARAMS["csw"], PARAMS["csw_qed"], psi, sites, dagger=dagger)
        assert np.abs(got - ref).max() < 1e-13 * np.abs(ref).max(), dagger
    with pytest.raises(ValueError):
        O.Dhat_at_sites(lat, U, A, PARAMS["q"], PARAMS["m0"],
                        PARAMS["csw"], PARAMS["csw_qed"], psi, np.flatnonzero(lat.par == 1)[:1])
