"""Plant plausible mistakes in the oracle (on the CPU) and check that the pins catch each one."""
import numpy as np
import pytest

from oracle import qxd_oracle as O
from paper_2502_02490_gb300 import synth
from tests import dense, fields
from tests.test_oracle_free import D_of_p, momentum

PARAMS = dict(q=-1 / 3, m0=-0.1, csw=1.9, csw_qed=1.0)


def pin_free_field():
    L = (4, 4, 4, 4)
    U, A = fields.unit_field(L)
    op = O.Operator(O.Lattice(L), U, A, **PARAMS)
    p = momentum(L, (1, 1, 0, 1), True)
    u = np.arange(12).reshape(4, 3) + 0.5j
    return np.abs(op.D(fields.plane_wave(L, p, u)) - fields.plane_wave(L, p, D_of_p(p, PARAMS["m0"]) @ u)).max() < 1e-12


def pin_dense():
    L = (2, 2, 2, 2)
    lat = O.Lattice(L)
    U, A = synth.gauge_field(L, 1000, 0.3)
    op = O.Operator(lat, U, A, **PARAMS)
    H = dense.dense_hop(L, U * np.exp(1j * PARAMS["q"] * A)[..., None, None], True)
    psi = synth.gaussian_spinor(L, 1)
    want = (dense.block_diag_sites(op.C) - 0.5 * H) @ psi.ravel()
    return np.abs(op.D(psi).ravel() - want).max() < 1e-12


def pin_flux():
    L, mu, nu = (4, 4, 4, 4), 1, 2
    lat = O.Lattice(L)
    phi, B = fields.uniform_flux_angles(L, mu, nu)
    k = np.array([1, 2, -3])
    U = np.zeros((lat.V, 4, 3, 3), dtype=complex)
    for m in range(4):
        U[:, m] = np.exp(1j * phi[:, m, None] * k)[:, :, None] * np.eye(3)
    d = 1j * np.sin(k * B)
    F = np.diag(d - d.sum() / 3)
    C = O.clover_matrix(lat, U, phi, q=0.5, m0=0.0, csw=1.3, csw_qed=0.7)
    want = 4 * np.eye(12) + 1.3 * 0.5j * np.kron(O.sigma(mu, nu), F) \
        + 0.5 * 0.7 * 0.5j * np.kron(O.sigma(mu, nu) * 1j * np.sin(B), np.eye(3))
    return np.abs(C - want).max() < 1e-13


def pin_schur():
    L = (2, 4, 2, 2)
    lat = O.Lattice(L)
    U, A = synth.gauge_field(L, 1000, 0.3)
    op = O.Operator(lat, U, A, **PARAMS)
    eta = synth.gaussian_spinor(L, 3)
    psi, info = O.solve_eo_cg(op, eta, tol=1e-11, maxiter=3000, max_outer=2)
    return np.linalg.norm(eta - op.D(psi)) / np.linalg.norm(eta) < 1e-10


PINS = [pin_free_field, pin_dense, pin_flux, pin_schur]


def _hop_variant(fwd_proj=+1, bwd_dagger=True, use_sign=True):
    def hop(lat, W, psi):
        out = np.zeros_like(psi)
        for mu in range(4):
            f, sf = lat.neighbour(mu, +1)
            b, sb = lat.neighbour(mu, -1)
            if not use_sign:
                sf, sb = np.ones_like(sf), np.ones_like(sb)
            t = np.einsum("xab,xtb->xta", W[:, mu], psi[f]) * sf[:, None, None]
            out += np.einsum("st,xta->xsa", O.I4 - fwd_proj * O.GAMMA[mu], t)
            Wb = O.dag(W[b, mu]) if bwd_dagger else np.swapaxes(W[b, mu], -1, -2)
            t = np.einsum("xab,xtb->xta", Wb, psi[b]) * sb[:, None, None]
            out += np.einsum("st,xta->xsa", O.I4 + O.GAMMA[mu], t)
        return out
    return hop


def _leaves_drop_third(lat, M, mu, nu):
    fm, fn, bm, bn = lat.fwd(mu), lat.fwd(nu), lat.bwd(mu), lat.bwd(nu)
    Um, Un = M[:, mu], M[:, nu]
    q = Um @ Un[fm] @ O.dag(Um[fn]) @ O.dag(Un)
    q = q + Un @ O.dag(Um[bm[fn]]) @ O.dag(Un[bm]) @ Um[bm]
    q = q + O.dag(Un[bn]) @ Um[bn] @ Un[fm[bn]] @ O.dag(Um)
    return q


def _su3_not_traceless(lat, U, mu, nu, sites=None):
    return (O._leaves(lat, U, mu, nu) - O._leaves(lat, U, nu, mu)) / 8.0


def _dhat_wrong_sign(self, psi_e):
    e, o = self.even, self.odd
    t = self.Doo_inv(self.block(psi_e, o, e))
    return self.block(psi_e, e, e) + self.block(t, e, o)


MUTANTS = {
    "forward projector 1+gamma": ("hop", _hop_variant(fwd_proj=-1)),
    "backward link not conjugated": ("hop", _hop_variant(bwd_dagger=False)),
    "antiperiodic sign dropped": ("hop", _hop_variant(use_sign=False)),
    "third clover leaf dropped": ("_leaves", _leaves_drop_third),
    "SU(3) field strength not traceless": ("field_strength_su3", _su3_not_traceless),
}


@pytest.mark.parametrize("name", list(MUTANTS))
def test_pins_catch_planted_mistake(name, monkeypatch):
    attr, fn = MUTANTS[name]
    assert all(p() for p in PINS[:3])  # all pins pass on the real oracle
    monkeypatch.setattr(O, attr, fn)
    assert not all(p() for p in PINS[:3]), f"no pin caught: {name}"


def test_pins_catch_wrong_schur_sign(monkeypatch):
    assert pin_schur()
    monkeypatch.setattr(O.Operator, "Dhat", _dhat_wrong_sign)
    assert not pin_schur()
