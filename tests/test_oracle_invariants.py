"""Invariants that pin the oracle's D and clover term on random fields."""
import numpy as np
import pytest

from oracle import qxd_oracle as O
from paper_2502_02490_gb300 import synth
from tests import fields

PARAMS = dict(q=-1 / 3, m0=-0.1, csw=1.9, csw_qed=1.0)


def rand_spinor(L, seed):
    return synth.gaussian_spinor(L, seed)


@pytest.mark.parametrize("L,cstar", [((4, 4, 4, 4), False), ((2, 4, 2, 6), False), ((4, 2, 2, 2), True)])
def test_gamma5_hermiticity(L, cstar):
    lat = O.Lattice(L, antiperiodic=True, cstar=cstar)
    U, A = synth.gauge_field(lat.dims, 1000, 0.3)
    op = O.Operator(lat, U, A, **PARAMS)
    phi, psi = rand_spinor(lat.dims, 1), rand_spinor(lat.dims, 2)
    lhs = O.vdot(phi, op.D(psi))
    rhs = O.vdot(O.g5(op.D(O.g5(phi))), psi)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)
    # the starred form of the same identity: <phi, D psi> = <psi, g5 D g5 phi>^*
    assert abs(lhs - np.conj(O.vdot(psi, O.g5(op.D(O.g5(phi)))))) < 1e-12 * abs(lhs)


@pytest.mark.parametrize("L,cstar,anti", [((4, 4, 4, 4), False, True), ((2, 4, 2, 4), False, False),
                                          ((2, 2, 4, 2), True, True)])
def test_gauge_covariance(L, cstar, anti):
    lat = O.Lattice(L, antiperiodic=anti, cstar=cstar)
    U, A = synth.gauge_field(lat.dims, 1001, 0.4)
    V = lat.V
    Om = synth.random_su3(V, 77)
    al = synth.random_angles(V, 78)
    U2, A2 = fields.gauge_transform(lat.dims, [lat.fwd(m) for m in range(4)], U, A, Om, al)
    q = PARAMS["q"]
    op, op2 = O.Operator(lat, U, A, **PARAMS), O.Operator(lat, U2, A2, **PARAMS)
    psi = rand_spinor(lat.dims, 3)

    def transform(v):
        return np.exp(1j * q * al)[:, None, None] * np.einsum("xab,xsb->xsa", Om, v)

    lhs = op2.D(transform(psi))
    rhs = transform(op.D(psi))
    assert np.abs(lhs - rhs).max() < 1e-13 * np.abs(rhs).max()


def test_clover_hermitian_and_chirality_block_diagonal():
    L = (4, 4, 2, 4)
    lat = O.Lattice(L)
    U, A = synth.gauge_field(L, 1002, 0.5)
    C = O.clover_matrix(lat, U, A, **PARAMS)
    assert np.abs(C - O.dag(C)).max() < 1e-15 * 10
    assert np.abs(C[:, :6, 6:]).max() < 1e-15 and np.abs(C[:, 6:, :6]).max() < 1e-15
    # commutes with gamma5 x 1_colour
    G = np.kron(O.GAMMA5, np.eye(3))
    assert np.abs(G @ C - C @ G).max() < 1e-15


def test_clover_vanishes_on_pure_gauge_and_is_linear():
    L = (2, 4, 4, 2)
    lat = O.Lattice(L)
    V = lat.V
    Om = synth.random_su3(V, 31)
    al = synth.random_angles(V, 32)
    U0, A0 = fields.unit_field(L)
    U, A = fields.gauge_transform(L, [lat.fwd(m) for m in range(4)], U0, A0, Om, al)
    C = O.clover_matrix(lat, U, A, q=0.7, m0=0.25, csw=1.9, csw_qed=1.3)
    assert np.abs(C - 4.25 * np.eye(12)).max() < 1e-14
    U, A = synth.gauge_field(L, 1003, 0.4)
    c0 = O.clover_matrix(lat, U, A, q=0.5, m0=0.0, csw=0.0, csw_qed=0.0)
    c1 = O.clover_matrix(lat, U, A, q=0.5, m0=0.0, csw=1.0, csw_qed=0.0)
    c2 = O.clover_matrix(lat, U, A, q=0.5, m0=0.0, csw=0.0, csw_qed=1.0)
    c3 = O.clover_matrix(lat, U, A, q=0.5, m0=0.0, csw=2.5, csw_qed=-1.5)
    assert np.abs((c3 - c0) - (2.5 * (c1 - c0) - 1.5 * (c2 - c0))).max() < 1e-14


@pytest.mark.parametrize("mu,nu", [(0, 1), (2, 3), (1, 3), (3, 0)])
def test_uniform_u1_flux_closed_form(mu, nu):
    """Every plaquette of the (mu,nu) plane carries angle B: Fhat^U(1)_{mu nu} = i sin B, others 0,
    and the clover term equals (4 + m0) + q c_sw^QED (i/2) sigma_{mu nu} (i sin B) exactly."""
    L = (4, 6, 4, 2)
    lat = O.Lattice(L, antiperiodic=True)
    A, B = fields.uniform_flux_angles(L, mu, nu, n=1)
    for a in range(4):
        for b in range(4):
            if a == b:
                continue
            f = O.field_strength_u1(lat, A, a, b)
            want = 1j * np.sin(B) * ((a, b) == (mu, nu)) - 1j * np.sin(B) * ((a, b) == (nu, mu))
            assert np.abs(f - want).max() < 1e-15
    U, _ = fields.unit_field(L)
    q, cq, m0 = -1 / 3, 1.0, 0.1
    C = O.clover_matrix(lat, U, A, q=q, m0=m0, csw=1.9, csw_qed=cq)
    want = (4 + m0) * np.eye(12) + q * cq * 0.5j * np.kron(O.sigma(mu, nu) * 1j * np.sin(B), np.eye(3))
    assert np.abs(C - want).max() < 1e-14


def test_uniform_su3_diagonal_flux_closed_form():
    """SU(3) links diag(e^{i k1 phi}, e^{i k2 phi}, e^{-i (k1+k2) phi}) built from a uniform U(1) flux:
    Fhat = diag(i sin(k_a B)) minus its trace / 3."""
    L, mu, nu = (4, 4, 4, 4), 1, 2
    lat = O.Lattice(L)
    phi, B = fields.uniform_flux_angles(L, mu, nu, n=1)
    k = np.array([1, 2, -3])
    U = np.zeros((lat.V, 4, 3, 3), dtype=np.complex128)
    for m in range(4):
        U[:, m] = np.exp(1j * phi[:, m, None] * k)[:, :, None] * np.eye(3)
    F = O.field_strength_su3(lat, U, mu, nu)
    d = 1j * np.sin(k * B)
    want = np.diag(d - d.sum() / 3)
    assert np.abs(F - want).max() < 1e-15
    assert np.abs(O.field_strength_su3(lat, U, 0, 3)).max() < 1e-15


@pytest.mark.parametrize("L,cstar", [((4, 4, 2, 6), False), ((2, 2, 4, 2), True)])
def test_sampled_sites_equal_full_operator(L, cstar):
    lat = O.Lattice(L, antiperiodic=True, cstar=cstar)
    U, A = synth.gauge_field(lat.dims, 1004, 0.4)
    op = O.Operator(lat, U, A, **PARAMS)
    psi = rand_spinor(lat.dims, 5)
    sites = np.random.default_rng(0).choice(lat.V, 17, replace=False)
    full = op.D(psi)[sites]
    got = O.D_at_sites(lat, U, A, PARAMS["q"], PARAMS["m0"], PARAMS["csw"], PARAMS["csw_qed"], psi, sites)
    assert np.abs(got - full).max() < 1e-14 * np.abs(full).max()
