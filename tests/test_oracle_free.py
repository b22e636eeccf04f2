"""Free-field (U = 1) and constant-phase closed forms for D (pins hop signs, m0, BC, basis)."""
import numpy as np
import pytest

from oracle import qxd_oracle as O
from tests import fields


def momentum(L, n, antiperiodic):
    p = 2 * np.pi * np.asarray(n, dtype=float) / np.asarray(L)
    if antiperiodic:
        p[0] = (2 * n[0] + 1) * np.pi / L[0]
    return p


def D_of_p(p, m0):
    """D(p) = m0 + sum_mu (1 - cos p_mu) + i sum_mu gamma_mu sin p_mu (4x4)."""
    return (m0 + np.sum(1 - np.cos(p))) * np.eye(4) + 1j * sum(O.GAMMA[mu] * np.sin(p[mu]) for mu in range(4))


@pytest.mark.parametrize("L,anti", [((4, 4, 4, 4), True), ((6, 4, 2, 4), False), ((4, 2, 6, 8), True)])
@pytest.mark.parametrize("n", [(0, 0, 0, 0), (1, 1, 0, 1), (2, 1, 1, 3)])
def test_free_field_plane_wave(L, anti, n):
    m0 = -0.1
    U, A = fields.unit_field(L)
    lat = O.Lattice(L, antiperiodic=anti)
    op = O.Operator(lat, U, A, q=-1 / 3, m0=m0, csw=1.9, csw_qed=1.0)
    p = momentum(L, n, anti)
    u = np.random.default_rng(1).standard_normal((4, 3)) + 1j * np.random.default_rng(2).standard_normal((4, 3))
    psi = fields.plane_wave(L, p, u)
    expect = fields.plane_wave(L, p, D_of_p(p, m0) @ u)
    assert np.abs(op.D(psi) - expect).max() < 1e-13


def test_constant_u1_phase_shifts_momentum():
    L, m0, q = (4, 4, 6, 2), 0.3, 2 / 3
    a = np.array([0.2, -0.7, 1.1, 0.4])
    U, _ = fields.unit_field(L)
    A = np.broadcast_to(a, (U.shape[0], 4)).copy()
    lat = O.Lattice(L, antiperiodic=True)
    op = O.Operator(lat, U, A, q=q, m0=m0, csw=1.9, csw_qed=1.0)
    p = momentum(L, (1, 0, 1, 1), True)
    u = np.arange(12).reshape(4, 3) * (1 + 0.5j)
    psi = fields.plane_wave(L, p, u)
    expect = fields.plane_wave(L, p, D_of_p(p + q * a, m0) @ u)
    assert np.abs(op.D(psi) - expect).max() < 1e-12


def test_constant_diagonal_su3_shifts_momentum_per_colour():
    # U_mu = diag(e^{i t_mu}, e^{i s_mu}, e^{-i(t_mu+s_mu)}): colour a sees momentum p + phase_a.
    L, m0 = (4, 4, 4, 4), -0.2
    t = np.array([0.3, -0.2, 0.5, 0.1])
    s = np.array([-0.4, 0.6, 0.2, -0.3])
    ph = np.stack([t, s, -(t + s)], axis=1)  # (mu, colour)
    V = 256
    U = np.zeros((V, 4, 3, 3), dtype=np.complex128)
    for mu in range(4):
        U[:, mu] = np.diag(np.exp(1j * ph[mu]))
    lat = O.Lattice(L, antiperiodic=True)
    op = O.Operator(lat, U, np.zeros((V, 4)), q=0.0, m0=m0, csw=1.9, csw_qed=0.0)
    p = momentum(L, (0, 1, 2, 1), True)
    u = np.random.default_rng(5).standard_normal((4, 3)) + 0j
    psi = fields.plane_wave(L, p, u)
    got = op.D(psi)
    for a in range(3):
        e = fields.plane_wave(L, p, (D_of_p(p + ph[:, a], m0) @ u[:, a])[:, None])[..., 0]
        assert np.abs(got[:, :, a] - e).max() < 1e-12


def test_free_field_solve_matches_closed_form_inverse():
    L, m0 = (4, 4, 4, 4), 0.05
    U, A = fields.unit_field(L)
    lat = O.Lattice(L, antiperiodic=True)
    op = O.Operator(lat, U, A, q=-1 / 3, m0=m0, csw=1.9, csw_qed=1.0)
    p = momentum(L, (1, 2, 0, 1), True)
    u = np.random.default_rng(3).standard_normal((4, 3)) + 1j
    eta = fields.plane_wave(L, p, u)
    psi, info = O.solve_eo_cg(op, eta, tol=1e-12)
    expect = fields.plane_wave(L, p, np.linalg.solve(D_of_p(p, m0), u))
    assert info["true_rel_residual"] <= 1e-12
    assert np.abs(psi - expect).max() < 1e-10
