"""Pins for the gamma-matrix basis (chiral, gamma5 diagonal) and sigma_{mu nu}."""
import numpy as np

from oracle import qxd_oracle as O


def test_clifford_algebra_and_hermiticity():
    for mu in range(4):
        assert np.allclose(O.GAMMA[mu], O.GAMMA[mu].conj().T)
        for nu in range(4):
            ac = O.GAMMA[mu] @ O.GAMMA[nu] + O.GAMMA[nu] @ O.GAMMA[mu]
            assert np.allclose(ac, 2 * (mu == nu) * np.eye(4))


def test_gamma5_is_chirality_diagonal():
    assert np.allclose(O.GAMMA5, np.diag([1, 1, -1, -1]))
    for mu in range(4):
        assert np.allclose(O.GAMMA5 @ O.GAMMA[mu], -O.GAMMA[mu] @ O.GAMMA5)


def test_sigma_block_diagonal_hermitian():
    for mu in range(4):
        for nu in range(4):
            s = O.sigma(mu, nu)
            assert np.allclose(s, s.conj().T)
            assert np.allclose(s[:2, 2:], 0) and np.allclose(s[2:, :2], 0)
            assert np.allclose(s, -O.sigma(nu, mu))
