"""C* boundary conditions (Sec. 4.2): doubling in x with charge-conjugated mirror fields."""
import numpy as np
import pytest

from oracle import qxd_oracle as O
from paper_2502_02490_gb300 import synth

PARAMS = dict(q=-1 / 3, m0=-0.1, csw=1.9, csw_qed=1.0)


def conj_matrix():
    """M with M gamma_mu^* M^-1 = gamma_mu for all mu, found as the null space of a linear system."""
    rows = []
    for g in O.GAMMA:
        # vec(M g^*) - vec(g M) = (g^*^T kron I - I kron g) vec(M) in column-major vec
        rows.append(np.kron(g.conj().T, np.eye(4)) - np.kron(np.eye(4), g))
    _, s, vh = np.linalg.svd(np.vstack(rows))
    assert s[-1] < 1e-12 and s[-2] > 1e-3
    M = vh[-1].conj().reshape(4, 4, order="F")
    return M / np.sqrt(abs(np.linalg.det(M)) ** 0.5)


def mirror(psi, dims, L1, M):
    """(T psi)(x) = M psi(x - L1 e1)^* on the doubled lattice."""
    p = psi.reshape(dims + (4, 3))
    p = np.roll(p, L1, axis=1)
    return np.einsum("st,...ta->...sa", M, p.conj()).reshape(-1, 4, 3)


def cstar_op(L, seed=1005, eps=0.35):
    lat = O.Lattice(L, antiperiodic=True, cstar=True)
    U, A = synth.gauge_field(L, seed, eps)
    U2, A2 = O.cstar_double_gauge(U, A, L)
    return lat, O.Operator(lat, U2, A2, **PARAMS), (U, A)


@pytest.mark.parametrize("L", [(2, 2, 2, 2), (4, 2, 4, 2)])
def test_D_commutes_with_charge_conjugated_shift(L):
    M = conj_matrix()
    for mu in range(4):
        assert np.abs(M @ O.GAMMA[mu].conj() @ np.linalg.inv(M) - O.GAMMA[mu]).max() < 1e-12
    lat, op, _ = cstar_op(L)
    psi = synth.gaussian_spinor(lat.dims, 6)
    lhs = op.D(mirror(psi, lat.dims, L[1], M))
    rhs = mirror(op.D(psi), lat.dims, L[1], M)
    assert np.abs(lhs - rhs).max() < 1e-13 * np.abs(rhs).max()


def test_doubled_hop_equals_direct_cstar_definition():
    """On mirror-symmetric fields the doubled hop equals the C* hop on the physical lattice:
    a hop across any spatial boundary meets the charge conjugate M psi^* (and the conjugate link
    when it comes from the far side)."""
    L = (2, 4, 2, 4)
    M = conj_matrix()
    lat, op, (U, A) = cstar_op(L)
    q = PARAMS["q"]
    W = O.hop_links(U, A, q)
    phys = np.random.default_rng(0).standard_normal((int(np.prod(L)), 4, 3)) * (1 + 0.3j)
    full = np.concatenate([phys.reshape(L + (4, 3)),
                           np.einsum("st,...ta->...sa", M, phys.reshape(L + (4, 3)).conj())], axis=1)
    got = O.hop(lat, op.W, full.reshape(-1, 4, 3)).reshape(lat.dims + (4, 3))[:, : L[1]]
    # direct definition on the physical lattice
    want = np.zeros(L + (4, 3), dtype=complex)
    Wr = W.reshape(L + (4, 3, 3))
    ps = phys.reshape(L + (4, 3))
    for c in np.ndindex(*L):
        acc = np.zeros((4, 3), dtype=complex)
        for mu in range(4):
            # forward
            y = list(c); y[mu] += 1; crossed = y[mu] == L[mu]; y[mu] %= L[mu]
            sign = -1.0 if (mu == 0 and crossed) else 1.0
            v = ps[tuple(y)]
            if crossed and mu > 0:
                v = M @ v.conj()
            acc += sign * (np.eye(4) - O.GAMMA[mu]) @ (Wr[c][mu] @ v.T).T
            # backward
            y = list(c); y[mu] -= 1; crossed = y[mu] < 0; y[mu] %= L[mu]
            sign = -1.0 if (mu == 0 and crossed) else 1.0
            v = ps[tuple(y)]
            link = Wr[tuple(y)][mu]
            if crossed and mu > 0:
                v = M @ v.conj()
                link = link.conj()
            acc += sign * (np.eye(4) + O.GAMMA[mu]) @ (link.conj().T @ v.T).T
        want[c] = acc
    assert np.abs(got - want).max() < 1e-13 * np.abs(want).max()


def test_solution_of_mirrored_source_is_mirrored_solution():
    """T (psi -> M psi^* shifted by L1) is antilinear with T^2 = -1 (M M^* = -1), so no field is
    T-invariant; the consequence of [D, T] = 0 for solves is D psi = eta  =>  D (T psi) = T eta."""
    L = (2, 2, 2, 2)
    M = conj_matrix()
    assert np.abs(M @ M.conj() + np.eye(4)).max() < 1e-12
    lat, op, _ = cstar_op(L)
    eta = synth.gaussian_spinor(lat.dims, 7)
    psi, info = O.solve_eo_cg(op, eta, tol=1e-12)
    psi2, info2 = O.solve_eo_cg(op, mirror(eta, lat.dims, L[1], M), tol=1e-12)
    assert info["true_rel_residual"] <= 1e-12 and info2["true_rel_residual"] <= 1e-12
    assert np.abs(mirror(psi, lat.dims, L[1], M) - psi2).max() < 1e-10 * np.abs(psi).max()
