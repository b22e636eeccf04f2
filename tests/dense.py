"""Brute-force dense Wilson hopping matrix from an explicit edge loop (test helper).

Written independently of the oracle's vectorised hop: its own gamma matrices (the chiral
basis), its own coordinate arithmetic, Kronecker products per edge.  Sizes: 12V x 12V.
"""
import numpy as np

_s = [np.array([[0, 1], [1, 0]]), np.array([[0, -1j], [1j, 0]]), np.array([[1, 0], [0, -1]])]
_Z, _I = np.zeros((2, 2)), np.eye(2)
GAMMA = [np.block([[_Z, -_I], [-_I, _Z]]).astype(complex)] + \
        [np.block([[_Z, -1j * s], [1j * s, _Z]]).astype(complex) for s in _s]


def site_index(c, L):
    return ((c[0] * L[1] + c[1]) * L[2] + c[2]) * L[3] + c[3]


def dense_hop(L, W, antiperiodic=True, cstar_L1=None):
    """Matrix H with (H psi)_x = sum_mu (1-g_mu) W_mu(x) psi_{x+mu} + (1+g_mu) W_mu(x-mu)^+ psi_{x-mu}.

    cstar_L1: if given, the lattice is the C*-doubled one and hops across the y/z boundary
    shift x by cstar_L1 (mod L[1])."""
    V = int(np.prod(L))
    H = np.zeros((12 * V, 12 * V), dtype=complex)
    for x in range(V):
        c = list(np.unravel_index(x, L))
        for mu in range(4):
            for step in (+1, -1):
                y = list(c)
                y[mu] += step
                sign = 1.0
                if y[mu] < 0 or y[mu] >= L[mu]:
                    y[mu] %= L[mu]
                    if mu == 0 and antiperiodic:
                        sign = -1.0
                    if cstar_L1 is not None and mu in (2, 3):
                        y[1] = (y[1] + cstar_L1) % L[1]
                iy = site_index(y, L)
                if step == +1:
                    blk = np.kron(np.eye(4) - GAMMA[mu], W[x, mu])
                else:
                    blk = np.kron(np.eye(4) + GAMMA[mu], W[iy, mu].conj().T)
                H[12 * x:12 * x + 12, 12 * iy:12 * iy + 12] += sign * blk
    return H


def block_diag_sites(C):
    """Dense matrix with the site matrices C (V, 12, 12) on the diagonal."""
    V = C.shape[0]
    M = np.zeros((12 * V, 12 * V), dtype=complex)
    for x in range(V):
        M[12 * x:12 * x + 12, 12 * x:12 * x + 12] = C[x]
    return M
