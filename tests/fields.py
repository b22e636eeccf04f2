"""Test-side field recipes built on the seeded generators (no operator arithmetic here)."""
import numpy as np

from paper_2502_02490_gb300 import synth


def coords(L):
    return np.stack(np.meshgrid(*[np.arange(n) for n in L], indexing="ij"), axis=-1).reshape(-1, 4)


def random_config(L, seed=1000, eps=0.3):
    U, A = synth.gauge_field(L, seed, eps)
    return U, A


def unit_field(L):
    V = synth.volume(L)
    U = np.broadcast_to(np.eye(3, dtype=np.complex128), (V, 4, 3, 3)).copy()
    return U, np.zeros((V, 4))


def uniform_flux_angles(L, mu, nu, n=1):
    """U(1) angles with the same plaquette angle B = 2 pi n / (L_mu L_nu) on every plaquette of
    the (mu, nu) plane and zero flux elsewhere (periodic lattice).

    A_nu(x) = B x_mu everywhere; A_mu(x) = -B L_mu x_nu on the last mu-slice closes the torus.
    """
    c = coords(L)
    B = 2 * np.pi * n / (L[mu] * L[nu])
    A = np.zeros((len(c), 4))
    A[:, nu] = B * c[:, mu]
    last = c[:, mu] == L[mu] - 1
    A[last, mu] = -B * L[mu] * c[last, nu]
    return A, B


def plane_wave(L, p, u):
    """psi(x) = exp(i p.x) u for a spinor u (4, 3)."""
    c = coords(L)
    ph = np.exp(1j * (c @ np.asarray(p, dtype=float)))
    return ph[:, None, None] * u[None]


def gauge_transform(L, nbr_fwd, U, A, Omega, alpha):
    """U_mu(x) -> Omega(x) U_mu(x) Omega(x+mu)^+,  A_mu(x) -> A_mu(x) + alpha(x) - alpha(x+mu).

    nbr_fwd[mu] is the index array of x + mu_hat (the lattice's own neighbour map)."""
    U2 = np.empty_like(U)
    A2 = np.empty_like(A)
    for mu in range(4):
        f = nbr_fwd[mu]
        U2[:, mu] = Omega @ U[:, mu] @ np.conj(np.swapaxes(Omega[f], -1, -2))
        A2[:, mu] = A[:, mu] + alpha - alpha[f]
    return U2, A2
