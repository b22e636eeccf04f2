"""Plain FP64 CPU oracle for the O(a)-improved QCD+QED Wilson-clover Dirac operator.

TEST INFRASTRUCTURE ONLY.  This module is the slow, obviously correct statement of what
the GPU path computes.  Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU
baseline leg may import it; the product library never does, and the two share no code.

Everything is numpy complex128/float64, vectorised over lattice sites only: each step is
the definition written out site by site (explicit 4x4 gamma matrices acting on full
12-component spinors, no spin projection, no even-odd tricks inside D).

Arrays are in lexicographic site order (Eq. lexi of Sec. 4.1.1: x3 fastest, time first),
shapes: spinor (V, 4, 3) [site, spin alpha, colour a]; links (V, 4, 3, 3) [site, mu, row,
col], row-major (Sec. 2 and Sec. 4.1.4); U(1) angles (V, 4).

Conventions taken where the paper is silent (each also listed in the design notes):
  * gamma basis: openQCD's chiral basis, gamma5 = diag(1, 1, -1, -1); upper 6x6 clover block
    = spins 0,1 (chirality +).  The paper needs a chiral basis for its two 6x6 blocks (Sec. 2).
  * sigma_{mu nu} = (i/2)[gamma_mu, gamma_nu]; the clover sum runs over all ordered mu != nu.
  * Fhat_{mu nu} = (Q_{mu nu} - Q_{nu mu}) / 8, Q the sum of the four plaquette leaves at x.
    SU(3): made traceless.  U(1): built from the unit-charge phases exp(iA), scaled by q.
  * 4 + m0 sits in the clover blocks, so D_ee = A_ee and D_oo = A_oo.
  * antiperiodic time: factor -1 on every hop across t = T-1 <-> 0, not on plaquettes.
  * Schur complement Dhat = D_ee - D_eo D_oo^-1 D_oe (non-symmetric form).
  * C* (Sec. 4.2): lattice doubled in x; mirror links U* and angles -A; a hop across the y
    or z boundary also shifts x by L1 (mod 2 L1).
"""
from __future__ import annotations

import numpy as np

# ---------------------------------------------------------------------------------------
# Gamma matrices (chiral basis) and sigma_{mu nu}
# ---------------------------------------------------------------------------------------
_I2 = np.eye(2, dtype=np.complex128)
_Z2 = np.zeros((2, 2), dtype=np.complex128)
PAULI = [
    np.array([[0, 1], [1, 0]], dtype=np.complex128),
    np.array([[0, -1j], [1j, 0]], dtype=np.complex128),
    np.array([[1, 0], [0, -1]], dtype=np.complex128),
]


def _block(a, b, c, d):
    return np.block([[a, b], [c, d]])


GAMMA = [_block(_Z2, -_I2, -_I2, _Z2)] + [_block(_Z2, -1j * s, 1j * s, _Z2) for s in PAULI]
GAMMA5 = GAMMA[0] @ GAMMA[1] @ GAMMA[2] @ GAMMA[3]
I4 = np.eye(4, dtype=np.complex128)


def sigma(mu, nu):
    """sigma_{mu nu} = (i/2)[gamma_mu, gamma_nu]."""
    return 0.5j * (GAMMA[mu] @ GAMMA[nu] - GAMMA[nu] @ GAMMA[mu])


def dag(m):
    """Hermitian conjugate over the last two axes."""
    return np.conj(np.swapaxes(m, -1, -2))


# ---------------------------------------------------------------------------------------
# Site indexing: Eq. lexi and Eq. ipt (Sec. 4.1.1)
# ---------------------------------------------------------------------------------------
def lexi(x, L):
    """Lambda(x, L) = L3 L2 L1 x0 + L3 L2 x1 + L3 x2 + x3 (Eq. lexi)."""
    x = np.asarray(x)
    return ((x[..., 0] * L[1] + x[..., 1]) * L[2] + x[..., 2]) * L[3] + x[..., 3]


def coords_of(L):
    """Coordinates (V, 4) of all sites in lexicographic order."""
    return np.stack(np.meshgrid(*[np.arange(n) for n in L], indexing="ij"), axis=-1).reshape(-1, 4)


def parity(x):
    """P(x) = (1 - (-1)^{sum_mu x_mu}) / 2: 0 for even sites, 1 for odd (Eq. ipt)."""
    return np.asarray(x).sum(axis=-1) % 2


def ipt(x, L, B=None):
    """openQxD site index (Eq. ipt): floor((V_B Lambda(n, N_B) + Lambda(b, B)) / 2) + P(x) V / 2.

    B is the cache-block extent; B = L (the default) is one block.
    """
    L = np.asarray(L)
    B = L if B is None else np.asarray(B)
    x = np.asarray(x)
    n = x // B
    b = x % B
    VB = int(np.prod(B))
    V = int(np.prod(L))
    return (VB * lexi(n, L // B) + lexi(b, B)) // 2 + parity(x) * (V // 2)


def to_ipt_order(arr, L, B=None):
    """Reorder a lexicographic-order site array into openQxD (Eq. ipt) order."""
    idx = ipt(coords_of(L), L, B)
    out = np.empty_like(arr)
    out[idx] = arr
    return out


def from_ipt_order(arr, L, B=None):
    """Inverse of :func:`to_ipt_order`."""
    return arr[ipt(coords_of(L), L, B)]


def openqxd_gauge(U, A, L, B=None, cstar=False):
    """openQxD's gauge storage (Sec. 4.1.4): eight links at every odd site, none stored at even ones.

    For the odd site x with index x^ (Eq. ipt, blocks B), row x^ - V/2 holds, for mu = 0..3,
    U_mu(x) at 2 mu and U_mu(x - mu) at 2 mu + 1 (the reading of the forward/backward order; the
    paper states only that forward and backward links are stored at odd points).  x - mu is the
    lattice neighbour: periodic wrap, and with ``cstar`` (L the doubled lattice) a step across
    the y or z boundary also moves x1 by L1 / 2 (Sec. 4.2).  U: [V][4][3][3] and A: [V][4] in
    lexicographic order on L; returns (u8 [V/2][8][3][3], a8 [V/2][8]).
    """
    L = tuple(L)
    V = int(np.prod(L))
    c = coords_of(L)
    odd = parity(c) == 1
    row = ipt(c[odd], L, B) - V // 2
    u8 = np.empty((V // 2, 8, 3, 3), dtype=U.dtype)
    a8 = np.empty((V // 2, 8))
    for mu in range(4):
        back = c[odd].copy()
        crossed = back[:, mu] == 0
        back[:, mu] = (back[:, mu] - 1) % L[mu]
        if cstar and mu >= 2:
            back[crossed, 1] = (back[crossed, 1] + L[1] // 2) % L[1]
        u8[row, 2 * mu] = U[lexi(c[odd], L), mu]
        u8[row, 2 * mu + 1] = U[lexi(back, L), mu]
        a8[row, 2 * mu] = A[lexi(c[odd], L), mu]
        a8[row, 2 * mu + 1] = A[lexi(back, L), mu]
    return u8, a8


# ---------------------------------------------------------------------------------------
# Lattice geometry with boundary conditions
# ---------------------------------------------------------------------------------------
class Lattice:
    """Geometry of the lattice on which D acts.

    L = (T, L1, L2, L3) are the physical extents.  With ``cstar`` the lattice is doubled in
    x (Sec. 4.2), so the fields live on (T, 2 L1, L2, L3).  ``antiperiodic`` selects the
    time boundary condition.
    """

    def __init__(self, L, antiperiodic=True, cstar=False):
        self.phys = tuple(int(v) for v in L)
        self.cstar = bool(cstar)
        self.dims = (self.phys[0], 2 * self.phys[1], self.phys[2], self.phys[3]) if cstar else self.phys
        self.antiperiodic = bool(antiperiodic)
        self.V = int(np.prod(self.dims))
        self.coords = coords_of(self.dims)
        self.par = parity(self.coords)
        self._nbr = {}

    def neighbour(self, mu, step):
        """Index of x + step*mu_hat for every site x, and the boundary sign of that hop.

        The sign is -1 on hops that cross the time boundary when it is antiperiodic.  With
        C*, a hop across the y or z boundary lands on the mirror copy: x1 -> x1 + L1 mod 2 L1.
        """
        key = (mu, step)
        if key not in self._nbr:
            c = self.coords.copy()
            c[:, mu] += step
            wrapped = (c[:, mu] < 0) | (c[:, mu] >= self.dims[mu])
            c[:, mu] %= self.dims[mu]
            sign = np.ones(self.V)
            if mu == 0 and self.antiperiodic:
                sign[wrapped] = -1.0
            if self.cstar and mu in (2, 3):
                c[wrapped, 1] = (c[wrapped, 1] + self.phys[1]) % self.dims[1]
            self._nbr[key] = (lexi(c, self.dims), sign)
        return self._nbr[key]

    def fwd(self, mu):
        return self.neighbour(mu, +1)[0]

    def bwd(self, mu):
        return self.neighbour(mu, -1)[0]


def cstar_double_gauge(U, A, L):
    """Gauge field on the C*-doubled lattice (Sec. 4.2): mirror links U* and angles -A.

    U (V,4,3,3) and A (V,4) live on the physical lattice L; the result lives on
    (T, 2 L1, L2, L3) with U(x + L1 e1) = U(x)^* and A(x + L1 e1) = -A(x).
    """
    T, L1, L2, L3 = L
    Ur = U.reshape(T, L1, L2, L3, 4, 3, 3)
    Ar = A.reshape(T, L1, L2, L3, 4)
    U2 = np.concatenate([Ur, np.conj(Ur)], axis=1).reshape(-1, 4, 3, 3)
    A2 = np.concatenate([Ar, -Ar], axis=1).reshape(-1, 4)
    return U2, A2


def hop_links(U, A, q):
    """U(3) hop links exp(i q A_mu(x)) U_mu(x) (Sec. 4.3)."""
    return U * np.exp(1j * q * A)[..., None, None]


# ---------------------------------------------------------------------------------------
# Hopping term and the Wilson-clover operator
# ---------------------------------------------------------------------------------------
def hop(lat, W, psi):
    """(H psi)(x) = sum_mu [(1 - gamma_mu) W_mu(x) psi(x+mu) + (1 + gamma_mu) W_mu(x-mu)^dag psi(x-mu)].

    Full 4x4 gamma matrices on 12-component spinors; boundary signs per :meth:`Lattice.neighbour`.
    D = (4 + m0) - H/2 + clover, as in the operator of the method.
    """
    out = np.zeros_like(psi)
    for mu in range(4):
        f, sf = lat.neighbour(mu, +1)
        b, sb = lat.neighbour(mu, -1)
        t = np.einsum("xab,xtb->xta", W[:, mu], psi[f]) * sf[:, None, None]
        out += np.einsum("st,xta->xsa", I4 - GAMMA[mu], t)
        t = np.einsum("xab,xtb->xta", dag(W[b, mu]), psi[b]) * sb[:, None, None]
        out += np.einsum("st,xta->xsa", I4 + GAMMA[mu], t)
    return out


def _leaves(lat, M, mu, nu, sites=None):
    """Q_{mu nu}(x): sum of the four plaquette leaves at x in the (mu, nu) plane.

    M has shape (V, 4, n, n) (n = 3 for SU(3), n = 1 for U(1) phases).  Each leaf is the
    ordered product around one of the four plaquettes touching x, all with the mu -> nu
    orientation:
      U_mu(x) U_nu(x+mu) U_mu(x+nu)^+ U_nu(x)^+
      U_nu(x) U_mu(x+nu-mu)^+ U_nu(x-mu)^+ U_mu(x-mu)
      U_mu(x-mu)^+ U_nu(x-mu-nu)^+ U_mu(x-mu-nu) U_nu(x-nu)
      U_nu(x-nu)^+ U_mu(x-nu) U_nu(x-nu+mu) U_mu(x)^+
    `sites` restricts x to the given site indices (default: all sites).
    """
    x = np.arange(lat.V) if sites is None else np.asarray(sites)
    fm, fn, bm, bn = lat.fwd(mu), lat.fwd(nu), lat.bwd(mu), lat.bwd(nu)
    Um, Un = M[:, mu], M[:, nu]
    q = Um[x] @ Un[fm[x]] @ dag(Um[fn[x]]) @ dag(Un[x])
    q = q + Un[x] @ dag(Um[bm[fn[x]]]) @ dag(Un[bm[x]]) @ Um[bm[x]]
    bmn = bn[bm[x]]
    q = q + dag(Um[bm[x]]) @ dag(Un[bmn]) @ Um[bmn] @ Un[bn[x]]
    q = q + dag(Un[bn[x]]) @ Um[bn[x]] @ Un[fm[bn[x]]] @ dag(Um[x])
    return q


def _leaf_sum(lat, M, mu, nu, sites):
    return _leaves(lat, M, mu, nu) if sites is None else _leaves(lat, M, mu, nu, sites=sites)


def field_strength_su3(lat, U, mu, nu, sites=None):
    """Fhat_{mu nu} = (Q_{mu nu} - Q_{nu mu}) / 8 minus its trace / 3 (traceless), per site."""
    F = (_leaf_sum(lat, U, mu, nu, sites) - _leaf_sum(lat, U, nu, mu, sites)) / 8.0
    tr = np.trace(F, axis1=-2, axis2=-1)
    return F - tr[:, None, None] / 3.0 * np.eye(3)


def field_strength_u1(lat, A, mu, nu, sites=None):
    """Fhat^{U(1)}_{mu nu} = (Q_{mu nu} - Q_{nu mu}) / 8 from the unit-charge phases exp(i A)."""
    P = np.exp(1j * A)[..., None, None]
    return ((_leaf_sum(lat, P, mu, nu, sites) - _leaf_sum(lat, P, nu, mu, sites)) / 8.0)[:, 0, 0]


def clover_matrix(lat, U, A, q, m0, csw, csw_qed, sites=None):
    """Site-diagonal 12x12 matrix (4 + m0) + c_sw (i/4) sigma.F^SU(3) + q c_sw^QED (i/4) sigma.F^U(1).

    Sums run over all ordered pairs mu != nu.  Index 3*alpha + a.  Shape (V, 12, 12), or
    (len(sites), 12, 12) when `sites` is given.
    """
    n = lat.V if sites is None else len(sites)
    C = np.zeros((n, 12, 12), dtype=np.complex128)
    C += (4.0 + m0) * np.eye(12)
    for mu in range(4):
        for nu in range(4):
            if mu == nu:
                continue
            s = sigma(mu, nu)
            F = field_strength_su3(lat, U, mu, nu, sites)
            C += csw * 0.25j * np.einsum("st,xab->xsatb", s, F).reshape(n, 12, 12)
            f1 = field_strength_u1(lat, A, mu, nu, sites)
            C += q * csw_qed * 0.25j * np.einsum("st,x,ab->xsatb", s, f1, np.eye(3)).reshape(n, 12, 12)
    return C


def hop_at(lat, W, psi, sites):
    """(H psi)(x) for x in `sites` only; the same sum as :func:`hop`."""
    x = np.asarray(sites)
    out = np.zeros((len(x), 4, 3), dtype=np.complex128)
    for mu in range(4):
        f, sf = lat.neighbour(mu, +1)
        b, sb = lat.neighbour(mu, -1)
        t = np.einsum("xab,xtb->xta", W[x, mu], psi[f[x]]) * sf[x, None, None]
        out += np.einsum("st,xta->xsa", I4 - GAMMA[mu], t)
        t = np.einsum("xab,xtb->xta", dag(W[b[x], mu]), psi[b[x]]) * sb[x, None, None]
        out += np.einsum("st,xta->xsa", I4 + GAMMA[mu], t)
    return out


def D_at_sites(lat, U, A, q, m0, csw, csw_qed, psi, sites):
    """(D psi)(x) for x in `sites`: the clover matrix and the hop evaluated at those sites only."""
    C = clover_matrix(lat, U, A, q, m0, csw, csw_qed, sites=sites)
    Cpsi = np.einsum("xij,xj->xi", C, psi[np.asarray(sites)].reshape(-1, 12)).reshape(-1, 4, 3)
    return Cpsi - 0.5 * hop_at(lat, hop_links(U, A, q), psi, sites)


def Dhat_at_sites(lat, U, A, q, m0, csw, csw_qed, psi, sites, dagger=False):
    """(Dhat psi_e)(x) for even sites x in `sites`: D_ee psi - D_eo D_oo^-1 D_oe psi at x only.

    psi is a full-length field whose odd sites are ignored (only psi_e enters).  The Schur
    complement of the even-odd split, evaluated as its definition reads: D_oe psi_e = -1/2 H
    psi_e at the odd neighbours y of the sampled x, then D_oo^-1 = A_oo^-1 (the 12x12 clover
    matrix inverted at each y), then D_ee psi_e - D_eo t = A(x) psi(x) + 1/2 (H t)(x), where t
    lives on those odd neighbours only (H at x reads nothing else).  dagger: gamma5 Dhat gamma5.
    """
    x = np.asarray(sites)
    if np.any(lat.par[x] != 0):
        raise ValueError("Dhat_at_sites takes even sites")
    pe = np.where((lat.par == 0)[:, None, None], psi, 0)
    if dagger:
        pe = g5(pe)
    W = hop_links(U, A, q)
    ys = np.unique(np.concatenate([lat.neighbour(mu, s)[0][x] for mu in range(4) for s in (+1, -1)]))
    Doe = -0.5 * hop_at(lat, W, pe, ys)                                    # (D_oe psi_e)(y)
    Cy = clover_matrix(lat, U, A, q, m0, csw, csw_qed, sites=ys)
    t = np.zeros_like(pe)
    t[ys] = np.linalg.solve(Cy, Doe.reshape(-1, 12)[..., None])[..., 0].reshape(-1, 4, 3)
    Cx = clover_matrix(lat, U, A, q, m0, csw, csw_qed, sites=x)
    Dee = np.einsum("xij,xj->xi", Cx, pe[x].reshape(-1, 12)).reshape(-1, 4, 3)
    out = Dee - (-0.5 * hop_at(lat, W, t, x))                              # D_ee psi_e - D_eo t
    return g5(out) if dagger else out


class Operator:
    """The Wilson-clover operator D on a given lattice, gauge field and parameters."""

    def __init__(self, lat, U, A, q, m0, csw, csw_qed):
        self.lat = lat
        self.W = hop_links(U, A, q)
        self.C = clover_matrix(lat, U, A, q, m0, csw, csw_qed)
        self.even = lat.par == 0
        self.odd = ~self.even
        self._Cinv_odd = None

    # full operator -------------------------------------------------------------------
    def clover_apply(self, psi):
        return np.einsum("xij,xj->xi", self.C, psi.reshape(-1, 12)).reshape(psi.shape)

    def D(self, psi):
        """D psi = A psi - (1/2) H psi."""
        return self.clover_apply(psi) - 0.5 * hop(self.lat, self.W, psi)

    def Ddag_g5(self, psi):
        """gamma5 D gamma5 psi (equals D^dagger psi by gamma5-hermiticity)."""
        return g5(self.D(g5(psi)))

    # even-odd blocks -----------------------------------------------------------------
    def block(self, psi_in, out_mask, in_mask):
        """D_{out,in}: D applied to psi_in restricted to `in_mask` sites, result restricted to `out_mask`."""
        v = np.where(in_mask[:, None, None], psi_in, 0)
        return np.where(out_mask[:, None, None], self.D(v), 0)

    def Doo_inv(self, psi):
        """D_oo^-1 = A_oo^-1 (the hop only links opposite parities): inverse 12x12 per odd site."""
        if self._Cinv_odd is None:
            self._Cinv_odd = np.linalg.inv(self.C[self.odd])
        out = np.zeros_like(psi)
        out[self.odd] = np.einsum("xij,xj->xi", self._Cinv_odd, psi[self.odd].reshape(-1, 12)).reshape(-1, 4, 3)
        return out

    def Dhat(self, psi_e):
        """Dhat psi_e = D_ee psi_e - D_eo D_oo^-1 D_oe psi_e (full-length arrays, zero on odd sites)."""
        e, o = self.even, self.odd
        t = self.Doo_inv(self.block(psi_e, o, e))
        return self.block(psi_e, e, e) - self.block(t, e, o)

    def Dhat_dag(self, psi_e):
        """Dhat^dagger = gamma5 Dhat gamma5."""
        return g5(self.Dhat(g5(psi_e)))

    def schur_source(self, eta):
        """eta_hat_e = eta_e - D_eo D_oo^-1 eta_o."""
        e, o = self.even, self.odd
        eo = np.where(o[:, None, None], eta, 0)
        return np.where(e[:, None, None], eta, 0) - self.block(self.Doo_inv(eo), e, o)

    def reconstruct(self, psi_e, eta):
        """psi_o = D_oo^-1 (eta_o - D_oe psi_e); returns the full solution."""
        e, o = self.even, self.odd
        eo = np.where(o[:, None, None], eta, 0)
        psi_o = self.Doo_inv(eo - self.block(psi_e, o, e))
        return np.where(e[:, None, None], psi_e, 0) + psi_o


def g5(psi):
    """gamma5 psi = diag(1, 1, -1, -1) on the spin index."""
    return np.einsum("st,xta->xsa", GAMMA5, psi)


def vdot(a, b):
    """<a, b> = sum a^* b."""
    return np.vdot(a.ravel(), b.ravel())


def norm(a):
    return float(np.sqrt(np.vdot(a.ravel(), a.ravel()).real))


def true_rel_residual(op, psi, eta):
    """||eta - D psi||_2 / ||eta||_2 of the full system."""
    return norm(eta - op.D(psi)) / norm(eta)


def cgls(apply_A, apply_Adag, b, tol, maxiter, x0=None):
    """Conjugate gradient on A^+ A x = A^+ b, tracking the residual s = b - A x of A x = b.

    Stops when ||s|| <= tol.  Returns (x, iterations, ||s||).
    """
    x = np.zeros_like(b) if x0 is None else x0.copy()
    s = b - apply_A(x) if x0 is not None else b.copy()
    r = apply_Adag(s)
    p = r.copy()
    gamma = norm(r) ** 2
    it = 0
    snorm = norm(s)
    while snorm > tol and it < maxiter:
        q = apply_A(p)
        alpha = gamma / norm(q) ** 2
        x = x + alpha * p
        s = s - alpha * q
        r = apply_Adag(s)
        gamma_new = norm(r) ** 2
        p = r + (gamma_new / gamma) * p
        gamma = gamma_new
        snorm = norm(s)
        it += 1
    return x, it, snorm


def solve_eo_cg(op, eta, tol=1e-10, maxiter=100000, max_outer=10):
    """Even-odd preconditioned CG (CG on Dhat^+ Dhat) for D psi = eta, judged by the full residual.

    Each round solves the Schur system for the current full residual and adds the
    correction; stops once ||eta - D psi|| / ||eta|| <= tol.  Returns (psi, info dict).
    """
    psi = np.zeros_like(eta)
    nrm = norm(eta)
    total = 0
    res = 1.0
    for outer in range(max_outer):
        r = eta - op.D(psi)
        res = norm(r) / nrm
        if res <= tol:
            break
        bh = op.schur_source(r)
        xe, it, _ = cgls(op.Dhat, op.Dhat_dag, bh, 0.5 * tol * nrm, maxiter)
        total += it
        psi = psi + op.reconstruct(xe, r)
    return psi, {"iterations": total, "true_rel_residual": true_rel_residual(op, psi, eta), "outer": outer}


# ---------------------------------------------------------------------------------------
# Clover packing (Sec. 4.1.3)
# ---------------------------------------------------------------------------------------
_UPPER = [(i, j) for i in range(6) for j in range(i + 1, 6)]          # row-major strict upper
_LOWER_COLMAJOR = [(i, j) for j in range(6) for i in range(j + 1, 6)]  # column-major strict lower


def pack36(M):
    """Hermitian 6x6 blocks (..., 6, 6) -> 36 reals: 6 real diagonal entries, then
    (Re, Im) of the 15 strictly-upper entries in row-major order (openQxD packing)."""
    out = np.empty(M.shape[:-2] + (36,))
    for i in range(6):
        out[..., i] = M[..., i, i].real
    for k, (i, j) in enumerate(_UPPER):
        out[..., 6 + 2 * k] = M[..., i, j].real
        out[..., 7 + 2 * k] = M[..., i, j].imag
    return out


def unpack36(p):
    """Inverse of :func:`pack36` (rebuilds the lower triangle by Hermiticity)."""
    M = np.zeros(p.shape[:-1] + (6, 6), dtype=np.complex128)
    for i in range(6):
        M[..., i, i] = p[..., i]
    for k, (i, j) in enumerate(_UPPER):
        M[..., i, j] = p[..., 6 + 2 * k] + 1j * p[..., 7 + 2 * k]
        M[..., j, i] = np.conj(M[..., i, j])
    return M


def pack36_lower_colmajor(M):
    """Same 6 diagonal reals, then (Re, Im) of the strictly-lower entries in column-major
    order -- the other library's packing that the paper contrasts with openQxD's."""
    out = np.empty(M.shape[:-2] + (36,))
    for i in range(6):
        out[..., i] = M[..., i, i].real
    for k, (i, j) in enumerate(_LOWER_COLMAJOR):
        out[..., 6 + 2 * k] = M[..., i, j].real
        out[..., 7 + 2 * k] = M[..., i, j].imag
    return out


def clover_blocks(C):
    """The two chirality blocks (V, 2, 6, 6) of site matrices C (V, 12, 12): + = spins 0,1."""
    return np.stack([C[:, :6, :6], C[:, 6:, 6:]], axis=1)


def packed_clover(op):
    """Clover field as [V][2][36] reals in lexicographic site order (openQxD 36-real packing)."""
    return pack36(clover_blocks(op.C))


# ---------------------------------------------------------------------------------------
# Gauge-equivariant parallel-transport convolution (PTC) network (learned preconditioner)
# ---------------------------------------------------------------------------------------
# Paths p = 0 (stay), 1 + mu (from x + mu_hat), 5 + mu (from x - mu_hat).  The transport uses the
# hop links and the operator's boundary signs, so the network commutes with gauge
# transformations and obeys the same boundary conditions as D.
NPATH = 9


def path_swap(p):
    """The path whose transport is the adjoint of path p's: +mu <-> -mu, 0 -> 0."""
    return 0 if p == 0 else (p + 4 if p < 5 else p - 4)


def transport(lat, W, psi, p):
    """(T_p psi)(x): psi itself (p = 0), W_mu(x) psi(x + mu) (p = 1 + mu), W_mu(x - mu)^+ psi(x - mu)
    (p = 5 + mu), with the boundary sign of the hop."""
    if p == 0:
        return psi.copy()
    if p < 5:
        mu = p - 1
        f, sf = lat.neighbour(mu, +1)
        return np.einsum("xab,xsb->xsa", W[:, mu], psi[f]) * sf[:, None, None]
    mu = p - 5
    b, sb = lat.neighbour(mu, -1)
    return np.einsum("xab,xsb->xsa", dag(W[b, mu]), psi[b]) * sb[:, None, None]


def ptc_layer(lat, W, omega, h):
    """out_c(x) = sum_{c', p} omega[c, c', p] (T_p h_{c'})(x); omega (Cout, Cin, 9, 4, 4) spin
    matrices, h (Cin, V, 4, 3).  Linear, no nonlinearity."""
    cout, cin = omega.shape[:2]
    out = np.zeros((cout,) + h.shape[1:], dtype=np.complex128)
    for ci in range(cin):
        for p in range(NPATH):
            T = transport(lat, W, h[ci], p)
            out += np.einsum("ost,xta->oxsa", omega[:, ci, p], T)
    return out


def ptc_net(lat, W, weights, b):
    """M(b): the layers applied in order to the one-channel input b (V, 4, 3); returns (V, 4, 3)."""
    h = b[None]
    for om in weights:
        h = ptc_layer(lat, W, om, h)
    return h[0]


def ptc_loss(lat, W, weights, bs, vs):
    """Sum over samples of ||M(b_i) - v_i||^2 (the training loss, b_i = D v_i)."""
    return float(sum(np.vdot(ptc_net(lat, W, weights, b) - v, ptc_net(lat, W, weights, b) - v).real
                     for b, v in zip(bs, vs)))


def ptc_layer_adjoint(lat, W, omega, g):
    """Adjoint of ptc_layer applied to g (Cout, V, 4, 3): sum_{c, p} T_{swap p}(omega[c, c', p]^+ g_c)."""
    cout, cin = omega.shape[:2]
    out = np.zeros((cin,) + g.shape[1:], dtype=np.complex128)
    for c in range(cout):
        for p in range(NPATH):
            for ci in range(cin):
                mg = np.einsum("ts,xta->xsa", omega[c, ci, p].conj(), g[c])
                out[ci] += transport(lat, W, mg, path_swap(p))
    return out


def ptc_loss_grad(lat, W, weights, bs, vs):
    """Gradient of ptc_loss with respect to the conjugate weights, dL/d(omega^*), per layer
    (the real-parameter gradient is 2 Re / 2 Im of it), by the chain rule through the layers."""
    grads = [np.zeros_like(om) for om in weights]
    for b, v in zip(bs, vs):
        hs = [b[None]]
        for om in weights:
            hs.append(ptc_layer(lat, W, om, hs[-1]))
        g = (hs[-1][0] - v)[None]
        for li in range(len(weights) - 1, -1, -1):
            om, h = weights[li], hs[li]
            cout, cin = om.shape[:2]
            for ci in range(cin):
                for p in range(NPATH):
                    T = transport(lat, W, h[ci], p)
                    grads[li][:, ci, p] += np.einsum("oxsa,xta->ost", g, T.conj())
            g = ptc_layer_adjoint(lat, W, om, g)
    return grads
