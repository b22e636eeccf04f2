"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the CPU oracle.

This module holds only random-number generation and the field recipe; it contains
none of the Dirac operator's arithmetic and imports neither the oracle nor the CUDA
binding.  Every array is returned in lexicographic site order, i.e. C-contiguous over
the coordinates (x0, x1, x2, x3) = (t, x, y, z), with x3 fastest (the txyz convention
of the paper's Sec. 4.1.1).

Generator: SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014) used counter-style -- output i of the stream with seed s is
mix64(s + (i+1)*0x9E3779B97F4A7C15) -- so any site's numbers can be drawn on their own.
Uniforms are the top 53 bits; normals come from the Box-Muller transform.

Gauge links follow the recipe U = exp(i eps H), H = sum_a w_a lambda_a / 2 with w_a ~ N(0,1)
and lambda_a the Gell-Mann matrices, and U(1) angles A = eps * theta, theta ~ N(0,1); the
hop link is exp(i q A) U (Sec. 4.3, Eq. for the U(3) field).
"""
from __future__ import annotations

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# Seeds per workload: gauge field 1000+k, sources 2000+k (k = workload number 0..4).
GAUGE_SEED_BASE = 1000
SOURCE_SEED_BASE = 2000


def splitmix64(counter, seed):
    """Output number `counter` (0-based) of the SplitMix64 stream started at `seed`."""
    c = np.asarray(counter, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + (c + np.uint64(1)) * GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(counter, seed):
    """Uniform double in [0, 1) from the top 53 bits of the SplitMix64 output."""
    return (splitmix64(counter, seed) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def normal_pairs(pair_index, seed):
    """Box-Muller: pair j uses uniforms 2j, 2j+1 and returns two N(0,1) numbers."""
    j = np.asarray(pair_index, dtype=np.uint64)
    u1 = uniform(np.uint64(2) * j, seed)
    u2 = uniform(np.uint64(2) * j + np.uint64(1), seed)
    r = np.sqrt(-2.0 * np.log1p(-u1))  # 1 - u1 lies in (0, 1]
    return r * np.cos(2.0 * np.pi * u2), r * np.sin(2.0 * np.pi * u2)


def normals(index, seed):
    """N(0,1) number `index` of the stream: element (index mod 2) of pair index // 2."""
    idx = np.asarray(index, dtype=np.uint64)
    a, b = normal_pairs(idx >> np.uint64(1), seed)
    return np.where((idx & np.uint64(1)) == 0, a, b)


def gell_mann():
    """The eight Gell-Mann matrices, shape (8, 3, 3), complex128."""
    l = np.zeros((8, 3, 3), dtype=np.complex128)
    l[0, 0, 1] = l[0, 1, 0] = 1
    l[1, 0, 1], l[1, 1, 0] = -1j, 1j
    l[2, 0, 0], l[2, 1, 1] = 1, -1
    l[3, 0, 2] = l[3, 2, 0] = 1
    l[4, 0, 2], l[4, 2, 0] = -1j, 1j
    l[5, 1, 2] = l[5, 2, 1] = 1
    l[6, 1, 2], l[6, 2, 1] = -1j, 1j
    l[7, 0, 0] = l[7, 1, 1] = 1 / np.sqrt(3)
    l[7, 2, 2] = -2 / np.sqrt(3)
    return l


_LAMBDA = gell_mann()
# normals per link: 8 algebra coefficients + 1 U(1) angle, padded to 10 (5 Box-Muller pairs)
_PER_LINK = 10


def volume(L):
    return int(L[0]) * int(L[1]) * int(L[2]) * int(L[3])


def _expi_hermitian(H, eps):
    """exp(i eps H) for a batch of Hermitian 3x3 matrices via the eigen-decomposition."""
    w, v = np.linalg.eigh(H)
    return np.einsum("nab,nb,ncb->nac", v, np.exp(1j * eps * w), v.conj())


def _gauge_chunk(s0, s1, seed, eps):
    links = np.arange(4 * s0, 4 * s1, dtype=np.uint64)
    pair = links[:, None] * np.uint64(_PER_LINK // 2) + np.arange(_PER_LINK // 2, dtype=np.uint64)[None, :]
    a, b = normal_pairs(pair, seed)
    z = np.stack([a, b], axis=-1).reshape(len(links), _PER_LINK)
    H = np.einsum("nk,kab->nab", z[:, :8], _LAMBDA) * 0.5
    return _expi_hermitian(H, eps).reshape(s1 - s0, 4, 3, 3), eps * z[:, 8].reshape(s1 - s0, 4)


def gauge_field(L, seed, eps, chunk=1 << 18, workers=None):
    """SU(3) links and U(1) angles on the lattice L = (T, L1, L2, L3).

    Returns (U, A): U complex128 of shape (V, 4, 3, 3) with U[x, mu] = exp(i eps H_{x,mu}),
    A float64 of shape (V, 4) with A[x, mu] = eps * theta_{x,mu}.  Site x is the
    lexicographic index.  Link (x, mu) uses normals (4x+mu)*10 + k, k = 0..9, so the result does
    not depend on the chunking; lattices of 2^21 sites or more are generated by a pool of
    processes (spawn context) unless workers=1.
    """
    import os

    V = volume(L)
    U = np.empty((V, 4, 3, 3), dtype=np.complex128)
    A = np.empty((V, 4), dtype=np.float64)
    bounds = [(s0, min(V, s0 + chunk)) for s0 in range(0, V, chunk)]
    if workers is None:
        workers = min(16, os.cpu_count() or 1) if V >= (1 << 21) else 1
    if workers > 1 and len(bounds) > 1:
        import concurrent.futures as cf
        import multiprocessing as mp

        with cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
            futs = [ex.submit(_gauge_chunk, s0, s1, seed, eps) for s0, s1 in bounds]
            for (s0, s1), f in zip(bounds, futs):
                U[s0:s1], A[s0:s1] = f.result()
    else:
        for s0, s1 in bounds:
            U[s0:s1], A[s0:s1] = _gauge_chunk(s0, s1, seed, eps)
    return U, A


def gaussian_spinor(L, seed, chunk=1 << 20):
    """Gaussian spinor field psi[x, alpha, a] with Re, Im ~ N(0, 1); shape (V, 4, 3) complex128.

    Site x uses normals 24x + 2(3 alpha + a) (real part) and 24x + 2(3 alpha + a) + 1 (imaginary).
    """
    V = volume(L)
    out = np.empty((V, 4, 3), dtype=np.complex128)
    for s0 in range(0, V, chunk):
        s1 = min(V, s0 + chunk)
        pair = np.arange(12 * s0, 12 * s1, dtype=np.uint64)
        a, b = normal_pairs(pair, seed)
        out[s0:s1] = (a + 1j * b).reshape(s1 - s0, 4, 3)
    return out


def point_source(L, alpha, colour, site=0):
    """delta_{x,site} delta_{spin,alpha} delta_{colour,a}: one spin-colour point source."""
    out = np.zeros((volume(L), 4, 3), dtype=np.complex128)
    out[site, alpha, colour] = 1.0
    return out


def random_su3(n, seed, eps=1.0):
    """n random SU(3) matrices exp(i eps H) (for gauge transformations in tests)."""
    pair = np.arange(4 * n, dtype=np.uint64).reshape(n, 4)
    a, b = normal_pairs(pair, seed)
    z = np.stack([a, b], axis=-1).reshape(n, 8)
    return _expi_hermitian(np.einsum("nk,kab->nab", z, _LAMBDA) * 0.5, eps)


def random_angles(n, seed, scale=1.0):
    """n angles scale * N(0,1)."""
    return scale * normals(np.arange(n, dtype=np.uint64), seed)
