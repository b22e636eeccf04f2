"""Pins for the seeded input generators (SplitMix64 stream, Box-Muller, link recipe)."""
import os

import numpy as np

from paper_2502_02490_gb300 import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_splitmix64_reference_outputs():
    vals = [int(l) for l in open(os.path.join(GOLD, "splitmix64_seed1234567.txt")) if l[0].isdigit()]
    got = [int(v) for v in synth.splitmix64(np.arange(5), 1234567)]
    assert got == vals


def test_normals_moments():
    z = synth.normals(np.arange(400000), 7)
    assert abs(z.mean()) < 5e-3
    assert abs(z.var() - 1) < 1e-2
    u = synth.uniform(np.arange(100000), 3)
    assert u.min() >= 0 and u.max() < 1


def test_links_are_su3_and_chunk_independent():
    L = (2, 2, 2, 4)
    U, A = synth.gauge_field(L, 11, 0.4)
    Ub, Ab = synth.gauge_field(L, 11, 0.4, chunk=3)
    assert np.array_equal(U, Ub) and np.array_equal(A, Ab)
    UU = np.einsum("xmab,xmcb->xmac", U, U.conj())
    assert np.abs(UU - np.eye(3)).max() < 1e-14
    assert np.abs(np.linalg.det(U) - 1).max() < 1e-14
    # per-site counters: a larger lattice's first sites carry the same links (same Lambda)
    U2, _ = synth.gauge_field((4, 2, 2, 4), 11, 0.4)
    assert np.array_equal(U2[: synth.volume(L)], U)


def test_eps_zero_is_unit_field():
    U, A = synth.gauge_field((2, 2, 2, 2), 5, 0.0)
    assert np.abs(U - np.eye(3)).max() < 1e-14 and np.abs(A).max() == 0


def test_gaussian_spinor_follows_the_documented_recipe():
    """The Gaussian field recipe that qxd_train_precond also draws on the device (include/qxd.h):
    component (alpha, a) at lexicographic site x is r (cos th + i sin th) with r = sqrt(-2 ln(1 - u_2j)),
    th = 2 pi u_(2j+1), j = 12 x + 3 alpha + a and u_n the top 53 bits of SplitMix64 output n.
    Restated here with Python integers and the math module, independently of numpy."""
    import math

    mask = (1 << 64) - 1

    def sm64(seed, n):
        z = (seed + (n + 1) * 0x9E3779B97F4A7C15) & mask
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & mask
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & mask
        return z ^ (z >> 31)

    L, seed = (2, 4, 2, 2), 500
    psi = synth.gaussian_spinor(L, seed)
    for x in (0, 1, 17, 31):
        for alpha in range(4):
            for a in range(3):
                j = 12 * x + 3 * alpha + a
                u1 = (sm64(seed, 2 * j) >> 11) * 2.0 ** -53
                u2 = (sm64(seed, 2 * j + 1) >> 11) * 2.0 ** -53
                r = math.sqrt(-2.0 * math.log1p(-u1))
                want = complex(r * math.cos(2 * math.pi * u2), r * math.sin(2 * math.pi * u2))
                assert abs(psi[x, alpha, a] - want) <= 1e-15 * max(1.0, abs(want)), (x, alpha, a)
