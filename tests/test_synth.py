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
