"""Pins for the site orderings of Sec. 4.1.1 (Eq. lexi and Eq. ipt)."""
import numpy as np
import pytest

from oracle import qxd_oracle as O


@pytest.mark.parametrize("L", [(2, 2, 2, 2), (4, 6, 2, 8), (3, 5, 7, 2)])
def test_lexi_is_c_order_ravel(L):
    c = O.coords_of(L)
    assert np.array_equal(O.lexi(c, L), np.ravel_multi_index(c.T, L))
    assert np.array_equal(O.lexi(c, L), np.arange(np.prod(L)))


@pytest.mark.parametrize("L,B", [((2, 2, 2, 2), None), ((4, 6, 2, 8), None), ((8, 4, 4, 4), (4, 2, 2, 4)),
                                 ((4, 4, 4, 8), (2, 2, 4, 4))])
def test_ipt_bijection_and_even_first(L, B):
    c = O.coords_of(L)
    V = int(np.prod(L))
    idx = O.ipt(c, L, B)
    assert np.array_equal(np.sort(idx), np.arange(V))
    even = O.parity(c) == 0
    assert idx[even].max() < V // 2 and idx[~even].min() >= V // 2


@pytest.mark.parametrize("L", [(2, 2, 2, 2), (4, 6, 2, 8)])
def test_ipt_single_block_keeps_lexicographic_order_within_parity(L):
    c = O.coords_of(L)
    idx = O.ipt(c, L)
    lam = O.lexi(c, L)
    for p in (0, 1):
        m = O.parity(c) == p
        assert np.array_equal(np.argsort(idx[m]), np.argsort(lam[m]))
        # the index within the parity is floor(Lambda / 2)
        assert np.array_equal(idx[m] - p * len(c) // 2, lam[m] // 2)


def test_ipt_blocks_are_contiguous():
    L, B = (8, 4, 4, 4), (4, 2, 2, 4)
    c = O.coords_of(L)
    V, VB = 512, 64
    idx = O.ipt(c, L, B)
    nb = np.array(L) // np.array(B)
    blk = O.lexi(c // np.array(B), nb)
    for p in (0, 1):
        for n in range(int(np.prod(nb))):
            m = (blk == n) & (O.parity(c) == p)
            got = np.sort(idx[m])
            start = p * V // 2 + n * VB // 2
            assert np.array_equal(got, np.arange(start, start + VB // 2))


def test_small_example_by_hand():
    # 2^4 lattice: Lambda(0,0,0,1) = 1 is odd -> V/2 + floor(1/2) = 8; (0,0,1,1) -> Lambda 3, even -> 1;
    # (1,1,1,1) -> Lambda 15, even -> 7; (1,0,0,0) -> Lambda 8, odd -> 8 + 4 = 12.
    L = (2, 2, 2, 2)
    pts = np.array([[0, 0, 0, 1], [0, 0, 1, 1], [1, 1, 1, 1], [1, 0, 0, 0]])
    assert list(O.ipt(pts, L)) == [8, 1, 7, 12]


def test_reorder_roundtrip():
    L = (4, 2, 6, 4)
    a = np.random.default_rng(0).standard_normal((int(np.prod(L)), 3))
    assert np.array_equal(O.from_ipt_order(O.to_ipt_order(a, L), L), a)
