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
                                 ((4, 4, 4, 8), (2, 2, 4, 4)), ((6, 6, 2, 4), (3, 3, 1, 2)),
                                 ((6, 2, 6, 6), (3, 1, 3, 3)), ((2, 4, 2, 2), (1, 1, 1, 1))])
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


def _pair_parity_argument(L, B):
    """Eq. ipt halves the blocked lexicographic index; it is a bijection onto each parity half iff
    every pair (2k, 2k + 1) of blocked indices holds one even and one odd site."""
    c = O.coords_of(L)
    L, B = np.asarray(L), np.asarray(B)
    blam = int(np.prod(B)) * O.lexi(c // B, L // B) + O.lexi(c % B, B)
    par = np.empty(int(np.prod(L)), dtype=int)
    par[blam] = O.parity(c)
    return np.all(par[0::2] != par[1::2])


@pytest.mark.parametrize("L,B", [((6, 6, 2, 4), (3, 3, 1, 2)), ((6, 2, 6, 6), (3, 1, 3, 3)), ((4, 4, 4, 8), (2, 2, 4, 4)),
                                 ((2, 6, 6, 6), (1, 3, 3, 3))])
def test_any_dividing_block_pairs_opposite_parities(L, B):
    assert _pair_parity_argument(L, B)


def test_openqxd_gauge_holds_every_link_once():
    """Every link (x, mu) has exactly one odd end: the eight-link table is a permutation of them."""
    L, B = (4, 2, 6, 4), (2, 2, 3, 2)
    V = int(np.prod(L))
    U = np.arange(V * 4 * 9, dtype=float).reshape(V, 4, 3, 3) + 0j  # entries tag (site, mu)
    A = np.arange(V * 4, dtype=float).reshape(V, 4)
    u8, a8 = O.openqxd_gauge(U, A, L, B)
    assert u8.shape == (V // 2, 8, 3, 3) and a8.shape == (V // 2, 8)
    assert np.array_equal(np.sort(a8.ravel()), np.arange(V * 4, dtype=float))
    assert np.array_equal(u8[..., 0, 0].real, a8 * 9)  # the link travels with its own angle


def test_openqxd_gauge_small_example_by_hand():
    """L = (2, 2, 2, 2), B = L: the odd site x = (0, 0, 0, 1) has Lambda = 1, index floor(1/2) + 8 = 8,
    so it is row 0; its backward t link is U_0((1, 0, 0, 1)) (periodic wrap), Lambda 9."""
    L = (2, 2, 2, 2)
    V = 16
    A = np.arange(V * 4, dtype=float).reshape(V, 4)
    U = np.zeros((V, 4, 3, 3), complex)
    _, a8 = O.openqxd_gauge(U, A, L)
    assert a8[0, 0] == A[1, 0] and a8[0, 1] == A[9, 0]  # U_0(x), U_0(x - 0)
    assert a8[0, 6] == A[1, 3] and a8[0, 7] == A[0, 3]  # U_3(x), U_3(x - 3) = U_3((0,0,0,0))


@pytest.mark.parametrize("L", [(4, 4, 2, 4), (4, 8, 4, 2)])
def test_openqxd_gauge_cstar_holds_every_link_once(L):
    """On a C* (x-doubled) lattice the backward neighbour across the y or z boundary is the shifted
    one (Sec. 4.2); every link of the doubled lattice still appears exactly once."""
    V = int(np.prod(L))
    A = np.arange(V * 4, dtype=float).reshape(V, 4)
    _, a8 = O.openqxd_gauge(np.zeros((V, 4, 3, 3), complex), A, L, (2, 2, 2, 2), cstar=True)
    assert np.array_equal(np.sort(a8.ravel()), np.arange(V * 4, dtype=float))
    lat = O.Lattice((L[0], L[1] // 2, L[2], L[3]), cstar=True)
    c = O.coords_of(L)
    odd = O.parity(c) == 1
    row = O.ipt(c[odd], L, (2, 2, 2, 2)) - V // 2
    for mu in range(4):
        back, _ = lat.neighbour(mu, -1)  # the oracle's own neighbour map
        assert np.array_equal(a8[row, 2 * mu + 1], A[back[np.flatnonzero(odd)], mu])
