"""The 36-real clover packing of Sec. 4.1.3 and its lower-triangle column-major counterpart."""
import numpy as np

from oracle import qxd_oracle as O


def rand_herm(n, seed):
    r = np.random.default_rng(seed)
    X = r.standard_normal((n, 6, 6)) + 1j * r.standard_normal((n, 6, 6))
    return X + np.conj(np.swapaxes(X, -1, -2))


def test_pack_roundtrip():
    M = rand_herm(10, 0)
    assert np.abs(O.unpack36(O.pack36(M)) - M).max() < 1e-15


def test_pack_layout_by_hand():
    M = np.zeros((6, 6), dtype=complex)
    M[np.arange(6), np.arange(6)] = np.arange(1, 7)
    M[0, 1], M[1, 0] = 10 + 11j, 10 - 11j
    M[4, 5], M[5, 4] = 20 - 21j, 20 + 21j
    M[0, 5], M[5, 0] = 30 + 31j, 30 - 31j
    p = O.pack36(M)
    assert list(p[:6]) == [1, 2, 3, 4, 5, 6]
    assert list(p[6:8]) == [10, 11]        # (0,1) comes first
    assert list(p[14:16]) == [30, 31]      # (0,5) is the fifth upper entry
    assert list(p[34:36]) == [20, -21]     # (4,5) comes last


def test_lower_column_major_is_conjugate_of_upper_row_major():
    M = rand_herm(5, 1)
    a, b = O.pack36(M), O.pack36_lower_colmajor(M)
    assert np.array_equal(a[..., :6], b[..., :6])
    assert np.array_equal(a[..., 6::2], b[..., 6::2])
    assert np.array_equal(a[..., 7::2], -b[..., 7::2])
