"""A CPU model of the packed BF16 gauge transport in the tensor-core PTC layers (layers with BF16
activations): the stored activation words (one complex number per 32-bit word, real part low)
times the BF16 link, t = u h for a forward path and t = u^+ h for a backward one, as a chain of
packed fused multiply-adds per output word: (Re u, Re u) x, then (-Im u, Im u) swap(x) (or
(Im u, -Im u) swap(x) for the conjugate), accumulated over the three colours.  Every operation
rounds once to BF16.  The model is checked against exact arithmetic on the same stored values:
it pins that the chain computes the complex product (a sign or operand slip fails the exactness
check on values that BF16 holds exactly) and that its rounding error stays within a few units of
BF16 roundoff of the transported spinor.

No GPU and no library code: numpy only, with an explicit round-to-nearest-even to 8 significant
bits, checked against the bfloat16 rounding of float32 bit patterns.
"""
import numpy as np
import pytest

from paper_2502_02490_gb300 import synth

U_BF16 = 2.0 ** -8  # unit roundoff of bfloat16 (8 significant bits)


def round_bf16(x):
    """Round float64 values to 8 significant bits, ties to even (bfloat16 for finite values in its
    range).  The model's fused multiply-adds are exact in float64 (a product of two 8-bit
    significands plus an 8-bit value), so this is one rounding per operation, as on the GPU."""
    x = np.asarray(x, dtype=np.float64)
    m, e = np.frexp(x)                      # x = m 2^e, 0.5 <= |m| < 1 (m = 0 for x = 0)
    return np.ldexp(np.round(m * 256.0) / 256.0, e)


def round_bf16_bits(x):
    """bfloat16 rounding of float32 values by their bit patterns (an independent route)."""
    f = np.asarray(x, dtype=np.float32)
    b = f.view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def cround(z):
    return round_bf16(z.real) + 1j * round_bf16(z.imag)


def transport_model(u, h, adjoint):
    """t[..., be, a] = sum_b U[a, b] h[..., be, b], U = u (forward) or u^+ (backward), evaluated
    as the packed chain with one BF16 rounding per fused multiply-add and component."""
    t_re = np.zeros(h.shape, dtype=np.float64)
    t_im = np.zeros(h.shape, dtype=np.float64)
    for a in range(3):
        for b in range(3):
            w = u[..., b, a] if adjoint else u[..., a, b]      # the stored link entry
            ur = w.real[..., None]
            ui = w.imag[..., None]
            xr, xi = h[..., b].real, h[..., b].imag
            if adjoint:                                      # conj(w) x = ur x + (ui, -ui) swap(x)
                lo, hi = ui * xi, -ui * xr
            else:                                            # w x = ur x + (-ui, ui) swap(x)
                lo, hi = -ui * xi, ui * xr
            if b == 0:
                re, im = round_bf16(ur * xr), round_bf16(ur * xi)
            else:
                re, im = round_bf16(ur * xr + t_re[..., a]), round_bf16(ur * xi + t_im[..., a])
            t_re[..., a] = round_bf16(lo + re)
            t_im[..., a] = round_bf16(hi + im)
    return t_re + 1j * t_im


def test_bf16_rounding_agrees_with_the_bit_pattern_rounding():
    r = np.random.default_rng(5)
    x = (r.standard_normal(50000) * np.exp(r.uniform(-20, 20, 50000))).astype(np.float32)
    # exact ties: 9 significant bits with the last one set, at several scales
    ties = (np.arange(257, 512, 2)[None, :] * 2.0 ** np.arange(-30, 31, 6)[:, None]).ravel()
    for v in (x.astype(np.float64), ties, -ties):
        assert np.array_equal(round_bf16(v), round_bf16_bits(v))


@pytest.mark.parametrize("adjoint", [False, True])
def test_packed_bf16_chain_is_the_complex_product_when_nothing_rounds(adjoint):
    """Small integers times powers of two: every intermediate is exact in BF16, so the chain must
    equal u h (forward) or u^+ h (backward) exactly."""
    r = np.random.default_rng(11 + adjoint)
    u = (r.integers(-7, 8, (64, 3, 3)) + 1j * r.integers(-7, 8, (64, 3, 3))) / 8.0
    h = (r.integers(-7, 8, (64, 4, 3)) + 1j * r.integers(-7, 8, (64, 4, 3))) / 4.0
    t = transport_model(u, h, adjoint)
    U = np.conj(np.swapaxes(u, -1, -2)) if adjoint else u
    assert np.array_equal(t, np.einsum("nab,nsb->nsa", U, h))


@pytest.mark.parametrize("adjoint", [False, True])
def test_packed_bf16_transport_within_a_few_units_of_roundoff(adjoint):
    L = (4, 4, 4, 4)
    U, A = synth.gauge_field(L, 1003, 0.3)
    W = cround(U * np.exp(1j * (-1 / 3) * A)[..., None, None])      # BF16 hop links e^{iqA} U
    h = cround(synth.gaussian_spinor(L, 77))                        # BF16 activations (V, 4, 3)
    worst = 0.0
    for mu in range(4):
        u = W[:, mu]
        t = transport_model(u, h, adjoint)
        Umat = np.conj(np.swapaxes(u, -1, -2)) if adjoint else u
        exact = np.einsum("nab,nsb->nsa", Umat, h)
        # error per site relative to the site's largest transported component
        err = np.abs(t - exact).reshape(len(h), -1).max(axis=1)
        ref = np.abs(exact).reshape(len(h), -1).max(axis=1)
        worst = max(worst, float((err / ref).max() / U_BF16))
    # six roundings per component (one per fused multiply-add), each at most u/2 of a partial
    # sum bounded by sqrt(2) max_b |h_b| sum_b |u_ab| <= sqrt(6) ||h||: a few u of the largest
    # transported component
    assert worst <= 6.0, worst
    print(f"adjoint={adjoint}: worst transported error {worst:.2f} u of BF16")
