"""A CPU model of the packed 16-bit arithmetic in the 16-bit hop (the FP16N/BF16N leg: spin
projection and 3x3 link product on the stored 16-bit values, every operation rounded to the
storage format, fused multiply-adds rounded once), checked against exact arithmetic on the same
stored values.  It pins the two claims the design rests on: no intermediate leaves the format's
range (stored spinor components lie in [-1, 1] after the per-site norm, link entries of unitary
matrices in [-1, 1]), and the transported half spinor of every leg carries an error of a few
units of roundoff of the format, inside the 8 u per-site bound of the GPU parity tests.

No GPU and no library code: numpy only, with float16 for FP16 and explicit rounding of float32
bit patterns for bfloat16.
"""
import numpy as np
import pytest

from paper_2502_02490_gb300 import synth


def round_bf16(x):
    """Round float64 values to bfloat16 (round to nearest, ties to even), returned as float64."""
    f = np.asarray(x, dtype=np.float32)
    b = f.view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def round_f16(x):
    return np.asarray(x, dtype=np.float64).astype(np.float16).astype(np.float64)


UNIT = {"f16": 2.0 ** -11, "bf16": 2.0 ** -8}
ROUND = {"f16": round_f16, "bf16": round_bf16}
MAXV = {"f16": 65504.0, "bf16": 3.39e38}


def cround(z, rnd):
    return rnd(z.real) + 1j * rnd(z.imag)


def leg_model(u, s_up, s_dn, rnd, i_times):
    """h = up + c dn (c = 1 or i, per spin row) and t = U h with every operation rounded:
    additions once, each product term u x folded into the running sum by one rounding per real
    component (a fused multiply-add), as the packed leg does."""
    dn = s_dn * (1j if i_times else 1.0)
    h = cround(s_up + dn, rnd)                        # (2 spins, 3 colours), one rounding per part
    t = np.zeros((2, 3), dtype=np.complex128)
    for a in range(3):
        for b in range(3):
            x = h[:, b]
            re = u[a, b].real * x.real + t[:, a].real    # fma(u.re, x.re, acc.re) ...
            re = rnd(re)
            re = rnd(-u[a, b].imag * x.imag + re)
            im = rnd(u[a, b].real * x.imag + t[:, a].imag)
            im = rnd(u[a, b].imag * x.real + im)
            t[:, a] = re + 1j * im
    return h, t


@pytest.mark.parametrize("fmt", ["f16", "bf16"])
def test_packed_16bit_leg_stays_in_range_within_a_few_units_of_roundoff(fmt):
    rnd, u_unit = ROUND[fmt], UNIT[fmt]
    L = (4, 4, 4, 4)
    U, A = synth.gauge_field(L, 1234, 0.4)
    W = U * np.exp(1j * (2 / 3) * A)[..., None, None]          # hop links e^{iqA} U, unitary
    psi = synth.gaussian_spinor(L, 4321).reshape(-1, 4, 3)
    worst, biggest = 0.0, 0.0
    for x in range(psi.shape[0]):
        nrm = np.abs(np.concatenate([psi[x].real.ravel(), psi[x].imag.ravel()])).max()
        s = cround(psi[x] / nrm, rnd)                             # stored spinor, |component| <= 1
        for mu in range(4):
            u = cround(W.reshape(-1, 4, 3, 3)[x, mu], rnd)        # stored link
            for i_times in (False, True):
                h, t = leg_model(u, s[:2], s[2:], rnd, i_times)
                h_exact = s[:2] + s[2:] * (1j if i_times else 1.0)
                t_exact = h_exact @ u.T                           # t[sp, a] = sum_b u[a, b] h[sp, b]
                assert np.all(np.isfinite(t))
                parts_h = max(np.abs(h.real).max(), np.abs(h.imag).max())
                assert parts_h <= 2.0                                 # sums of two values in [-1, 1]
                biggest = max(biggest, np.abs(t).max())
                err = np.abs(t - t_exact).max() / np.abs(t_exact).max()
                worst = max(worst, err / u_unit)
    # |(U h)_a| <= ||h|| <= sqrt(3) |h_b|max <= sqrt(3) * 2 sqrt(2): far inside either format's range
    assert biggest <= 2 * np.sqrt(6) + 1e-9 < MAXV[fmt]
    # each of the 12 roundings of a transported component errs by at most u/2 of a partial sum
    # bounded by sqrt(2) ||h||, so the error is a few u of ||h|| <= sqrt(3) max |t|: inside the
    # 8 u per site the GPU parity tests allow (measured on this field: 3.4 u FP16, 4.5 u BF16)
    assert worst <= 8.0, worst
    print(f"{fmt}: largest intermediate {biggest:.3f}, worst transported error {worst:.2f} u")
