"""Pins for the oracle's parallel-transport convolution network and its gradient."""
import numpy as np
import pytest

from oracle import qxd_oracle as O
from paper_2502_02490_gb300 import synth
from tests import fields


def setup(L=(4, 2, 2, 4), cstar=False, seed=1003):
    lat = O.Lattice(L, antiperiodic=True, cstar=cstar)
    U, A = synth.gauge_field(lat.dims, seed, 0.4)
    return lat, U, A, O.hop_links(U, A, -1 / 3)


def rand_weights(chans, seed, scale=0.2):
    r = np.random.default_rng(seed)
    return [scale * (r.standard_normal((co, ci, 9, 4, 4)) + 1j * r.standard_normal((co, ci, 9, 4, 4)))
            for ci, co in zip(chans[:-1], chans[1:])]


def test_single_layer_reproduces_the_wilson_operator():
    """One 1->1 layer with omega_0 = (4+m0), omega_{+mu} = -(1-g_mu)/2, omega_{-mu} = -(1+g_mu)/2 is D
    without the clover term: pins paths, link placement and boundary signs against D."""
    lat, U, A, W = setup((4, 4, 2, 4))
    m0 = -0.1
    om = np.zeros((1, 1, 9, 4, 4), dtype=complex)
    om[0, 0, 0] = (4 + m0) * np.eye(4)
    for mu in range(4):
        om[0, 0, 1 + mu] = -0.5 * (np.eye(4) - O.GAMMA[mu])
        om[0, 0, 5 + mu] = -0.5 * (np.eye(4) + O.GAMMA[mu])
    op = O.Operator(lat, U, A, q=-1 / 3, m0=m0, csw=0.0, csw_qed=0.0)
    psi = synth.gaussian_spinor(lat.dims, 1)
    assert np.abs(O.ptc_net(lat, W, [om], psi) - op.D(psi)).max() < 1e-13


def test_identity_net_is_scaled_identity():
    lat, U, A, W = setup()
    om = np.zeros((1, 1, 9, 4, 4), dtype=complex)
    om[0, 0, 0] = 0.7 * np.eye(4)
    psi = synth.gaussian_spinor(lat.dims, 2)
    assert np.abs(O.ptc_net(lat, W, [om], psi) - 0.7 * psi).max() < 1e-15


@pytest.mark.parametrize("cstar", [False, True])
def test_transport_adjointness(cstar):
    lat, U, A, W = setup((2, 2, 4, 2), cstar=cstar)
    a, b = synth.gaussian_spinor(lat.dims, 3), synth.gaussian_spinor(lat.dims, 4)
    for p in range(9):
        lhs = O.vdot(a, O.transport(lat, W, b, p))
        rhs = O.vdot(O.transport(lat, W, a, O.path_swap(p)), b)
        assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_network_gauge_equivariance():
    lat, U, A, W = setup((4, 2, 4, 2))
    ws = rand_weights([1, 3, 2, 1], 5)
    V = lat.V
    Om = synth.random_su3(V, 81)
    al = synth.random_angles(V, 82)
    U2, A2 = fields.gauge_transform(lat.dims, [lat.fwd(m) for m in range(4)], U, A, Om, al)
    W2 = O.hop_links(U2, A2, -1 / 3)
    psi = synth.gaussian_spinor(lat.dims, 6)

    def g(v):
        return np.exp(1j * (-1 / 3) * al)[:, None, None] * np.einsum("xab,xsb->xsa", Om, v)

    lhs = O.ptc_net(lat, W2, ws, g(psi))
    rhs = g(O.ptc_net(lat, W, ws, psi))
    assert np.abs(lhs - rhs).max() < 1e-12 * np.abs(rhs).max()


def test_gradient_matches_central_differences():
    lat, U, A, W = setup((2, 2, 2, 4))
    ws = rand_weights([1, 2, 1], 7)
    vs = [synth.gaussian_spinor(lat.dims, 10 + k) for k in range(2)]
    bs = [synth.gaussian_spinor(lat.dims, 20 + k) for k in range(2)]
    grads = O.ptc_loss_grad(lat, W, ws, bs, vs)
    r = np.random.default_rng(0)
    h = 1e-6
    for li in range(2):
        for _ in range(6):
            idx = tuple(r.integers(0, n) for n in ws[li].shape)
            for part, unit in ((0, 1.0), (1, 1j)):
                wp = [w.copy() for w in ws]
                wm = [w.copy() for w in ws]
                wp[li][idx] += h * unit
                wm[li][idx] -= h * unit
                fd = (O.ptc_loss(lat, W, wp, bs, vs) - O.ptc_loss(lat, W, wm, bs, vs)) / (2 * h)
                an = 2 * (grads[li][idx].real if part == 0 else grads[li][idx].imag)
                assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (li, idx, part, fd, an)


def test_pins_catch_planted_ptc_mistakes(monkeypatch):
    """A wrong adjoint path map, or a missing conjugate in the weight gradient, fails a pin."""
    lat, U, A, W = setup((2, 2, 2, 4))
    ws = rand_weights([1, 2, 1], 7)
    vs = [synth.gaussian_spinor(lat.dims, 10)]
    bs = [synth.gaussian_spinor(lat.dims, 20)]

    def grad_ok():
        g = O.ptc_loss_grad(lat, W, ws, bs, vs)
        idx = (0, 0, 3, 1, 2)
        wp, wm = [w.copy() for w in ws], [w.copy() for w in ws]
        wp[0][idx] += 1e-6
        wm[0][idx] -= 1e-6
        fd = (O.ptc_loss(lat, W, wp, bs, vs) - O.ptc_loss(lat, W, wm, bs, vs)) / 2e-6
        return abs(fd - 2 * g[0][idx].real) <= 1e-6 * max(1.0, abs(fd))

    assert grad_ok()
    monkeypatch.setattr(O, "path_swap", lambda p: p)
    assert not grad_ok()
