"""The learned preconditioner on the GPU: network forward and gradient against the oracle,
checkpointing, training, and flexible GCR with and without the network."""
import numpy as np
import pytest

from oracle import qxd_oracle as O
from paper_2502_02490_gb300 import synth
from tests.gpu_util import Case, as_c128

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def qxd():
    import __graft_entry__

    __graft_entry__.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2502_02490_gb300 import qxd as q

    return q


def layer_weights(flat, chans):
    out, off = [], 0
    for ci, co in zip(chans[:-1], chans[1:]):
        n = co * ci * 9 * 16
        out.append(flat[off:off + n].reshape(co, ci, 9, 4, 4))
        off += n
    return out


def random_flat(n, seed, scale=0.2):
    r = np.random.default_rng(seed)
    return scale * (r.standard_normal(n) + 1j * r.standard_normal(n))


# BF16 tensor-core layers: operands rounded to 8 significant bits (unit roundoff u = 2^-8), FP32
# accumulation; each layer's products carry at most 2u relative error, so the network output is
# within 4 u per layer in norm with a factor 2 to spare for cancellation.
TC_TOL_PER_LAYER = 4 * 2.0 ** -8


@pytest.mark.parametrize("prec", ["f32", "bf16_tc"])
@pytest.mark.parametrize("L,cstar,chans", [((4, 2, 2, 4), False, [1, 3, 2, 1]), ((2, 2, 4, 2), True, [1, 4, 1]),
                                           ((6, 4, 4, 6), False, [1, 16, 16, 1]),
                                           ((8, 6, 6, 4), False, [1, 8, 5, 1]),
                                           ((4, 2, 2, 4), True, [1, 8, 8, 1])])
def test_net_forward_matches_oracle(qxd, L, cstar, chans, prec):
    c = Case(qxd, torch, L, cstar=cstar)
    net = qxd.net_create(c.lat, chans, seed=1)
    try:
        qxd.net_set_precision(net, qxd.NET_F32 if prec == "f32" else qxd.NET_BF16_TC)
        w = random_flat(qxd.net_num_weights(net), 3)
        qxd.net_set_weights(net, w)
        w32 = w.real.astype(np.float32) + 1j * w.imag.astype(np.float32)  # the GPU holds FP32 weights
        psi = synth.gaussian_spinor(c.dims, 11)
        x = c.dev_tensor(psi)
        y = torch.empty_like(x)
        qxd.net_apply(net, y, x)
        ref = O.ptc_net(c.lat_o, O.hop_links(c.U, c.A, c.q), layer_weights(w32, chans), psi)
        got = as_c128(y, psi.shape)
        err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        tol = 2e-6 if prec == "f32" else TC_TOL_PER_LAYER * (len(chans) - 1)
        print(f"net {chans} {prec}: rel err {err:.3e} (tol {tol:.1e})")
        assert err < tol
    finally:
        qxd.net_destroy(net)
        c.close()


def test_net_gradient_matches_oracle(qxd):
    L, chans = (2, 2, 2, 4), [1, 2, 2, 1]
    c = Case(qxd, torch, L)
    net = qxd.net_create(c.lat, chans, seed=2)
    try:
        w = random_flat(qxd.net_num_weights(net), 5)
        qxd.net_set_weights(net, w)
        w32 = w.real.astype(np.float32) + 1j * w.imag.astype(np.float32)
        vs = np.stack([synth.gaussian_spinor(c.dims, 40 + k) for k in range(2)])
        bs = np.stack([synth.gaussian_spinor(c.dims, 50 + k) for k in range(2)])
        loss, g = qxd.net_loss_grad(net, vs, bs, 2)
        W = O.hop_links(c.U, c.A, c.q)
        ws = layer_weights(w32, chans)
        ref_loss = O.ptc_loss(c.lat_o, W, ws, list(bs), list(vs))
        ref_g = np.concatenate([gl.ravel() for gl in O.ptc_loss_grad(c.lat_o, W, ws, list(bs), list(vs))])
        assert abs(loss - ref_loss) < 1e-5 * ref_loss
        assert np.linalg.norm(g - ref_g) / np.linalg.norm(ref_g) < 1e-5
    finally:
        qxd.net_destroy(net)
        c.close()


def test_net_checkpoint_roundtrip(qxd, tmp_path):
    c = Case(qxd, torch, (2, 2, 2, 2))
    net = qxd.net_create(c.lat, [1, 3, 1], seed=9)
    try:
        path = tmp_path / "net.qxdnet"
        qxd.net_save(net, path)
        net2 = qxd.net_load(c.lat, path)
        assert np.array_equal(qxd.net_get_weights(net), qxd.net_get_weights(net2))
        qxd.net_destroy(net2)
    finally:
        qxd.net_destroy(net)
        c.close()


def test_training_lowers_the_loss_and_fgcr_solves(qxd):
    c = Case(qxd, torch, (4, 4, 4, 4), m0=-0.3)
    net = qxd.net_create(c.lat, [1, 4, 4, 1], seed=3)
    try:
        vs = np.stack([synth.gaussian_spinor(c.dims, 100 + k) for k in range(8)])
        hist = qxd.net_train(net, vs, 8, epochs=30, batch=4, lr=3e-3)
        assert hist[-1] < 0.7 * hist[0], hist
        eta = synth.gaussian_spinor(c.dims, 2000)
        b = c.dev_tensor(eta)
        res = {}
        for name, n in (("net", net), ("none", None)):
            x = torch.empty_like(b)
            st, info = qxd.solve(c.lat, x, b, solver=qxd.SOLVER_MP_FGCR_NET, inner_prec=qxd.F32, tol=1e-10,
                                 gcr_restart=16, net=n)
            assert st == qxd.OK
            assert O.true_rel_residual(c.op, as_c128(x, eta.shape), eta) <= 1e-10
            res[name] = info["iters_inner"]
        print("loss", hist[0], "->", hist[-1], "FGCR iterations with / without net:", res)
        assert res["net"] < res["none"], res  # what the trained network gains
    finally:
        qxd.net_destroy(net)
        c.close()


def test_learned_solve_falls_back_to_plain_solver(qxd):
    c = Case(qxd, torch, (4, 4, 4, 4), m0=-0.3)
    net = qxd.net_create(c.lat, [1, 4, 1], seed=5)  # untrained
    try:
        eta = synth.gaussian_spinor(c.dims, 2100)
        b = c.dev_tensor(eta)
        x = torch.empty_like(b)
        kw = dict(solver=qxd.SOLVER_MP_FGCR_NET, inner_prec=qxd.F32, tol=1e-10, gcr_restart=8, net=net, maxiter=3,
                  max_outer=1)
        st, info = qxd.solve(c.lat, x, b, check=False, **kw)
        assert st == qxd.ENOCONV and info["fallback_used"] == 0
        for fb in (qxd.SOLVER_CG_EO, qxd.SOLVER_MP_BICGSTAB_EO):
            st, info = qxd.solve(c.lat, x, b, check=False, fallback=fb, **kw)
            assert st == qxd.OK and info["fallback_used"] == 1 and info["status"] == qxd.OK, info
            assert O.true_rel_residual(c.op, as_c128(x, eta.shape), eta) <= 1e-10
    finally:
        qxd.net_destroy(net)
        c.close()


@pytest.mark.parametrize("L,cstar", [((4, 4, 4, 4), False), ((4, 2, 2, 4), True)])
def test_train_precond_matches_host_samples(qxd, L, cstar):
    """qxd_train_precond draws its samples on the device with the same counter-based recipe as the
    host generator: training on them gives the loss history and weights of qxd_net_train on the
    host-drawn fields of the same seeds."""
    c = Case(qxd, torch, L, cstar=cstar)
    nets = []
    try:
        kw = dict(epochs=3, batch=2, lr=2e-3)
        net_a, hist_a = qxd.train_precond(c.lat, [1, 4, 1], nsamp=4, sample_seed=500, net_seed=7, **kw)
        nets.append(net_a)
        net_b = qxd.net_create(c.lat, [1, 4, 1], seed=7)
        nets.append(net_b)
        vs = c.dev_tensor(np.stack([synth.gaussian_spinor(c.dims, 500 + i) for i in range(4)]))
        hist_b = qxd.net_train(net_b, vs, 4, **kw)
        print("loss per epoch (device / host samples):", hist_a, hist_b)
        assert np.all(hist_a > 0)
        np.testing.assert_allclose(hist_a, hist_b, rtol=1e-6)
        wa, wb = qxd.net_get_weights(net_a), qxd.net_get_weights(net_b)
        assert np.linalg.norm(wa - wb) <= 1e-5 * np.linalg.norm(wb)
    finally:
        for n in nets:
            qxd.net_destroy(n)
        c.close()


@pytest.mark.parametrize("prec", ["f32", "bf16_tc"])
@pytest.mark.parametrize("L,cstar,chans", [((4, 2, 2, 4), False, [1, 3, 2, 1]), ((2, 2, 4, 2), True, [1, 4, 1]),
                                           ((6, 4, 4, 6), False, [1, 16, 16, 1]),
                                           ((8, 6, 6, 4), False, [1, 8, 5, 1])])
def test_net_adjoint_matches_oracle(qxd, L, cstar, chans, prec):
    """qxd_net_apply_adjoint against the oracle's adjoint layers run last to first, and
    <phi, M psi> = <M^+ phi, psi> for the GPU's own forward and adjoint networks."""
    c = Case(qxd, torch, L, cstar=cstar)
    net = qxd.net_create(c.lat, chans, seed=1)
    try:
        qxd.net_set_precision(net, qxd.NET_F32 if prec == "f32" else qxd.NET_BF16_TC)
        w = random_flat(qxd.net_num_weights(net), 13)
        qxd.net_set_weights(net, w)
        w32 = w.real.astype(np.float32) + 1j * w.imag.astype(np.float32)
        W = O.hop_links(c.U, c.A, c.q)
        phi = synth.gaussian_spinor(c.dims, 21)
        psi = synth.gaussian_spinor(c.dims, 22)
        x = c.dev_tensor(phi)
        y = torch.empty_like(x)
        qxd.net_apply_adjoint(net, y, x)
        got = as_c128(y, phi.shape)
        g = phi[None]
        for om in reversed(layer_weights(w32, chans)):
            g = O.ptc_layer_adjoint(c.lat_o, W, om, g)
        ref = g[0]
        err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        tol = 2e-6 if prec == "f32" else TC_TOL_PER_LAYER * (len(chans) - 1)
        assert err < tol, err
        # the adjoint identity with the GPU's forward network
        xp = c.dev_tensor(psi)
        yp = torch.empty_like(xp)
        qxd.net_apply(net, yp, xp)
        lhs = np.vdot(phi, as_c128(yp, psi.shape))
        rhs = np.vdot(got, psi)
        assert abs(lhs - rhs) <= 2 * tol * np.linalg.norm(phi) * np.linalg.norm(as_c128(yp, psi.shape)) + 1e-12
        print(f"adjoint {chans} {prec}: rel err {err:.2e}, <phi, M psi> - <M+ phi, psi> = {abs(lhs - rhs):.2e}")
    finally:
        qxd.net_destroy(net)
        c.close()


@pytest.mark.parametrize("use_net", [False, True])
@pytest.mark.parametrize("L,cstar,m0", [((4, 4, 4, 4), False, -0.1), ((4, 2, 2, 4), True, -0.1),
                                        ((6, 4, 4, 8), False, -2.6)])
def test_cgnr_solve(qxd, use_net, L, cstar, m0):
    """QXD_SOLVER_MP_CGNR (CG on the normal equations of D M on the full lattice, FP32 inner,
    FP64 defect correction), with and without the network as M, judged by the oracle's true
    residual; m0 = -2.6 puts the spectrum of D around the origin (indefinite)."""
    c = Case(qxd, torch, L, cstar=cstar, m0=m0)
    net = qxd.net_create(c.lat, [1, 4, 1], seed=5) if use_net else None
    try:
        eta = synth.gaussian_spinor(c.dims, 2300)
        b = c.dev_tensor(eta)
        x = torch.empty_like(b)
        st, info = qxd.solve(c.lat, x, b, solver=qxd.SOLVER_MP_CGNR, net=net, tol=1e-10, maxiter=20000)
        assert st == qxd.OK, info
        res = O.true_rel_residual(c.op, as_c128(x, eta.shape), eta)
        assert res <= 1e-10, (res, info)
        assert abs(info["true_rel_res"] - res) <= 1e-12 + 1e-3 * res
        print(f"CGNR {L} cstar={cstar} m0={m0} net={use_net}: {info}")
    finally:
        if net:
            qxd.net_destroy(net)
        c.close()


def test_learned_preconditioner_at_a_scaled_down_near_critical_point(qxd):
    """8^4 with the workload's field recipe at m0 = -2.63, where D is indefinite (the odd clover
    blocks nearly singular, eo-CG slow): flexible GCR without a network stagnates, with a small
    trained network it reaches the inner target; at the physical branch's slowest point the
    network cuts the iterations of CG on the normal equations.  Judged by the oracle's residual."""
    L = (8, 8, 8, 8)
    c = Case(qxd, torch, L, eps=0.3, seed=1003, m0=-2.63)
    try:
        eta = synth.gaussian_spinor(c.dims, 2003)
        b = c.dev_tensor(eta)
        x = torch.empty_like(b)
        vs = c.dev_tensor(np.stack([synth.gaussian_spinor(c.dims, 5000 + k) for k in range(32)]))
        net = qxd.net_create(c.lat, [1, 4, 4, 1], seed=7)
        try:
            qxd.net_train(net, vs, 32, epochs=20, batch=8, lr=2e-3)
            kw = dict(solver=qxd.SOLVER_MP_FGCR_NET, tol=1e-10, gcr_restart=32, maxiter=400, max_outer=1, check=False)
            st0, plain = qxd.solve(c.lat, x, b, net=None, **kw)
            st1, learned = qxd.solve(c.lat, x, b, net=net, **kw)
            res = O.true_rel_residual(c.op, as_c128(x, eta.shape), eta)  # x of the learned solve
            print(f"m0=-2.63 FGCR: plain {plain['true_rel_res']:.2e} after {plain['iters_inner']}, learned "
                  f"{learned['true_rel_res']:.2e} after {learned['iters_inner']}")
            assert plain["true_rel_res"] > 0.1 and plain["iters_inner"] == 400, plain
            assert learned["iters_inner"] < 400 and res < 2e-5, (learned, res)
            # the full solve to 1e-10 with the network as right preconditioner
            st, full = qxd.solve(c.lat, x, b, solver=qxd.SOLVER_MP_FGCR_NET, tol=1e-10, gcr_restart=32, net=net,
                                 maxiter=3000)
            assert st == qxd.OK and O.true_rel_residual(c.op, as_c128(x, eta.shape), eta) <= 1e-10, full
        finally:
            qxd.net_destroy(net)
        # physical branch: the network reduces the iterations of the normal-equation solve
        qxd.build_clover(c.lat, -0.12, c.csw, c.csw_qed)
        op = O.Operator(c.lat_o, c.U, c.A, c.q, -0.12, c.csw, c.csw_qed)
        net = qxd.net_create(c.lat, [1, 4, 4, 1], seed=7)
        try:
            qxd.net_train(net, vs, 32, epochs=20, batch=8, lr=2e-3)
            st0, plain = qxd.solve(c.lat, x, b, solver=qxd.SOLVER_MP_CGNR, tol=1e-10, net=None, maxiter=5000)
            st1, learned = qxd.solve(c.lat, x, b, solver=qxd.SOLVER_MP_CGNR, tol=1e-10, net=net, maxiter=5000)
            assert st1 == qxd.OK and O.true_rel_residual(op, as_c128(x, eta.shape), eta) <= 1e-10
            print(f"m0=-0.12 CGNR: {plain['iters_inner']} iterations without the network, {learned['iters_inner']} with")
            assert learned["iters_inner"] * 2 < plain["iters_inner"], (plain, learned)
        finally:
            qxd.net_destroy(net)
    finally:
        c.close()
