"""GPU operator parity against the CPU oracle, through the C ABI (clover, D, Dhat, precisions)."""
import numpy as np
import pytest

from oracle import qxd_oracle as O
from paper_2502_02490_gb300 import synth
from tests.gpu_util import Case, rel_max_err

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

# lattices spanning several 128-site tiles with ragged tails, extent-2 directions, both BCs
SHAPES = [((2, 2, 2, 2), True), ((4, 4, 4, 4), True), ((6, 6, 6, 6), True), ((8, 8, 8, 8), False),
          ((2, 4, 6, 8), True), ((4, 2, 2, 6), False), ((10, 6, 4, 6), True)]


@pytest.fixture(scope="module")
def qxd():
    import __graft_entry__

    __graft_entry__.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2502_02490_gb300 import qxd as q

    return q


@pytest.mark.parametrize("L,anti", SHAPES)
def test_apply_D_f64(qxd, L, anti):
    c = Case(qxd, torch, L, anti=anti)
    try:
        psi = synth.gaussian_spinor(c.dims, 2000)
        err = rel_max_err(c.apply_D(psi), c.op.D(psi))
        assert err < 1e-13, err
    finally:
        c.close()


@pytest.mark.parametrize("order", [0, 1])
@pytest.mark.parametrize("L,cstar", [((4, 4, 4, 4), False), ((4, 2, 2, 2), True), ((2, 4, 2, 4), True),
                                     ((4, 6, 2, 2), False)])
def test_clover_and_D_orders_and_cstar(qxd, L, cstar, order):
    c = Case(qxd, torch, L, cstar=cstar, order=order, eps=0.5, seed=1004)
    try:
        got = np.empty((c.V, 2, 36))
        qxd.get_clover(c.lat, got)
        ref = c.to_boundary(O.packed_clover(c.op))
        assert rel_max_err(got, ref) < 1e-13
        psi = synth.gaussian_spinor(c.dims, 2001)
        assert rel_max_err(c.apply_D(psi), c.op.D(psi)) < 1e-13
    finally:
        c.close()


@pytest.mark.parametrize("dagger", [0, 1])
@pytest.mark.parametrize("L", [(4, 4, 4, 4), (6, 6, 6, 6), (2, 4, 6, 8)])
def test_apply_Dhat_f64(qxd, L, dagger):
    c = Case(qxd, torch, L)
    try:
        psi = synth.gaussian_spinor(c.dims, 2002)
        psi[c.lat_o.par == 1] = 0
        ref = c.op.Dhat_dag(psi) if dagger else c.op.Dhat(psi)
        got = c.apply_Dhat(c.even_half(psi), dagger=dagger)
        assert rel_max_err(got, c.even_half(ref)) < 1e-13
    finally:
        c.close()


# normwise relative error bounds: 8 units of roundoff of the storage format
BOUNDS = {1: 8 * 2.0 ** -24, 2: 8 * 2.0 ** -11, 3: 8 * 2.0 ** -8}


@pytest.mark.parametrize("prec", [1, 2, 3])
def test_low_precision_operators_within_roundoff_bounds(qxd, prec):
    c = Case(qxd, torch, (6, 4, 4, 8))
    try:
        psi = synth.gaussian_spinor(c.dims, 2003)
        ref = c.op.D(psi)
        e = np.linalg.norm(c.apply_D(psi, prec) - ref) / np.linalg.norm(ref)
        assert e < BOUNDS[prec], (prec, e)
        psi[c.lat_o.par == 1] = 0
        refh = c.even_half(c.op.Dhat(psi))
        eh = np.linalg.norm(c.apply_Dhat(c.even_half(psi), prec) - refh) / np.linalg.norm(refh)
        assert eh < BOUNDS[prec], (prec, eh)
        print(f"prec {prec}: D rel err {e:.2e}, Dhat rel err {eh:.2e}")
    finally:
        c.close()


def test_host_pointers_and_nrhs(qxd):
    c = Case(qxd, torch, (4, 4, 2, 6), on_device=False)
    try:
        psis = np.stack([synth.gaussian_spinor(c.dims, 2010 + k) for k in range(3)])
        out = np.empty_like(psis)
        qxd.apply_D(c.lat, out, psis, qxd.F64, nrhs=3)
        for k in range(3):
            assert rel_max_err(out[k], c.op.D(psis[k])) < 1e-13
    finally:
        c.close()


def test_vector_ops(qxd):
    c = Case(qxd, torch, (2, 2, 2, 2), build=False)
    try:
        r = np.random.default_rng(0)
        for n in [0, 1, 1000, 123457]:
            a = r.standard_normal(n) + 1j * r.standard_normal(n)
            b = r.standard_normal(n) + 1j * r.standard_normal(n)
            ta, tb = c.dev_tensor(a), c.dev_tensor(b)
            if n:
                assert abs(qxd.vec_dot(c.lat, ta, tb, n) - np.vdot(a, b)) < 1e-12 * n
            else:
                assert qxd.vec_dot(c.lat, ta, tb, n) == 0
            assert abs(qxd.vec_norm2(c.lat, ta, n) - np.vdot(a, a).real) <= 1e-12 * max(n, 1)
            qxd.vec_axpy(c.lat, 0.5 - 2j, ta, tb, n)
            torch.cuda.synchronize()
            got = tb.cpu().numpy().view(np.complex128)
            assert np.abs(got - (b + (0.5 - 2j) * a)).max(initial=0) < 1e-13
    finally:
        c.close()


def test_vector_ops_refuse_host_and_misaligned_pointers(qxd):
    import ctypes

    c = Case(qxd, torch, (2, 2, 2, 2), build=False)
    try:
        t = torch.zeros(2 * 100 + 1, dtype=torch.float64, device="cuda:0")
        host = np.zeros(200)
        re, im = ctypes.c_double(), ctypes.c_double()
        vp = ctypes.c_void_p
        for pa, pb in [(host.ctypes.data, t.data_ptr()), (t.data_ptr(), t.data_ptr() + 8)]:
            st = qxd.lib.qxd_vec_dot(vp(c.lat), vp(pa), vp(pb), 100, ctypes.byref(re), ctypes.byref(im))
            assert st == qxd.EINVAL
            st = qxd.lib.qxd_vec_axpy(vp(c.lat), 1.0, 0.0, vp(pa), vp(pb), 100)
            assert st == qxd.EINVAL
        assert qxd.lib.qxd_vec_norm2(vp(c.lat), vp(t.data_ptr() + 8), 100, ctypes.byref(re)) == qxd.EINVAL
        with pytest.raises(ValueError):
            qxd.vec_dot(c.lat, host, host, 100)
        assert qxd.vec_norm2(c.lat, t[:200], 100) == 0.0
    finally:
        c.close()


def test_reductions_are_deterministic(qxd):
    c = Case(qxd, torch, (2, 2, 2, 2), build=False)
    try:
        a = c.dev_tensor(np.random.default_rng(1).standard_normal(1 << 20) * (1 + 1j))
        vals = {qxd.vec_norm2(c.lat, a, 1 << 20) for _ in range(5)}
        assert len(vals) == 1
    finally:
        c.close()


def test_state_and_argument_errors(qxd):
    c = Case(qxd, torch, (2, 2, 2, 2), build=False)
    try:
        x = c.dev_tensor(np.zeros((c.V, 4, 3), dtype=complex))
        with pytest.raises(qxd.QxdError) as e:
            qxd.apply_D(c.lat, x, x)
        assert e.value.status == qxd.ESTATE
        qxd.build_clover(c.lat, -0.1, 1.9, 1.0)
        with pytest.raises(qxd.QxdError) as e:
            qxd.apply_D(c.lat, x, x, nrhs=0)
        assert e.value.status == qxd.EINVAL
        with pytest.raises(qxd.QxdError) as e:
            qxd.build_clover(c.lat, -4.0, 0.0, 0.0)  # A = 0: every block singular
        assert e.value.status == qxd.ESINGULAR
    finally:
        c.close()
