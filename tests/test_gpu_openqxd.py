"""openQxD layout interop (Sec. 4.1): cache-blocked Eq. ipt site order for every exchanged field,
and the gauge field stored as eight links per odd site, checked against the oracle in FP64."""
import numpy as np
import pytest

from oracle import qxd_oracle as O
from paper_2502_02490_gb300 import synth
from tests.gpu_util import Case, rel_max_err

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


# (T, L1, L2, L3), C*, blocks (odd block extents included: any divisor tiles Eq. ipt)
CASES = [((8, 4, 4, 4), False, (4, 2, 2, 4)), ((6, 6, 2, 4), False, (3, 3, 1, 2)), ((4, 4, 6, 6), False, (2, 1, 3, 3)),
         ((4, 2, 2, 2), True, (2, 1, 2, 2)), ((4, 4, 2, 4), True, (2, 2, 1, 2))]


@pytest.mark.parametrize("openqxd", [False, True])
@pytest.mark.parametrize("L,cstar,B", CASES)
def test_blocked_order_and_openqxd_gauge(qxd, L, cstar, B, openqxd):
    c = Case(qxd, torch, L, cstar=cstar, order=qxd.ORDER_IPT, eps=0.5, seed=1007, blocks=B, openqxd_gauge=openqxd)
    try:
        got = np.empty((c.V, 2, 36))
        qxd.get_clover(c.lat, got)
        assert rel_max_err(got, c.to_boundary(O.packed_clover(c.op))) < 1e-13
        psi = synth.gaussian_spinor(c.dims, 2002)
        assert rel_max_err(c.apply_D(psi), c.op.D(psi)) < 1e-13
    finally:
        c.close()


def test_openqxd_gauge_equals_canonical_load(qxd):
    """The same field through both loaders gives the same operator bit for bit."""
    L, B = (4, 4, 4, 4), (2, 2, 2, 2)
    a = Case(qxd, torch, L, order=qxd.ORDER_IPT, blocks=B, seed=1011)
    b = Case(qxd, torch, L, order=qxd.ORDER_IPT, blocks=B, seed=1011, openqxd_gauge=True)
    try:
        psi = synth.gaussian_spinor(a.dims, 7)
        assert np.array_equal(a.apply_D(psi), b.apply_D(psi))
    finally:
        a.close()
        b.close()


def test_block_and_order_errors(qxd):
    c = Case(qxd, torch, (4, 4, 4, 4), build=False)  # lexicographic lattice
    d = Case(qxd, torch, (4, 4, 4, 4), order=qxd.ORDER_IPT, build=False)
    try:
        with pytest.raises(qxd.QxdError) as e:
            qxd.set_ipt_blocks(c.lat, (2, 2, 2, 2))
        assert e.value.status == qxd.EINVAL
        for bad in ((3, 2, 2, 2), (0, 2, 2, 2), (4, 4, 4, 8)):
            with pytest.raises(qxd.QxdError) as e:
                qxd.set_ipt_blocks(d.lat, bad)
            assert e.value.status == qxd.EINVAL
        u8 = torch.zeros(c.V // 2 * 8 * 18, dtype=torch.float64, device="cuda")
        with pytest.raises(qxd.QxdError) as e:
            qxd.load_gauge_openqxd(c.lat, u8, None, 0.0)
        assert e.value.status == qxd.EINVAL
    finally:
        c.close()
        d.close()
