"""Links updated on the device (qxd_update_links): after replacing k links of the resident field,
the clover term (rebuilt at the sites whose plaquettes hold them) and D in every precision match
the oracle built on the updated field.  Judged at the FP64 operator tolerance (1e-13)."""
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


def _updated_case(qxd, c, k, seed, on_device):
    """Replace k random distinct links of the case's physical field; returns the oracle operator of
    the updated field and the lexicographic link entries that changed."""
    Vp = synth.volume(c.L)
    rng = np.random.default_rng(seed)
    lex = rng.choice(4 * Vp, size=k, replace=False) if k < 4 * Vp else np.arange(4 * Vp)
    newU = synth.random_su3(len(lex), seed + 1, eps=0.5)
    newA = synth.random_angles(len(lex), seed + 2)
    U2 = c.U_phys.reshape(-1, 3, 3).copy()
    A2 = c.A_phys.reshape(-1).copy()
    U2[lex] = newU
    A2[lex] = newA
    U2, A2 = U2.reshape(c.U_phys.shape), A2.reshape(c.A_phys.shape)
    # the entries in the lattice's site order (IPT: the boundary index of the physical site)
    if c.order == qxd.ORDER_IPT:
        x = O.coords_of(c.L)[lex // 4]
        B = None if c.blocks is None else tuple(b if b != L2 else L1 for b, L1, L2 in zip(c.blocks, c.L, c.dims))
        idx = O.ipt(x, c.L, B) * 4 + lex % 4
    else:
        idx = lex
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    su3 = np.ascontiguousarray(newU)
    ang = np.ascontiguousarray(newA)
    if on_device:
        qxd.update_links(c.lat, torch.from_numpy(idx).to(c.dev), torch.from_numpy(su3.view(np.float64)).to(c.dev),
                         torch.from_numpy(ang).to(c.dev))
    else:
        qxd.update_links(c.lat, idx, su3, ang)
    Uf, Af = (O.cstar_double_gauge(U2, A2, c.L) if c.cstar else (U2, A2))
    return O.Operator(c.lat_o, Uf, Af, c.q, c.m0, c.csw, c.csw_qed)


@pytest.mark.parametrize("L,cstar,order,blocks,k,on_device", [
    ((4, 4, 4, 4), False, 0, None, 7, True),
    ((6, 4, 2, 4), False, 0, None, 40, False),
    ((4, 2, 2, 4), True, 0, None, 5, True),
    ((4, 4, 4, 4), False, 1, (2, 2, 2, 2), 9, True),
    ((4, 4, 4, 4), False, 0, None, 4 * 256, True),  # every link: the full rebuild path
])
def test_update_links_matches_oracle(qxd, L, cstar, order, blocks, k, on_device):
    c = Case(qxd, torch, L, cstar=cstar, order=order, blocks=blocks)
    try:
        op = _updated_case(qxd, c, k, 77, on_device)
        clov = np.empty((c.V, 2, 36))
        qxd.get_clover(c.lat, clov)
        ref = O.pack36(O.clover_blocks(op.C))
        ref_b = c.to_boundary(ref)
        assert np.abs(clov - ref_b).max() <= 1e-13 * np.abs(ref).max()
        psi = synth.gaussian_spinor(c.dims, 41)
        Dref = op.D(psi)
        got = c.apply_D(psi, qxd.F64)
        assert np.abs(got - Dref).max() <= 1e-13 * np.abs(Dref).max()
        for prec, u in ((qxd.F32, 2.0 ** -24), (qxd.F16N, 2.0 ** -11), (qxd.BF16N, 2.0 ** -8)):
            g = c.apply_D(psi, prec)
            assert np.linalg.norm(g - Dref) / np.linalg.norm(Dref) <= 8 * u, prec
        if c.order != qxd.ORDER_LEXI:
            return
        # the Schur complement uses the rebuilt odd-site inverse
        pe = c.even_half(psi)
        pfull = np.where((c.lat_o.par == 0)[:, None, None], psi, 0)
        Dh = op.Dhat(pfull)[c.lat_o.par == 0]
        assert np.abs(c.apply_Dhat(pe) - Dh).max() <= 1e-13 * np.abs(Dh).max()
    finally:
        c.close()


def test_update_links_refuses_bad_input(qxd):
    c = Case(qxd, torch, (4, 4, 2, 2))
    try:
        with pytest.raises(qxd.QxdError) as e:
            qxd.update_links(c.lat, np.array([0, 4 * c.V], dtype=np.int64), synth.random_su3(2, 3))
        assert e.value.status == qxd.EINVAL
        # the valid link was written and the clover is now marked unbuilt
        x = c.dev_tensor(synth.gaussian_spinor(c.dims, 1))
        with pytest.raises(qxd.QxdError) as e:
            qxd.apply_D(c.lat, torch.empty_like(x), x)
        assert e.value.status == qxd.ESTATE
        qxd.build_clover(c.lat, c.m0, c.csw, c.csw_qed)
        assert qxd.lib.qxd_update_links(c.lat, -1, None, None, None, 0) == qxd.EINVAL
        assert qxd.lib.qxd_update_links(c.lat, 0, None, None, None, 0) == qxd.OK
    finally:
        c.close()
