"""Multi-right-hand-side apply and solve (12 spin-colour point sources) against the oracle."""
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


def point_sources(dims, site=0):
    return np.stack([synth.point_source(dims, k // 3, k % 3, site) for k in range(12)])


@pytest.mark.parametrize("L,nrhs,cstar", [((6, 6, 6, 6), 12, False), ((4, 2, 2, 6), 13, False),
                                          ((2, 2, 4, 2), 5, True)])
def test_mrhs_apply_matches_oracle_and_single_rhs(qxd, L, nrhs, cstar):
    c = Case(qxd, torch, L, cstar=cstar)
    try:
        psis = np.stack([synth.gaussian_spinor(c.dims, 3000 + k) for k in range(nrhs)])
        x = c.dev_tensor(psis)
        y = torch.empty_like(x)
        qxd.apply_D(c.lat, y, x, qxd.F32, nrhs=nrhs)
        got = as_c128(y, psis.shape)
        for k in range(nrhs):
            ref = c.op.D(psis[k])
            e = np.linalg.norm(got[k] - ref) / np.linalg.norm(ref)
            assert e < 8 * 2.0 ** -24, (k, e)
            single = c.apply_D(psis[k], qxd.F32)
            assert np.linalg.norm(got[k] - single) / np.linalg.norm(single) < 1e-6
    finally:
        c.close()


@pytest.mark.parametrize("L,cstar", [((4, 4, 4, 4), False), ((4, 2, 2, 4), True)])
def test_mrhs_solve_point_sources(qxd, L, cstar):
    c = Case(qxd, torch, L, cstar=cstar)
    try:
        eta = point_sources(c.dims)
        b = c.dev_tensor(eta)
        x = torch.empty_like(b)
        st, infos = qxd.solve_mrhs(c.lat, x, b, 12, solver=qxd.SOLVER_MP_BICGSTAB_EO, inner_prec=qxd.F32, tol=1e-10)
        assert st == qxd.OK
        psi = as_c128(x, eta.shape)
        for k in range(12):
            res = O.true_rel_residual(c.op, psi[k], eta[k])
            assert res <= 1e-10, (k, res, infos[k])
        print(f"{L} cstar={cstar}: {infos[0]}")
    finally:
        c.close()


def test_mrhs_solve_with_a_zero_source(qxd):
    c = Case(qxd, torch, (4, 4, 2, 2))
    try:
        eta = np.stack([synth.gaussian_spinor(c.dims, 5), np.zeros((c.V, 4, 3), complex),
                        synth.gaussian_spinor(c.dims, 6)])
        b = c.dev_tensor(eta)
        x = torch.empty_like(b)
        st, infos = qxd.solve_mrhs(c.lat, x, b, 3, solver=qxd.SOLVER_MP_BICGSTAB_EO, inner_prec=qxd.F32)
        assert st == qxd.OK
        psi = as_c128(x, eta.shape)
        assert np.abs(psi[1]).max() == 0
        for k in (0, 2):
            assert O.true_rel_residual(c.op, psi[k], eta[k]) <= 1e-10
    finally:
        c.close()


UNIT16 = {"f16n": 2.0 ** -11, "bf16n": 2.0 ** -8}


@pytest.mark.parametrize("prec", ["f16n", "bf16n"])
@pytest.mark.parametrize("L,nrhs,cstar", [((6, 6, 6, 6), 12, False), ((4, 2, 2, 6), 13, False),
                                          ((2, 2, 4, 2), 5, True), ((8, 6, 4, 6), 7, False)])
def test_mrhs16_apply_per_site(qxd, prec, L, nrhs, cstar):
    """The 16-bit multi-RHS hop (tile-staged links and clover, groups of right-hand sides) against
    the FP64 oracle site by site: max error over a site's 12 entries <= 8 u max |ref| there, and
    within 4 u per site of the single-RHS 16-bit operator (which projects and transports in packed
    16-bit arithmetic, where the multi-RHS hop computes in FP32 on the same stored values)."""
    c = Case(qxd, torch, L, cstar=cstar)
    try:
        psis = np.stack([synth.gaussian_spinor(c.dims, 3100 + k) for k in range(nrhs)])
        x = c.dev_tensor(psis)
        y = torch.empty_like(x)
        qxd.apply_D(c.lat, y, x, qxd.PREC[prec], nrhs=nrhs)
        got = as_c128(y, psis.shape)
        worst = 0.0
        for k in range(nrhs):
            ref = c.op.D(psis[k])
            e = np.abs(got[k] - ref).reshape(c.V, -1).max(axis=1) / np.abs(ref).reshape(c.V, -1).max(axis=1)
            worst = max(worst, float(e.max()) / UNIT16[prec])
            single = c.apply_D(psis[k], qxd.PREC[prec])
            d = np.abs(got[k] - single).reshape(c.V, -1).max(axis=1) / np.abs(single).reshape(c.V, -1).max(axis=1)
            assert d.max() <= 4 * UNIT16[prec], (k, d.max() / UNIT16[prec])
        assert worst <= 8, worst
        print(f"{L} nrhs={nrhs} {prec}: worst per-site error {worst:.2f} u")
    finally:
        c.close()


@pytest.mark.parametrize("prec", ["f16n", "bf16n"])
@pytest.mark.parametrize("L,cstar", [((4, 4, 4, 4), False), ((4, 2, 2, 4), True), ((8, 4, 6, 4), False)])
def test_mrhs16_solve_point_sources(qxd, prec, L, cstar):
    """The multi-RHS solve with the 16-bit inner operator: every right-hand side judged by the
    oracle's FP64 true residual."""
    c = Case(qxd, torch, L, cstar=cstar)
    try:
        eta = point_sources(c.dims)
        b = c.dev_tensor(eta)
        x = torch.empty_like(b)
        st, infos = qxd.solve_mrhs(c.lat, x, b, 12, solver=qxd.SOLVER_MP_BICGSTAB_EO, inner_prec=qxd.PREC[prec],
                                   tol=1e-10)
        assert st == qxd.OK, infos[0]
        psi = as_c128(x, eta.shape)
        for k in range(12):
            res = O.true_rel_residual(c.op, psi[k], eta[k])
            assert res <= 1e-10, (k, res, infos[k])
        print(f"{L} cstar={cstar} {prec}: {infos[0]}")
    finally:
        c.close()
