"""Three-level multigrid on the GPU (the multigrid GCR of Sec. 5.1) against the multigrid oracle:
the coarsest operator A2 entry by entry, the level-2 vectors, one level-1 K-cycle, one fine
preconditioner application, and MG-GCR solves to the paper's 1e-12 judged by the oracle's true
residual."""
import numpy as np
import pytest

from oracle import dfl_oracle as F
from oracle import mg_oracle as M
from oracle import qxd_oracle as O
from oracle import sap_oracle as S
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


def dense_stencil(A, nbr):
    """A nearest-neighbour stencil operator [nb][9][ns][ns] as a dense matrix."""
    nb, _, ns, _ = A.shape
    D = np.zeros((nb * ns, nb * ns), dtype=np.complex128)
    for b in range(nb):
        for s in range(9):
            bp = nbr[b, s]
            D[b * ns:(b + 1) * ns, bp * ns:(bp + 1) * ns] += A[b, s]
    return D


def cvecs(n, k, seed):
    return np.stack([synth.gaussian_spinor((n, 1, 1, 1), seed + j).reshape(-1)[:n] for j in range(k)])


def levels(qxd, c, L, block, cstar, ns1, agg, ns2, seed=4000):
    """Deflation (level 1) and aggregation (level 2) set up on the GPU and in the oracle from the
    same vectors; returns (oracle Deflation, oracle Aggregation, level-2 vectors)."""
    vs = np.stack([synth.gaussian_spinor(c.dims, seed + k) for k in range(ns1)])
    qxd.dfl_setup(c.lat, block, c.dev_tensor(vs))
    dfl = F.Deflation(c.op, S.sap_blocks(c.dims, block, cstar_L1=L[1] if cstar else None), list(vs))
    v2 = np.ascontiguousarray(cvecs(dfl.n, ns2, seed + 100))
    qxd.mg_setup(c.lat, v2, agg=agg)
    ag = M.Aggregation(dfl.A, M.block_grid(c.dims, block), ns1, agg, list(v2))
    return dfl, ag, v2


@pytest.mark.parametrize("L,block,cstar,ns1,agg,ns2", [
    ((4, 4, 4, 4), (2, 2, 2, 2), False, 3, (1, 1, 2, 2), 3),
    ((8, 4, 4, 4), (2, 2, 2, 2), False, 2, (2, 1, 1, 2), 4),   # level-2 grid 2 x 2 x 2 x 1
    ((4, 4, 4, 4), (2, 2, 2, 2), True, 3, (1, 2, 1, 1), 2),    # C*: 4 x 8 x 4 x 4, x shift of one aggregate
])
def test_coarsest_operator_matches_oracle(qxd, L, block, cstar, ns1, agg, ns2):
    """A2 = P2^+ A1 P2 from the GPU's stencil Galerkin product equals the oracle's dense product
    entry by entry (1e-10 of its largest entry)."""
    c = Case(qxd, torch, L, cstar=cstar)
    try:
        dfl, ag, v2 = levels(qxd, c, L, block, cstar, ns1, agg, ns2)
        A2, nbr2 = qxd.mg_get_coarse(c.lat)
        got = dense_stencil(A2, nbr2)
        err = np.abs(got - ag.A2).max() / np.abs(ag.A2).max()
        print(f"{L} cstar={cstar} agg {agg}: A2 {got.shape} max rel err {err:.2e}")
        assert err < 1e-10, err
        assert qxd.mg_info(c.lat)["nb2"] == ag.nb2
    finally:
        c.close()


def test_level2_vectors_and_level1_solve_match_oracle(qxd):
    """Inverse iteration on level 1 and one K-cycle, both FP64 on the GPU, against the oracle."""
    L = (4, 4, 4, 4)
    c = Case(qxd, torch, L)
    try:
        dfl, ag, v2 = levels(qxd, c, L, (2, 2, 2, 2), False, 4, (1, 1, 2, 2), 3)
        start = np.ascontiguousarray(cvecs(dfl.n, 2, 4300))
        out = np.empty_like(start)
        qxd.mg_generate(c.lat, start, out, n_it=2, k=6)
        ref = M.generate_level2(dfl.A, list(start), n_it=2, k=6, m=16)
        for j in range(2):
            err = np.linalg.norm(out[j] - ref[j]) / np.linalg.norm(ref[j])
            assert err < 1e-10, (j, err)
        # K1 with the set-up's default cycle (nu 2, n1 4, n2 8, m 8)
        mg = M.Multigrid(dfl, ag, None, nu=2, n1=4, n2=8, m=8)
        f = np.ascontiguousarray(cvecs(dfl.n, 1, 4400)[0])
        got = np.empty_like(f)
        qxd.mg_apply_level1(c.lat, got, f)
        want = mg.level1(f)
        err = np.linalg.norm(got - want) / np.linalg.norm(want)
        print(f"K1 rel err {err:.2e}, level-2 vectors {err:.2e}")
        assert err < 1e-10, err
        assert qxd.mg_info(c.lat)["level1_solves"] >= 1
    finally:
        c.close()


@pytest.mark.parametrize("ncy_pre", [0, 1])
def test_fine_preconditioner_matches_oracle(qxd, ncy_pre):
    """One application of the fine multigrid preconditioner (FP32 fine smoothing, FP64 coarse
    levels) against the oracle's FP64 one."""
    L = (4, 4, 4, 4)
    c = Case(qxd, torch, L)
    try:
        sb = (2, 2, 2, 2)
        vs = np.stack([synth.gaussian_spinor(c.dims, 4000 + k) for k in range(4)])
        qxd.dfl_setup(c.lat, (2, 2, 2, 2), c.dev_tensor(vs))
        dfl = F.Deflation(c.op, S.sap_blocks(c.dims, (2, 2, 2, 2)), list(vs))
        v2 = np.ascontiguousarray(cvecs(dfl.n, 3, 4100))
        qxd.mg_setup(c.lat, v2, agg=(1, 1, 2, 2), nu=2, n1=3, n2=6, m=8, ncy_pre=ncy_pre)
        ag = M.Aggregation(dfl.A, M.block_grid(c.dims, (2, 2, 2, 2)), 4, (1, 1, 2, 2), list(v2))
        mg = M.Multigrid(dfl, ag, S.sap_blocks(c.dims, sb), nu=2, n1=3, n2=6, m=8, ncy_pre=ncy_pre, ncy=1, nmr=4)
        r = synth.gaussian_spinor(c.dims, 4500)
        out = np.empty_like(r)
        qxd.mg_precond(c.lat, out, np.ascontiguousarray(r), sb, ncy=1, nmr=4)
        want = mg.precond(r)
        err = O.norm(out - want) / O.norm(want)
        print(f"ncy_pre {ncy_pre}: fine preconditioner rel err {err:.2e}")
        assert err < 1e-5, err
    finally:
        c.close()


@pytest.mark.parametrize("L,cstar,m0", [((8, 4, 4, 4), False, 0.0), ((4, 4, 4, 8), True, -0.1)])
def test_mg_gcr_solve(qxd, L, cstar, m0):
    """MG-GCR (level 1 from 8 SAP-improved random fields, level 2 by inverse iteration on level 1)
    to the paper's 1e-12, judged by the oracle; a field change makes the multigrid stale."""
    c = Case(qxd, torch, L, cstar=cstar, m0=m0)
    try:
        sb, db = (2, 2, 2, 2), (2, 2, 2, 2)
        start = c.dev_tensor(np.stack([synth.gaussian_spinor(c.dims, 4200 + k) for k in range(8)]))
        vecs = torch.empty_like(start)
        qxd.dfl_generate(c.lat, sb, start, vecs, n_it=4, ncy=1, nmr=4)
        qxd.dfl_setup(c.lat, db, vecs)
        n1 = qxd.dfl_info(c.lat)["nblocks"] * 8
        s2 = np.ascontiguousarray(cvecs(n1, 4, 4600))
        v2 = np.empty_like(s2)
        qxd.mg_generate(c.lat, s2, v2, n_it=3, k=8)
        agg = (2, 1, 1, 1) if not cstar else (1, 2, 1, 1)
        qxd.mg_setup(c.lat, v2, agg=agg, nu=2, n1=4, n2=8, m=8, ncy_pre=1)
        eta = synth.gaussian_spinor(c.dims, 2600)
        b = c.dev_tensor(eta)
        x = torch.empty_like(b)
        st, info = qxd.solve(c.lat, x, b, solver=qxd.SOLVER_MP_MG_GCR, tol=1e-12, sap_block=sb, sap_ncy=1,
                             sap_nmr=4, gcr_restart=16, maxiter=2000)
        assert st == qxd.OK, info
        res = O.true_rel_residual(c.op, as_c128(x, eta.shape), eta)
        assert res <= 1e-12, (res, info)
        st2, info2 = qxd.solve(c.lat, x, b, solver=qxd.SOLVER_MP_SAP_GCR, tol=1e-12, sap_block=sb, sap_ncy=2,
                               sap_nmr=4, gcr_restart=16, maxiter=2000)
        print(f"{L} cstar={cstar}: MG-GCR {info['iters_inner']} steps (residual {res:.1e}), SAP-GCR "
              f"{info2['iters_inner']} steps; {qxd.mg_info(c.lat)}")
        assert qxd.mg_info(c.lat)["level1_solves"] >= info["iters_inner"]
        qxd.build_clover(c.lat, m0, c.csw, c.csw_qed)  # the field changed: deflation and MG stale
        with pytest.raises(qxd.QxdError) as e:
            qxd.solve(c.lat, x, b, solver=qxd.SOLVER_MP_MG_GCR, tol=1e-12, sap_block=sb)
        assert e.value.status == qxd.ESTATE
    finally:
        c.close()


def test_mg_rejects_bad_input(qxd):
    L = (4, 4, 4, 4)
    c = Case(qxd, torch, L)
    try:
        x = c.dev_tensor(synth.gaussian_spinor(c.dims, 1))
        with pytest.raises(qxd.QxdError) as e:  # no deflation subspace yet
            qxd.mg_setup(c.lat, np.zeros((1, 16), complex), agg=(1, 1, 1, 1))
        assert e.value.status == qxd.ESTATE
        vs = np.stack([synth.gaussian_spinor(c.dims, 4000 + k) for k in range(2)])
        qxd.dfl_setup(c.lat, (2, 2, 2, 2), c.dev_tensor(vs))
        n1 = 16 * 2
        v = np.ascontiguousarray(cvecs(n1, 2, 7))
        for kw in [dict(agg=(3, 1, 1, 1)), dict(agg=(1, 1, 1, 1), nu=-1), dict(agg=(1, 1, 1, 1), m=17),
                   dict(agg=(1, 1, 1, 1), n1=0), dict(agg=(1, 1, 1, 1), ncy_pre=9)]:
            with pytest.raises(qxd.QxdError) as e:
                qxd.mg_setup(c.lat, v, **kw)
            assert e.value.status == qxd.EINVAL, kw
        with pytest.raises(qxd.QxdError) as e:  # 3 vectors on aggregates of one block of 2 entries
            qxd.mg_setup(c.lat, np.ascontiguousarray(cvecs(n1, 3, 9)), agg=(1, 1, 1, 1))
        assert e.value.status == qxd.EINVAL
        with pytest.raises(qxd.QxdError) as e:  # the same vector twice
            qxd.mg_setup(c.lat, np.ascontiguousarray(np.stack([v[0], v[0]])), agg=(2, 2, 2, 2))
        assert e.value.status == qxd.EINVAL and "dependent" in qxd.last_error(c.lat)
        with pytest.raises(qxd.QxdError) as e:  # a solve before mg_setup
            qxd.solve(c.lat, torch.empty_like(x), x, solver=qxd.SOLVER_MP_MG_GCR, tol=1e-10, sap_block=(2, 2, 2, 2))
        assert e.value.status == qxd.ESTATE
        qxd.mg_setup(c.lat, v, agg=(2, 2, 2, 2))
        qxd.dfl_setup(c.lat, (2, 2, 2, 2), c.dev_tensor(vs))  # a new level 1: level 2 is stale
        with pytest.raises(qxd.QxdError) as e:
            qxd.mg_apply_level1(c.lat, np.empty(n1, complex), np.ones(n1, complex))
        assert e.value.status == qxd.ESTATE
    finally:
        c.close()
