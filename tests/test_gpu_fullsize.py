"""Full-size parity: 32^3x64 (the bench workload) and 48^3x96 with C* (doubled to 96x48x48x96).

The oracle evaluates the same formulas at sampled sites (D_at_sites, clover at sites); the GPU
runs in the launch configuration bench.py times."""
import numpy as np
import pytest

from oracle import qxd_oracle as O
from paper_2502_02490_gb300 import synth
from tests.gpu_util import as_c128

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

WORKLOADS = {
    "32^3x64": dict(L=(64, 32, 32, 32), cstar=False, eps=0.4, q=2 / 3, m0=-0.2, gseed=1001, sseed=2001),
    "48^3x96 C*": dict(L=(96, 48, 48, 48), cstar=True, eps=0.35, q=-1 / 3, m0=-0.1, gseed=1004, sseed=2004),
}
CSW, CQ = 1.9, 1.0


@pytest.fixture(scope="module")
def qxd():
    import __graft_entry__

    __graft_entry__.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2502_02490_gb300 import qxd as q

    return q


@pytest.mark.parametrize("name", list(WORKLOADS))
def test_fullsize_operator_clover_and_solve(qxd, name):
    w = WORKLOADS[name]
    L = w["L"]
    lat_o = O.Lattice(L, antiperiodic=True, cstar=w["cstar"])
    U, A = synth.gauge_field(L, w["gseed"], w["eps"])
    eta = synth.gaussian_spinor(lat_o.dims, w["sseed"])
    dev = torch.device("cuda:0")
    stream = torch.cuda.current_stream(dev)
    lat = qxd.create_lattice(L, qxd.BC_ANTIPERIODIC, int(w["cstar"]), qxd.ORDER_LEXI, stream.cuda_stream)
    try:
        qxd.load_gauge(lat, torch.from_numpy(U.view(np.float64)).to(dev), torch.from_numpy(A).to(dev), w["q"])
        qxd.build_clover(lat, w["m0"], CSW, CQ)
        x = torch.from_numpy(eta.view(np.float64)).to(dev)
        y = torch.empty_like(x)
        qxd.apply_D(lat, y, x, qxd.F64)
        psi = torch.empty_like(x)
        st, info = qxd.solve(lat, psi, x, solver=qxd.SOLVER_MP_BICGSTAB_EO, inner_prec=qxd.F16N, tol=1e-10)
        torch.cuda.synchronize()
        assert st == qxd.OK and info["true_rel_res"] <= 1e-10, info
        Dy = as_c128(y, eta.shape)
        sol = as_c128(psi, eta.shape)
        del x, y, psi
        clov = np.empty((lat_o.V, 2, 36))
        qxd.get_clover(lat, clov)
        bad = qxd.check_guards(lat)  # no kernel of the full-size launches wrote past a buffer
    finally:
        qxd.destroy_lattice(lat)
    assert bad == 0, f"{bad} guard bytes overwritten"
    # oracle at sampled sites: every boundary class (time wrap, C* mirror crossings) is hit by
    # taking corners as well as random sites
    rng = np.random.default_rng(0)
    d = lat_o.dims
    corners = [O.lexi(np.array(c), d) for c in [(0, 0, 0, 0), (d[0] - 1, d[1] - 1, d[2] - 1, d[3] - 1),
                                                (0, d[1] // 2, d[2] - 1, 0), (d[0] - 1, 0, 0, d[3] - 1)]]
    sites = np.unique(np.concatenate([rng.choice(lat_o.V, 120, replace=False), corners]))
    Uf, Af = (O.cstar_double_gauge(U, A, L) if w["cstar"] else (U, A))
    ref = O.D_at_sites(lat_o, Uf, Af, w["q"], w["m0"], CSW, CQ, eta, sites)
    err = np.abs(Dy[sites] - ref).max() / np.abs(ref).max()
    assert err < 1e-13, err
    Cref = O.pack36(O.clover_blocks(O.clover_matrix(lat_o, Uf, Af, w["q"], w["m0"], CSW, CQ, sites=sites)))
    assert np.abs(clov[sites] - Cref).max() < 1e-13 * np.abs(Cref).max()
    r = eta[sites] - O.D_at_sites(lat_o, Uf, Af, w["q"], w["m0"], CSW, CQ, sol, sites)
    # the sampled residual must be consistent with a full residual <= 1e-10 ||eta||
    assert np.sqrt((np.abs(r) ** 2).sum() * lat_o.V / len(sites)) <= 3e-10 * np.linalg.norm(eta)
    print(f"{name}: apply_D rel err {err:.2e}, solve {info}")


# unit roundoff of the 16-bit storage formats (round to nearest): FP16 has an 11-bit
# significand, BF16 an 8-bit one
UNIT = {"f16n": 2.0 ** -11, "bf16n": 2.0 ** -8}
C_SITE = 8  # per-site bound: max_i |gpu_i - ref_i| <= C_SITE * u * max_i |ref_i| over one site's 12 entries


def _sample_sites(lat_o, n, parity, seed):
    """n random sites of the given parity (None: any) plus corners that cross the time and C*
    mirror boundaries (moved by one step in x3 where the corner has the other parity)."""
    d = lat_o.dims
    rng = np.random.default_rng(seed)
    pool = np.arange(lat_o.V) if parity is None else np.flatnonzero(lat_o.par == parity)
    corners = []
    for c in [(0, 0, 0, 0), (d[0] - 1, d[1] - 1, d[2] - 1, d[3] - 1), (0, d[1] // 2, d[2] - 1, 0),
              (d[0] - 1, 0, 0, d[3] - 1), (d[0] - 1, d[1] // 2 - 1, d[2] - 1, 0)]:
        c = np.array(c)
        if parity is not None and int(c.sum()) % 2 != parity:
            c[3] = (c[3] + 1) % d[3]
        corners.append(O.lexi(c, d))
    return np.unique(np.concatenate([rng.choice(pool, n, replace=False), corners]))


def _site_ratio(got, ref):
    """Per site: max |got - ref| / max |ref| over the site's 12 complex entries."""
    e = np.abs(got - ref).reshape(len(ref), -1).max(axis=1)
    m = np.abs(ref).reshape(len(ref), -1).max(axis=1)
    return e / m


@pytest.mark.parametrize("name", list(WORKLOADS))
def test_fullsize_16bit_dslash_per_site(qxd, name):
    """The 16-bit operators the mixed-precision solve runs (D and the Dhat the bench times, in the
    INV and DHAT2 hop instantiations and the launch configuration of the full-size lattice),
    site by site against the FP64 oracle at sampled sites."""
    w = WORKLOADS[name]
    L = w["L"]
    lat_o = O.Lattice(L, antiperiodic=True, cstar=w["cstar"])
    U, A = synth.gauge_field(L, w["gseed"], w["eps"])
    Uf, Af = (O.cstar_double_gauge(U, A, L) if w["cstar"] else (U, A))
    eta = synth.gaussian_spinor(lat_o.dims, w["sseed"])
    sites = _sample_sites(lat_o, 120, None, 0)
    esites = _sample_sites(lat_o, 120, 0, 1)
    erank = np.searchsorted(np.flatnonzero(lat_o.par == 0), esites)
    dev = torch.device("cuda:0")
    stream = torch.cuda.current_stream(dev)
    lat = qxd.create_lattice(L, qxd.BC_ANTIPERIODIC, int(w["cstar"]), qxd.ORDER_LEXI, stream.cuda_stream)
    got = {}
    try:
        qxd.load_gauge(lat, torch.from_numpy(U.view(np.float64)).to(dev), torch.from_numpy(A).to(dev), w["q"])
        qxd.build_clover(lat, w["m0"], CSW, CQ)
        x = torch.from_numpy(eta.view(np.float64)).to(dev)
        y = torch.empty_like(x)
        st_idx = torch.from_numpy(sites).to(dev)
        for prec in ("f16n", "bf16n"):
            qxd.apply_D(lat, y, x, qxd.PREC[prec])
            got[("D", prec, 0)] = as_c128(y.view(lat_o.V, 24)[st_idx], (len(sites), 4, 3))
        del y
        even_idx = torch.from_numpy(np.flatnonzero(lat_o.par == 0)).to(dev)
        xe = x.view(lat_o.V, 24)[even_idx].contiguous()
        del x
        ye = torch.empty_like(xe)
        er_idx = torch.from_numpy(erank).to(dev)
        for prec, dag in (("f16n", 0), ("f16n", 1), ("bf16n", 0)):
            qxd.apply_Dhat_eo(lat, ye, xe, qxd.PREC[prec], dag)
            got[("Dhat", prec, dag)] = as_c128(ye.view(-1, 24)[er_idx], (len(esites), 4, 3))
        del xe, ye
        torch.cuda.synchronize()
        bad = qxd.check_guards(lat)
    finally:
        qxd.destroy_lattice(lat)
    assert bad == 0, f"{bad} guard bytes overwritten"
    args = (w["q"], w["m0"], CSW, CQ)
    ref_D = O.D_at_sites(lat_o, Uf, Af, *args, eta, sites)
    ref_Dh = {dag: O.Dhat_at_sites(lat_o, Uf, Af, *args, eta, esites, dagger=bool(dag)) for dag in (0, 1)}
    worst = {}
    for (op, prec, dag), g in got.items():
        ref = ref_D if op == "D" else ref_Dh[dag]
        ratio = _site_ratio(g, ref) / UNIT[prec]
        worst[(op, prec, dag)] = float(ratio.max())
        assert ratio.max() <= C_SITE, (op, prec, dag, float(ratio.max()))
    print(f"{name}: worst per-site error in units of roundoff: " +
          ", ".join(f"{op}{'^+' if d else ''} {p} {v:.2f}" for (op, p, d), v in worst.items()))
