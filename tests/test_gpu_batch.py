"""Batched persistent solve of independent lattices of uneven volume (one cooperative launch per
outer round), checked lattice by lattice against the oracle's true residual."""
import numpy as np
import pytest

from oracle import qxd_oracle as O
from paper_2502_02490_gb300 import synth
from tests.gpu_util import Case, as_c128

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

# (T, L1, L2, L3), C*, eps, m0: uneven volumes, ragged against the 256-site tiles
SHAPES = [((4, 4, 4, 4), False, 0.2, 0.0), ((6, 4, 4, 6), False, 0.3, -0.1), ((2, 2, 4, 6), False, 0.4, 0.1),
          ((4, 2, 2, 4), True, 0.5, -0.05), ((8, 6, 6, 6), False, 0.35, -0.1)]


@pytest.fixture(scope="module")
def qxd():
    import __graft_entry__

    __graft_entry__.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2502_02490_gb300 import qxd as q

    return q


def make_cases(qxd, shapes=SHAPES):
    return [Case(qxd, torch, L, cstar=cs, eps=eps, m0=m0, seed=1100 + k) for k, (L, cs, eps, m0) in enumerate(shapes)]


def check(cs, xs, etas, infos, tol=1e-10):
    for c, x, e, info in zip(cs, xs, etas, infos):
        if not np.any(e):
            assert not np.any(as_c128(x, e.shape)), "zero source must give x = 0"
            continue
        res = O.true_rel_residual(c.op, as_c128(x, e.shape), e)
        assert res <= tol, (c.L, res, info)
        assert info["status"] == 0 and info["true_rel_res"] <= tol


def test_batch_solves_every_lattice(qxd):
    cs = make_cases(qxd)
    try:
        etas = [synth.gaussian_spinor(c.dims, 2100 + k) for k, c in enumerate(cs)]
        bs = [c.dev_tensor(e) for c, e in zip(cs, etas)]
        xs = [torch.full_like(b, float("nan")) for b in bs]  # x is output only
        for rep in range(2):  # the second call reuses the tuned tile shape and the cached state
            st, infos = qxd.solve_batch([c.lat for c in cs], xs, bs, tol=1e-10)
            assert st == qxd.OK, infos
            check(cs, xs, etas, infos)
        cfg = qxd.batch_last_config()
        assert cfg["sites_per_thread"] in (1, 2, 4) and cfg["threads"] == 256 and cfg["blocks_per_sm"] in (1, 2)
        print("batch:", [i["iters_inner"] for i in infos], infos[0]["iters_outer"], cfg)
        # another set led by the same lattice replaces the cached state
        sub = [cs[0], cs[2], cs[4]]
        st, infos = qxd.solve_batch([c.lat for c in sub], [xs[0], xs[2], xs[4]], [bs[0], bs[2], bs[4]], tol=1e-10)
        assert st == qxd.OK
        check(sub, [xs[0], xs[2], xs[4]], [etas[0], etas[2], etas[4]], infos)
    finally:
        for c in cs:
            c.close()


def test_batch_zero_source_and_single_lattice(qxd):
    cs = make_cases(qxd, SHAPES[:2])
    try:
        etas = [np.zeros((cs[0].V, 4, 3), complex), synth.gaussian_spinor(cs[1].dims, 31)]
        bs = [c.dev_tensor(e) for c, e in zip(cs, etas)]
        xs = [torch.full_like(b, 7.0) for b in bs]
        st, infos = qxd.solve_batch([c.lat for c in cs], xs, bs, tol=1e-10)
        assert st == qxd.OK
        check(cs, xs, etas, infos)
        st, infos = qxd.solve_batch([cs[1].lat], [xs[1]], [bs[1]], tol=1e-10)  # a batch of one
        assert st == qxd.OK
        check(cs[1:], xs[1:], etas[1:], infos)
    finally:
        for c in cs:
            c.close()


def test_batch_iteration_cap_reports_noconv(qxd):
    cs = make_cases(qxd, SHAPES[:2])
    try:
        bs = [c.dev_tensor(synth.gaussian_spinor(c.dims, 41 + k)) for k, c in enumerate(cs)]
        xs = [torch.empty_like(b) for b in bs]
        st, infos = qxd.solve_batch([c.lat for c in cs], xs, bs, check=False, tol=1e-10, maxiter=3, max_outer=1)
        assert st == qxd.ENOCONV
        assert all(i["status"] == qxd.ENOCONV for i in infos)
        assert all(torch.isfinite(x).all() for x in xs)
    finally:
        for c in cs:
            c.close()


def test_batch_barrier_timeout_is_reported_and_recoverable(qxd):
    cs = make_cases(qxd, SHAPES[:2])
    try:
        etas = [synth.gaussian_spinor(c.dims, 7 + k) for k, c in enumerate(cs)]
        bs = [c.dev_tensor(e) for c, e in zip(cs, etas)]
        xs = [torch.empty_like(b) for b in bs]
        lats = [c.lat for c in cs]
        st, infos = qxd.solve_batch(lats, xs, bs, check=False, tol=1e-10)
        assert st == qxd.OK, infos
        qxd.batch_set_spin_limit(1)  # every barrier wait gives up at once
        try:
            st, _ = qxd.solve_batch(lats, xs, bs, check=False, tol=1e-10)
        finally:
            qxd.batch_set_spin_limit(20000000)
        assert st == qxd.ETIMEOUT
        assert "timed out" in qxd.last_error(lats[0])
        st, infos = qxd.solve_batch(lats, xs, bs, check=False, tol=1e-10)  # the context is still usable
        assert st == qxd.OK, infos
        check(cs, xs, etas, infos)
    finally:
        for c in cs:
            c.close()


def test_batch_tuning_cache_file(qxd, tmp_path):
    """A newly tuned set is appended to the cache file; an entry in the file is used untuned."""
    path = tmp_path / "tune.txt"
    qxd.batch_tune_cache(str(path))
    cs = []
    try:
        # volumes 48 and 48: a set no other test tunes
        cs = make_cases(qxd, [((6, 2, 2, 2), False, 0.3, -0.1), ((2, 2, 2, 6), False, 0.3, -0.1)])
        etas = [synth.gaussian_spinor(c.dims, 2400 + k) for k, c in enumerate(cs)]
        bs = [c.dev_tensor(e) for c, e in zip(cs, etas)]
        xs = [torch.empty_like(b) for b in bs]
        st, infos = qxd.solve_batch([c.lat for c in cs], xs, bs, tol=1e-10)
        assert st == qxd.OK
        check(cs, xs, etas, infos)
        lines = path.read_text().splitlines()
        cfg = qxd.batch_last_config()
        assert len(lines) == 1, lines
        f = lines[0].split()
        assert f[:2] == ["qxd-batch-tune", "1"] and f[4] == "48,48,"
        assert (int(f[5]), int(f[6])) == (cfg["blocks_per_sm"], cfg["sites_per_thread"])
        # a hand-written entry for a lone lattice of volume 48 (a set not tuned in this process)
        path.write_text(lines[0] + "\n" + " ".join(f[:4] + ["48,", "1", "4"]) + "\n")
        st, infos = qxd.solve_batch([cs[1].lat], [xs[1]], [bs[1]], tol=1e-10)
        assert st == qxd.OK
        check([cs[1]], [xs[1]], [etas[1]], infos)
        cfg = qxd.batch_last_config()
        assert (cfg["blocks_per_sm"], cfg["sites_per_thread"]) == (1, 4), cfg
        assert len(path.read_text().splitlines()) == 2  # used, not re-tuned
    finally:
        qxd.batch_tune_cache(None)
        for c in cs:
            c.close()
