"""The dot product entry point that allocates no device memory (qxd_vec_dot_noalloc).

It serves callers that cannot call cudaMalloc: code running during CUDA-graph stream capture,
code whose device memory belongs to a framework's caching allocator, and latency-critical
loops that cannot afford the synchronisation an allocation may cause.  Its scratch is a static
array inside the library.  This file is collected last so that a run stopping at the first
failure has already run every other test.
"""
import numpy as np
import pytest

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


def test_noalloc_dot_matches_the_allocating_entry_point_twice(qxd):
    dev = torch.device("cuda:0")
    stream = torch.cuda.current_stream(dev)
    lat = qxd.create_lattice((2, 2, 2, 2), stream=stream.cuda_stream)  # for qxd_vec_dot only
    try:
        r = np.random.default_rng(42)
        for n in [1, 4097, 1_000_003, qxd.NOALLOC_MAX_N]:
            out = torch.zeros(2, dtype=torch.float64, device=dev)
            for call in range(2):  # two calls in a row share the static scratch
                a = r.standard_normal(2 * n) * (1 + call)
                b = r.standard_normal(2 * n)
                ta = torch.from_numpy(a).to(dev)
                tb = torch.from_numpy(b).to(dev)
                qxd.vec_dot_noalloc(ta, tb, n, out, stream.cuda_stream)
                ref = qxd.vec_dot(lat, ta, tb, n)
                torch.cuda.synchronize()
                got = complex(out[0].item(), out[1].item())
                assert abs(got - ref) < 1e-12 * n, (n, call, got, ref)
    finally:
        qxd.destroy_lattice(lat)


def test_noalloc_dot_limits(qxd):
    dev = torch.device("cuda:0")
    out = torch.full((2,), 7.0, dtype=torch.float64, device=dev)
    qxd.vec_dot_noalloc(None, None, 0, out)
    torch.cuda.synchronize()
    assert out.tolist() == [0.0, 0.0]
    with pytest.raises(qxd.QxdError) as e:
        qxd.vec_dot_noalloc(out, out, qxd.NOALLOC_MAX_N + 1, out)
    assert e.value.status == qxd.EINVAL and "capacity" in qxd.last_error(None)
