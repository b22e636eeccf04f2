"""The dot product entry point that allocates no device memory (qxd_vec_dot_noalloc).

It serves callers that cannot call cudaMalloc: code whose device memory belongs to a
framework's caching allocator, and latency-critical loops that cannot afford the
synchronisation an allocation may cause.  Its scratch is a static
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
                # FP64 summation error bound: a few units of roundoff times sum |a_k| |b_k|
                za, zb = a.view(np.complex128), b.view(np.complex128)
                scale = float(np.sum(np.abs(za) * np.abs(zb)))
                assert abs(got - np.vdot(za, zb)) <= 1e-13 * scale, (n, call, got)
                assert abs(got - ref) <= 1e-13 * scale, (n, call, got, ref)
                # the same inputs again give the same bits (fixed blocking and summation order)
                out2 = torch.zeros(2, dtype=torch.float64, device=dev)
                qxd.vec_dot_noalloc(ta, tb, n, out2, stream.cuda_stream)
                torch.cuda.synchronize()
                assert torch.equal(out, out2), (n, call)
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


def test_noalloc_dot_refuses_host_and_misaligned_pointers(qxd):
    """Pointers the kernel cannot use are refused on the host with QXD_EINVAL, before any launch."""
    import ctypes

    dev = torch.device("cuda:0")
    out = torch.zeros(2, dtype=torch.float64, device=dev)
    t = torch.zeros(2 * 64 + 1, dtype=torch.float64, device=dev)
    host = np.zeros(2 * 64)
    cases = [
        (host.ctypes.data, t.data_ptr(), out.data_ptr()),                 # a in host memory
        (t.data_ptr(), t.data_ptr() + 8, out.data_ptr()),                 # b only 8-byte aligned
        (t.data_ptr(), t.data_ptr(), host.ctypes.data),                   # out in host memory
        (t.data_ptr(), t.data_ptr(), out.data_ptr() + 4),                 # out not 8-byte aligned
    ]
    for pa, pb, po in cases:
        st = qxd.lib.qxd_vec_dot_noalloc(ctypes.c_void_p(pa), ctypes.c_void_p(pb), 64, ctypes.c_void_p(po), None)
        assert st == qxd.EINVAL, (pa, pb, po)
    with pytest.raises(ValueError):
        qxd.vec_dot_noalloc(host, host, 64, out)
    # the context is intact: a valid call still works
    qxd.vec_dot_noalloc(t[:128], t[:128], 64, out)
    torch.cuda.synchronize()
    assert out.tolist() == [0.0, 0.0]


def test_noalloc_dot_inside_a_captured_graph(qxd):
    """After a first call (which looks up the scratch address), the call records into a CUDA
    graph: the replay reads whatever the captured input buffers hold at replay time."""
    dev = torch.device("cuda:0")
    n = 100_003
    r = np.random.default_rng(7)
    ta = torch.zeros(2 * n, dtype=torch.float64, device=dev)
    tb = torch.zeros(2 * n, dtype=torch.float64, device=dev)
    out = torch.zeros(2, dtype=torch.float64, device=dev)
    qxd.vec_dot_noalloc(ta, tb, n, out, torch.cuda.current_stream(dev).cuda_stream)  # first call
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream(dev)
    side.wait_stream(torch.cuda.current_stream(dev))
    with torch.cuda.stream(side):
        with torch.cuda.graph(g, stream=side):
            qxd.vec_dot_noalloc(ta, tb, n, out, side.cuda_stream)
    torch.cuda.current_stream(dev).wait_stream(side)
    torch.cuda.synchronize()
    for trial in range(3):
        a = r.standard_normal(2 * n)
        b = r.standard_normal(2 * n)
        ta.copy_(torch.from_numpy(a))
        tb.copy_(torch.from_numpy(b))
        g.replay()
        torch.cuda.synchronize()
        got = complex(out[0].item(), out[1].item())
        za, zb = a.view(np.complex128), b.view(np.complex128)
        scale = float(np.sum(np.abs(za) * np.abs(zb)))
        assert abs(got - np.vdot(za, zb)) <= 1e-13 * scale, (trial, got)


def test_noalloc_dot_after_forgetting_the_scratch_address(qxd):
    """qxd_vec_dot_noalloc_forget drops the cached address; the next call looks it up again."""
    dev = torch.device("cuda:0")
    r = np.random.default_rng(3)
    a, b = r.standard_normal(2 * 5000), r.standard_normal(2 * 5000)
    ta, tb = torch.from_numpy(a).to(dev), torch.from_numpy(b).to(dev)
    out = torch.zeros(2, dtype=torch.float64, device=dev)
    qxd.vec_dot_noalloc_forget()
    qxd.vec_dot_noalloc(ta, tb, 5000, out)
    torch.cuda.synchronize()
    za, zb = a.view(np.complex128), b.view(np.complex128)
    got = complex(out[0].item(), out[1].item())
    assert abs(got - np.vdot(za, zb)) <= 1e-13 * float(np.sum(np.abs(za) * np.abs(zb)))
