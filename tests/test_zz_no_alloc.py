"""The allocation-free key-frame entry point (hot_key_frame_noalloc) on the GPU.

Some callers cannot allocate device memory at the point where they need the key
frame -- a host process whose device memory is all handed out up front to a pool
it does not own, or code running where the allocator is not reentrant -- so this
entry point keeps its scratch in a fixed array inside the library.  The test calls
it through the C ABI twice in a row (different inputs, so the second call must not
see the first call's scratch) and compares each result with the frame that
hot_build_tree computes for the same input, bit for bit as the other frame checks
do.  A third input spans 1025 reduction blocks, so the final reduction takes many
partial records per lane; its frame is compared with numpy's exact minimum and
maximum.  It lives in a file of its own that pytest collects last.
"""
import ctypes as C

import numpy as np
import pytest

from paper_1310_4502_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _inputs():
    w = W.make("plummer4096")
    rng = np.random.default_rng(5)
    n = 1 << 18
    x = rng.uniform(-2.0, 3.0, (n, 3)) * np.array([1.0, 0.25, 2.0])
    return [(w.pos, w.mass), (x, rng.uniform(0.5, 1.5, n) / n)]


def test_noalloc_key_frame_matches_build_tree():
    from paper_1310_4502_gb300 import hot
    dev = torch.device("cuda:0")
    results = []
    for pos, mass in _inputs():
        P = torch.tensor(pos, device=dev)
        M = torch.tensor(mass, device=dev)
        h = hot.Hot()
        h.build_tree(P, M)
        ref = h.debug_get("FRAME")
        frame = torch.full((4,), -1.0, dtype=torch.float64, device=dev)
        hot.key_frame_noalloc(P, M, frame)
        torch.cuda.synchronize()
        got = frame.cpu().numpy()
        assert np.array_equal(got, ref), (got, ref)
        results.append(got)
        h.close()
    assert not np.array_equal(results[0], results[1])


def test_noalloc_key_frame_errors():
    from paper_1310_4502_gb300 import hot
    L = hot.load()
    dev = torch.device("cuda:0")
    pos, mass = _inputs()[0]
    P = torch.tensor(pos, device=dev)
    M = torch.tensor(mass, device=dev)
    frame = torch.zeros(4, dtype=torch.float64, device=dev)
    st = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    # beyond the scratch capacity: rejected before any device work
    r = L.hot_key_frame_noalloc(C.c_void_p(P.data_ptr()), C.c_void_p(M.data_ptr()), (1 << 26) + 1,
                                C.c_void_p(frame.data_ptr()), st)
    assert r == hot.HOT_EOVERFLOW
    bad = P.clone()
    bad[17, 2] = float("inf")
    with pytest.raises(hot.HotError) as e:
        hot.key_frame_noalloc(bad, M, frame)
    assert e.value.code == hot.HOT_EINPUT
    # the status word does not leak into the next call
    hot.key_frame_noalloc(P, M, frame)
    h = hot.Hot()
    h.build_tree(P, M)
    assert np.array_equal(frame.cpu().numpy(), h.debug_get("FRAME"))


def test_noalloc_key_frame_many_blocks():
    """N = 2^24 + 1: 1025 partial records (16384 particles each), the last one holding a
    single particle; min and max are exact, so numpy's frame is the bit-exact reference."""
    from paper_1310_4502_gb300 import hot
    dev = torch.device("cuda:0")
    n = (1 << 24) + 1
    rng = np.random.default_rng(6)
    x = rng.standard_normal((n, 3)) * np.array([1.0, 3.0, 0.5])
    x[-1] = [-40.0, 0.0, 25.0]  # the extremes sit in the one-particle last block
    m = np.full(n, 1.0 / n)
    lo = x.min(axis=0)
    ext = (x.max(axis=0) - lo).max()
    ref = np.array([lo[0], lo[1], lo[2], ext])
    P = torch.tensor(x, device=dev)
    M = torch.tensor(m, device=dev)
    frame = torch.full((4,), -1.0, dtype=torch.float64, device=dev)
    for _ in range(2):
        hot.key_frame_noalloc(P, M, frame)
        torch.cuda.synchronize()
        assert np.array_equal(frame.cpu().numpy(), ref), (frame.cpu().numpy(), ref)
        frame.fill_(-1.0)
    with pytest.raises(ValueError):
        hot.key_frame_noalloc(P, M, frame[:3])
    with pytest.raises(ValueError):
        hot.key_frame_noalloc(P[:-1], M, frame)
    del P, M
    torch.cuda.empty_cache()
