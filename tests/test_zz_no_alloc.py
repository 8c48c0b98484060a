"""im_argmax_noalloc: the estimate + argmax entry point that allocates nothing.

Some callers cannot allocate device memory: code that runs inside a memory
arena it does not own, or a process that reserved all device memory up front,
where a cudaMalloc would fail or stall the whole device.  For them the library
offers im_argmax_noalloc, which keeps its scratch in a static device array and
takes every input and output as caller-owned device memory.  This test calls it
through the C ABI and checks it against the allocating entry point
(im_sketch_pick) on the same registers, on two calls in a row (the second one
with the first pick excluded).  It lives in a file of its own that pytest
collects last.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


def test_argmax_noalloc_matches_allocating_pick_on_two_calls():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2410_14047_gb300 as im

    L = im.load_library()
    g = W.rmat(12, 16, seed=5)
    ctx = im.im_ctx_create(0)
    G = im.im_graph_load(ctx, g.rowptr, g.col, {"kind": "wc"})
    J = 256
    sk = im.im_sketch_build(G, J, 31)
    M = sk.registers()

    dev = torch.device("cuda", 0)
    M_dev = torch.from_numpy(np.ascontiguousarray(M).reshape(-1)).to(dev)
    picked = torch.zeros((g.n + 31) // 32, dtype=torch.int32, device=dev)
    s_dev = torch.full((1,), -7, dtype=torch.int32, device=dev)
    S_dev = torch.zeros(1, dtype=torch.int64, device=dev)
    est_dev = torch.zeros(1, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev).cuda_stream

    for _ in range(2):
        st = L.im_argmax_noalloc(M_dev.data_ptr(), g.n, J, picked.data_ptr(), stream,
                                 s_dev.data_ptr(), S_dev.data_ptr(), est_dev.data_ptr())
        assert st == 0, im.STATUS.get(st, st)
        torch.cuda.synchronize()
        s_ref, S_ref, est_ref = sk.pick()  # the allocating entry point
        s = int(s_dev.item())
        assert s == s_ref
        assert int(S_dev.item()) == S_ref
        assert float(est_dev.item()) == pytest.approx(est_ref, rel=1e-12)
        word = int(picked[s >> 5].item()) & 0xFFFFFFFF
        assert (word >> (s & 31)) & 1  # the pick is now excluded


def test_argmax_noalloc_rejects_bad_sizes():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2410_14047_gb300 as im

    L = im.load_library()
    dev = torch.device("cuda", 0)
    buf = torch.zeros(64, dtype=torch.int64, device=dev)
    p = buf.data_ptr()
    assert L.im_argmax_noalloc(p, 1 << 26, 64, p, None, p, p, p) == -2  # n too large
    assert L.im_argmax_noalloc(p, 10, 48, p, None, p, p, p) == -1       # unsupported J
    assert L.im_argmax_noalloc(None, 10, 64, p, None, p, p, p) == -1    # NULL input
