"""im_argmax_noalloc: the estimate + argmax entry point that allocates nothing.

Some callers cannot allocate device memory: code that runs inside a memory
arena it does not own, or a process that reserved all device memory up front,
where a cudaMalloc would fail or stall the whole device.  For them the library
offers im_argmax_noalloc, which keeps its scratch in a static device array and
takes every input and output as caller-owned device memory.  These tests call
it through the C ABI, on two calls in a row (the second with the first pick
excluded), and check it against the oracle's sums and pick on the same
registers and against the allocating entry point (im_sketch_pick): on sketches
of a real graph at J = 16, 256 and 1024, and on register matrices large enough
that the kernel runs the largest grid the static array is sized for.  The file
is collected last.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2410_14047_gb300 as im
    return torch, im, im.load_library()


def _device_buffers(torch, M, n):
    dev = torch.device("cuda", 0)
    M_dev = torch.from_numpy(np.ascontiguousarray(M).reshape(-1)).to(dev)
    picked = torch.zeros((n + 31) // 32, dtype=torch.int32, device=dev)
    s_dev = torch.full((1,), -7, dtype=torch.int32, device=dev)
    S_dev = torch.zeros(1, dtype=torch.int64, device=dev)
    est_dev = torch.zeros(1, dtype=torch.float64, device=dev)
    return M_dev, picked, s_dev, S_dev, est_dev


def _two_calls(torch, im, L, M, J, sketch=None):
    """Two calls in a row; each pick checked against the oracle (and against
    im_sketch_pick when a sketch holds the same registers)."""
    n = M.shape[0]
    S = O.sums(M)
    M_dev, picked, s_dev, S_dev, est_dev = _device_buffers(torch, M, n)
    stream = torch.cuda.current_stream(torch.device("cuda", 0)).cuda_stream
    is_seed = np.zeros(n, np.uint8)
    got = []
    for _ in range(2):
        st = L.im_argmax_noalloc(M_dev.data_ptr(), n, J, picked.data_ptr(), stream,
                                 s_dev.data_ptr(), S_dev.data_ptr(), est_dev.data_ptr())
        assert st == 0, im.STATUS.get(st, st)
        torch.cuda.synchronize()
        s = int(s_dev.item())
        want = O.pick(S, is_seed)
        assert s == want
        assert int(S_dev.item()) & 0xFFFFFFFFFFFFFFFF == int(S[s])
        assert float(est_dev.item()) == pytest.approx(O.estimate(J, int(S[s])), rel=1e-12)
        if sketch is not None:
            s_ref, S_ref, est_ref = sketch.pick()  # the allocating entry point
            assert (s_ref, S_ref) == (s, int(S[s]))
            assert est_ref == pytest.approx(float(est_dev.item()), rel=1e-12)
        is_seed[s] = 1
        got.append(s)
    # exactly the two picks are marked excluded
    bits = picked.cpu().numpy().view(np.uint32)
    marked = np.nonzero(np.unpackbits(bits.view(np.uint8), bitorder="little")[:n])[0].tolist()
    assert marked == sorted(got)
    return got


@pytest.mark.parametrize("J", [16, 256, 1024])
def test_argmax_noalloc_matches_oracle_and_allocating_pick(env, J):
    torch, im, L = env
    g = W.rmat(12, 16, seed=5)
    ctx = im.im_ctx_create(0)
    G = im.im_graph_load(ctx, g.rowptr, g.col, {"kind": "wc"})
    sk = im.im_sketch_build(G, J, 31)
    _two_calls(torch, im, L, sk.registers(), J, sketch=sk)


def _random_registers(n, J, seed):
    """Ranks distributed like clz of a uniform hash, some visited registers,
    and the best row copied to a higher and a lower id (ties: lowest id)."""
    rng = np.random.default_rng(seed)
    M = np.minimum(rng.geometric(0.5, size=(n, J)) - 1, 32).astype(np.uint8)
    M[rng.random((n, J)) < 0.05] = 0xFF
    S = O.sums(M)
    best = int(np.argmin(S))
    M[n - 1] = M[best]
    M[n // 3] = M[best]
    return M


@pytest.mark.parametrize("n,J", [(1 << 20, 16), (50_000, 1024), (200_000, 256)])
def test_argmax_noalloc_at_the_largest_grid(env, n, J):
    # 1 << 20 rows at J = 16 (512 rows a block), 50,000 rows at J = 1024 (32)
    # and 200,000 rows at J = 256 (128) all need more than the 1216 blocks the
    # static array holds partials for: the grid is capped there and the
    # blocks stride over the rest
    torch, im, L = env
    M = _random_registers(n, J, seed=n + J)
    got = _two_calls(torch, im, L, M, J)
    S = O.sums(M)
    assert S[got[0]] == S[got[1]] == S.min()  # tied rows: lowest ids first


def test_argmax_noalloc_rejects_bad_arguments(env):
    torch, im, L = env
    dev = torch.device("cuda", 0)
    buf = torch.zeros(64, dtype=torch.int64, device=dev)
    p = buf.data_ptr()
    assert L.im_argmax_noalloc(p, 1 << 26, 64, p, None, p, p, p) == -2  # n too large
    assert L.im_argmax_noalloc(p, 0, 64, p, None, p, p, p) == -2        # n too small
    assert L.im_argmax_noalloc(p, 10, 48, p, None, p, p, p) == -1       # unsupported J
    assert L.im_argmax_noalloc(None, 10, 64, p, None, p, p, p) == -1    # NULL input
    # below their alignment (refused on the host, nothing is launched)
    assert L.im_argmax_noalloc(p + 8, 10, 64, p, None, p, p, p) == -1   # registers: 16 bytes
    assert L.im_argmax_noalloc(p, 10, 64, p + 2, None, p, p, p) == -1   # picked words: 4
    assert L.im_argmax_noalloc(p, 10, 64, p, None, p + 1, p, p) == -1   # s_out: 4
    assert L.im_argmax_noalloc(p, 10, 64, p, None, p, p + 4, p) == -1   # S_out: 8
    assert L.im_argmax_noalloc(p, 10, 64, p, None, p, p, p + 4) == -1   # est_out: 8
    torch.cuda.synchronize()
