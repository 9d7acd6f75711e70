"""A batched shuffle captured in a CUDA graph (with a caller workspace, the call allocates and
copies nothing from the host: the array table travels in kernel parameters) replays exactly:
after refilling the inputs, every replay gives the oracle's output for every array, plan group
fan-out onto the caller's auxiliary streams included.  The call is made once on the capturing
stream first (it creates that stream's auxiliary streams and sets kernel attributes)."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
import paper_2302_03317_gb300 as rip  # noqa: E402


def _oplan(p):
    return oracle.Plan(list(p.ks), list(p.Ts), list(p.Bs), p.base, p.max_levels)


@pytest.mark.parametrize("w", [4, 8])
def test_batched_call_captured_in_a_cuda_graph_replays_exactly(w):
    rng = np.random.default_rng(21)
    sizes = [int(v) for v in np.floor(2.0 ** (8 + 13 * rng.random(40)))] + [1 << 20, 300_001, 5, 1, 0]
    dt = torch.int32 if w == 4 else torch.int64
    bufs = [torch.empty(n, dtype=dt, device="cuda") for n in sizes]
    need = rip.rip_shuffle_batched_workspace_size(sizes, w, None)
    ws = torch.empty(max(need, 256), dtype=torch.uint8, device="cuda")
    ptrs = [b.data_ptr() for b in bufs]
    s = torch.cuda.Stream()

    def fill():
        for b in bufs:
            b.copy_(torch.arange(b.shape[0], dtype=dt, device="cuda"))

    def call(seed):
        rip.rip_shuffle_batched(ptrs, sizes, w, seed, None, ws.data_ptr(), need, s.cuda_stream)

    with torch.cuda.stream(s):
        fill()
        call(7)  # warm-up on the capturing stream
    s.synchronize()
    assert rip.rip_get_device_status(s.cuda_stream) == rip.RIP_OK
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        call(500)
    npdt = np.uint32 if w == 4 else np.uint64
    for rep in range(2):
        fill()
        torch.cuda.synchronize()
        g.replay()
        torch.cuda.synchronize()
        assert rip.rip_get_device_status(0) == rip.RIP_OK
        for i, (b, n) in enumerate(zip(bufs, sizes)):
            want = oracle.shuffle(np.arange(n, dtype=npdt), 500 + i, _oplan(rip.rip_default_plan(n, w)))
            got = b.cpu().numpy().view(npdt)
            assert np.array_equal(got, want), (rep, i, n)
