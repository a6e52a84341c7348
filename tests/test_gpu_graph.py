"""The fused step (fr_render: forward, loss and adjoint) enqueues only kernels
and asynchronous memory operations on the caller's stream, so it can be
recorded once into a CUDA graph and replayed; each replay equals the eager call
with the same arguments bit for bit."""
import numpy as np
import pytest

from paper_2101_05356_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("name", ["c1", "ico"])
def test_fused_step_replays_from_a_cuda_graph(name):
    from paper_2101_05356_gb300 import facert
    sc = synth.make_scene("c1") if name == "c1" else synth.make_scene("tiny", light_stage="ico")
    r = facert.Renderer(sc)
    pr = synth.random_params(sc, 4)
    if name == "ico":
        pr = synth.with_stage_geometry(sc, pr, seed=2)
    dp = r.device_params(pr)
    tgt = r.forward(dp, iteration=9) * 0.9
    img_e, loss_e, g_e = r.render(dp, tgt, iteration=2)
    torch.cuda.synchronize()

    img = r.image_buffer()
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    g = r.zero_grads(dp)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):                       # warm up outside the capture
        facert.fr_render(r.ctx, dp, tgt, img, loss, g, 2, 0)
    torch.cuda.current_stream().wait_stream(side)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        for t in g.values():
            t.zero_()
        facert.fr_render(r.ctx, dp, tgt, img, loss, g, 2, 0)
    for _ in range(2):
        img.zero_()
        loss.zero_()
        graph.replay()
        torch.cuda.synchronize()
        assert torch.equal(img, img_e)
        assert torch.equal(loss, loss_e)
        for k in g_e:
            assert torch.equal(g[k], g_e[k]), k
    assert r.status() == 0
