"""Continuous-batching server: a request's result is the same alone and in a
mixed batch; admission respects the slot count and the memory cap; a request
that cannot be served fails alone."""
import numpy as np
import pytest

from paper_2101_05356_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _requests(sc, specs, schedule, landmarks=False):
    from paper_2101_05356_gb300 import facert, serve
    from oracle import landmarks as olm
    reqs = []
    for rid, (w, h, spp, arrival) in enumerate(specs):
        import dataclasses
        s2 = dataclasses.replace(sc, width=w, height=h, spp=spp)
        r = facert.Renderer(s2)
        gt = synth.random_params(s2, 50 + rid, coef_scale=0.5)
        tgt = r.forward(r.device_params(gt), iteration=10 ** 7, face_id=rid).cpu().numpy()
        r.close()
        lm = olm.project(sc, gt, sc.landmarks, w, h).astype(np.float32) if landmarks else None
        reqs.append(serve.Request(rid=rid, target=tgt, spp=spp, schedule=schedule, arrival=arrival,
                                  init=synth.init_params(sc), landmarks=lm))
    return reqs


SPECS = [(64, 64, 4, 0.0), (48, 40, 2, 0.0), (64, 48, 8, 0.0)]


def test_each_result_is_the_same_alone_and_in_the_mix():
    """Each request of a mixed batch (sizes 64x64/4 spp, 48x40/2 spp, 64x48/8 spp)
    against the same request served alone.

    Images and Philox streams do not depend on the batch, and every gradient sum
    is kept in 64-bit fixed point (order-independent), so the final parameters
    must be bitwise identical; the reported loss is an FP64 sum of block partials
    in launch order and must agree to 1e-12."""
    from paper_2101_05356_gb300 import optim, serve
    sc = synth.make_scene("c1")
    sched = optim.Schedule(3, 2)
    all_reqs = _requests(sc, SPECS, sched)
    mixed = serve.Server(sc, max_slots=4, max_width=64, max_height=64, max_spp=8).run(all_reqs)
    for k in range(len(SPECS)):
        lone_req = _requests(sc, SPECS, sched)[k]
        ref = serve.Server(sc, max_slots=1, max_width=64, max_height=64, max_spp=8).run([lone_req])[0]
        got = mixed[k]
        assert got.rid == ref.rid == k
        assert got.final_loss == pytest.approx(ref.final_loss, rel=1e-12)
        for name in ("coef", "rot", "trans", "focal", "light_i", "diffuse", "specular", "roughness"):
            a, b = got.params[name], ref.params[name]
            assert np.array_equal(a, b), (k, name, float(np.abs(a.astype(np.float64) - b).max()))


def test_full_pipeline_is_the_same_alone_and_in_the_mix():
    """The same with every stage of a reconstruction: landmark initialisation,
    Stage I with the statistical albedo (batched tensor-core morph and its
    transpose) and the landmark term, Stage II."""
    from paper_2101_05356_gb300 import optim, serve
    sc = synth.make_scene("c1", albedo_k=8)
    sched = optim.Schedule(stage1=3, stage2=2, init=2)
    mixed = serve.Server(sc, max_slots=4, max_width=64, max_height=64, max_spp=8).run(
        _requests(sc, SPECS, sched, landmarks=True))
    for k in range(len(SPECS)):
        lone_req = _requests(sc, SPECS, sched, landmarks=True)[k]
        ref = serve.Server(sc, max_slots=1, max_width=64, max_height=64, max_spp=8).run([lone_req])[0]
        got = mixed[k]
        assert got.final_loss == pytest.approx(ref.final_loss, rel=1e-12)
        for name in ("coef", "rot", "trans", "light_i", "diffuse", "specular", "roughness"):
            assert np.array_equal(got.params[name], ref.params[name]), (k, name)


def test_memory_cap_and_slots_bound_admission():
    from paper_2101_05356_gb300 import optim, serve
    sc = synth.make_scene("c1")
    sched = optim.Schedule(2, 1)
    specs = [(64, 64, 4, 0.0)] * 4
    tight = serve.Server(sc, max_slots=4, max_width=64, max_height=64, max_spp=8)
    one = tight.state_bytes(_requests(sc, specs[:1], sched)[0])
    tight.mem_cap = int(1.5 * one)                    # room for one request at a time
    tight.run(_requests(sc, specs, sched))
    assert max(tight.batch_sizes) == 1 and len(tight.done) == 4
    roomy = serve.Server(sc, max_slots=2, max_width=64, max_height=64, max_spp=8)
    roomy.run(_requests(sc, specs, sched))
    assert max(roomy.batch_sizes) == 2 and len(roomy.done) == 4


def test_oversize_request_fails_alone():
    from paper_2101_05356_gb300 import optim, serve
    sc = synth.make_scene("c1")
    sched = optim.Schedule(1, 1)
    reqs = _requests(sc, [(64, 64, 4, 0.0), (32, 32, 2, 0.0)], sched)
    reqs[0].target = np.zeros((128, 128, 3), np.float32)     # bigger than the server's maximum
    srv = serve.Server(sc, max_slots=2, max_width=64, max_height=64, max_spp=8)
    srv.run(reqs)
    assert reqs[0].failed and reqs[0].final_loss is None
    assert reqs[1].failed is None and reqs[1].final_loss is not None
