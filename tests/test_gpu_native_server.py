"""The library's native server (fr_server_create / fr_submit / fr_poll, a
worker thread inside libfacert.so) against the Python continuous-batching
server: the same requests give bitwise the same final parameters and the same
final loss, through every stage of a reconstruction; admission respects the
slot count and the memory cap; requests that cannot be served fail alone."""
import dataclasses

import numpy as np
import pytest

from paper_2101_05356_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _requests(sc, specs, schedule, landmarks=False, stage_geometry=False):
    from oracle import landmarks as olm
    from paper_2101_05356_gb300 import facert, serve
    reqs = []
    for rid, (w, h, spp) in enumerate(specs):
        s2 = dataclasses.replace(sc, width=w, height=h, spp=spp)
        r = facert.Renderer(s2)
        gt = synth.random_params(s2, 70 + rid, coef_scale=0.5)
        init = synth.init_params(sc)
        if stage_geometry:
            gt = synth.with_stage_geometry(s2, gt, seed=rid + 1)
            init = synth.with_stage_geometry(sc, init)
        tgt = r.forward(r.device_params(gt), iteration=10 ** 7, face_id=rid).cpu().numpy()
        r.close()
        lm = olm.project(sc, gt, sc.landmarks, w, h).astype(np.float32) if landmarks else None
        reqs.append(serve.Request(rid=rid, target=tgt, spp=spp, schedule=schedule, init=init, landmarks=lm))
    return reqs


SPECS = [(64, 64, 4), (48, 40, 2), (64, 48, 8)]
KW = dict(max_width=64, max_height=64, max_spp=8)


def _compare(native, python, names):
    for got, ref in zip(native, python):
        assert got.failed is None and ref.failed is None
        assert got.native_id == ref.rid
        assert got.final_loss == pytest.approx(ref.final_loss, rel=1e-12)
        for n in names:
            a, b = got.params[n], np.asarray(ref.params[n]).reshape(got.params[n].shape)
            assert np.array_equal(a, b), (ref.rid, n, float(np.abs(a.astype(np.float64) - b).max()))


def test_full_pipeline_matches_the_python_server():
    """Landmark initialisation, Stage I with the statistical albedo (batched
    morph and transpose) and the landmark term, Stage II: three requests of
    different sizes and sample counts in one native batch against the Python
    server's."""
    from paper_2101_05356_gb300 import optim, serve
    sc = synth.make_scene("c1", albedo_k=8)
    sched = optim.Schedule(stage1=3, stage2=2, init=2)
    ref = serve.Server(sc, max_slots=4, **KW).run(_requests(sc, SPECS, sched, landmarks=True))
    ns = serve.NativeServer(sc, max_slots=3, **KW)
    try:
        got = ns.run(_requests(sc, SPECS, sched, landmarks=True))
        assert ns.stats["max_active"] >= 2
    finally:
        ns.close()
    _compare(got, ref, ("coef", "rot", "trans", "focal", "light_i", "diffuse", "specular", "roughness"))


def test_light_stage_geometry_matches_the_python_server():
    """Stage I with the virtual light stage's geometry (d, a, p) free."""
    from paper_2101_05356_gb300 import optim, serve
    sc = synth.make_scene("tiny", light_stage="ico")
    specs = [(24, 24, 2), (20, 16, 4)]
    sched = optim.Schedule(stage1=4, stage2=1)
    ref = serve.Server(sc, max_slots=2, max_width=24, max_height=24, max_spp=4).run(
        _requests(sc, specs, sched, stage_geometry=True))
    ns = serve.NativeServer(sc, max_slots=2, max_width=24, max_height=24, max_spp=4)
    try:
        got = ns.run(_requests(sc, specs, sched, stage_geometry=True))
    finally:
        ns.close()
    _compare(got, ref, ("coef", "rot", "trans", "light_i", "light_d", "light_a", "light_p", "diffuse"))
    assert not np.array_equal(got[0].params["light_d"], synth.with_stage_geometry(sc, synth.init_params(sc)).light_d)


def test_slots_and_memory_cap_bound_admission():
    from paper_2101_05356_gb300 import optim, serve
    sc = synth.make_scene("c1")
    sched = optim.Schedule(2, 1)
    specs = [(64, 64, 4)] * 4
    one = serve.NativeServer(sc, max_slots=4, mem_cap_bytes=1, **KW)     # only the first fits at a time
    try:
        reqs = one.run(_requests(sc, specs, sched))
        assert one.stats["max_active"] == 1 and all(r.final_loss is not None for r in reqs)
        single = one.stats["peak_bytes"]
    finally:
        one.close()
    two = serve.NativeServer(sc, max_slots=2, mem_cap_bytes=int(2.5 * single), **KW)
    try:
        two.run(_requests(sc, specs, sched))
        assert two.stats["max_active"] == 2 and two.stats["peak_bytes"] <= 2.5 * single
    finally:
        two.close()


def test_requests_that_cannot_run_fail_alone():
    from paper_2101_05356_gb300 import optim, serve
    sc = synth.make_scene("c1")
    sched = optim.Schedule(1, 1)
    reqs = _requests(sc, [(64, 64, 4), (32, 32, 2), (32, 32, 2)], sched)
    reqs[0].target = np.zeros((128, 128, 3), np.float32)          # above the server's image size
    reqs[2].spp = 16                                              # above the server's sample count
    ns = serve.NativeServer(sc, max_slots=2, **KW)
    try:
        ns.run(reqs)
    finally:
        ns.close()
    assert "larger" in reqs[0].failed and "spp" in reqs[2].failed
    assert reqs[1].failed is None and np.isfinite(reqs[1].final_loss)


def test_a_request_without_iterations_is_evaluated_at_its_initial_parameters():
    from paper_2101_05356_gb300 import optim, serve
    sc = synth.make_scene("c1")
    reqs = _requests(sc, [(32, 32, 2), (32, 32, 2)], optim.Schedule(0, 0))
    reqs[1].schedule = optim.Schedule(1, 0)
    ns = serve.NativeServer(sc, max_slots=2, **KW)
    try:
        got = ns.run(reqs)
    finally:
        ns.close()
    ref = serve.Server(sc, max_slots=2, **KW).run(_requests(sc, [(32, 32, 2), (32, 32, 2)], optim.Schedule(0, 0))[:1])
    init = synth.init_params(sc)
    for n in ("coef", "rot", "trans", "diffuse"):
        assert np.array_equal(got[0].params[n], np.asarray(getattr(init, n), np.float32).reshape(got[0].params[n].shape))
        assert np.array_equal(ref[0].params[n].reshape(got[0].params[n].shape), got[0].params[n])
    assert got[0].final_loss == pytest.approx(ref[0].final_loss, rel=1e-12)
    assert not np.array_equal(got[1].params["coef"], got[0].params["coef"])


def test_cancelled_and_non_finite_requests_fail_alone():
    """Host-side faults: a request cancelled while queued, one cancelled while
    running, and one with NaN initial parameters (its final loss is not
    finite) each fail with their reason; the others' results are bitwise
    those of the Python server."""
    import time
    from paper_2101_05356_gb300 import facert, optim, serve
    sc = synth.make_scene("c1")
    specs = [(32, 32, 2)] * 5
    sched = optim.Schedule(3, 1)
    reqs = _requests(sc, specs, sched)
    reqs[2].init.coef[0] = np.nan
    reqs[3].schedule = optim.Schedule(400, 0)            # long enough to be cancelled while running
    ns = serve.NativeServer(sc, max_slots=1, **KW)
    try:
        ids = [facert.fr_submit(ns.srv, q.target, q.init, q.spp, q.schedule.stage1, q.schedule.stage2)
               for q in reqs]
        assert facert.fr_cancel(ns.srv, ids[1])           # queued behind request 0 (one slot)
        t0 = time.time()
        while facert.fr_poll(ns.srv, ids[3])[1]["iterations"] < 1 and time.time() - t0 < 120:
            time.sleep(0.002)
        assert facert.fr_cancel(ns.srv, ids[3])
        assert facert.fr_server_wait(ns.srv, 600.0)
        res = [facert.fr_poll(ns.srv, i, ns._shapes(q.init)) for i, q in zip(ids, reqs)]
        stats = facert.fr_server_get_stats(ns.srv)
        assert not facert.fr_cancel(ns.srv, ids[0])       # already done
    finally:
        ns.close()
    assert res[1][1]["state"] == facert.REQ_FAILED and res[1][1]["error"] == "cancelled"
    assert res[1][1]["iterations"] == 0
    assert res[2][1]["state"] == facert.REQ_FAILED and "finite" in res[2][1]["error"]
    assert res[3][1]["state"] == facert.REQ_FAILED and res[3][1]["error"] == "cancelled"
    assert 0 < res[3][1]["iterations"] < 400
    assert stats["active"] == 0 and stats["queued"] == 0
    ok = [0, 4]
    ref = serve.Server(sc, max_slots=1, **KW).run([_requests(sc, specs, sched)[k] for k in ok])
    for k, rr in zip(ok, ref):
        done, r, params = res[k]
        assert done and r["state"] == facert.REQ_DONE
        assert r["final_loss"] == pytest.approx(rr.final_loss, rel=1e-12)
        for n in ("coef", "rot", "trans", "light_i", "diffuse"):
            assert np.array_equal(params[n], np.asarray(rr.params[n]).reshape(params[n].shape)), (k, n)


def test_bounded_wait_reports_timeout_and_the_context_stays_usable():
    """A device wait that nothing satisfies gives up after its poll limit and
    reports through the status word (FR_ETIMEOUT, then cleared); renders on
    the same context afterwards are unchanged."""
    from paper_2101_05356_gb300 import facert
    sc = synth.make_scene("tiny")
    r = facert.Renderer(sc, flags=facert.FLAG_MORPH_BF16)
    dp = r.device_params(synth.random_params(sc, 2))
    before = r.forward(dp, iteration=5)
    facert.fr_debug_wait_timeout(r.ctx, 1 << 12)
    assert facert.fr_sync_status(r.ctx) == facert.FR_ETIMEOUT
    assert r.status() == 0                               # read and cleared
    after = r.forward(dp, iteration=5)
    torch.cuda.synchronize()
    assert torch.equal(before, after)
    assert r.status() == 0


def test_results_are_the_same_alone_and_in_a_batch_of_40():
    """40 requests advanced together (the tensor-core morph then runs one
    64-wide MMA over the batch) against the same requests served alone
    (a 32-wide MMA): each result is bitwise the same."""
    from paper_2101_05356_gb300 import optim, serve
    sc = synth.make_scene("tiny")
    specs = [(24, 24, 2)] * 40
    sched = optim.Schedule(4, 2)        # long enough for all 40 to be admitted while the first still runs
    kw = dict(max_width=24, max_height=24, max_spp=2)
    ns = serve.NativeServer(sc, max_slots=40, mem_cap_bytes=1 << 40, **kw)
    try:
        got = ns.run(_requests(sc, specs, sched))
        assert ns.stats["max_active"] > 32
    finally:
        ns.close()
    for k in (0, 17, 39):
        lone = serve.NativeServer(sc, max_slots=1, **kw)
        try:
            req = _requests(sc, specs, sched)
            ref = lone.run(req[:k + 1])[k]          # ids 0..k so that request k keeps its face id
        finally:
            lone.close()
        assert got[k].final_loss == ref.final_loss
        for n in ("coef", "rot", "trans", "light_i", "diffuse", "specular", "roughness"):
            assert np.array_equal(got[k].params[n], ref.params[n]), (k, n)


def test_a_failed_result_read_fails_only_the_unread_requests():
    """Host-side fault in the retirement of a step: three requests finish in the
    same step and the third device-to-host read (the second request's final
    loss) is made to fail on the host.  The first request keeps its result
    (bitwise the Python server's); the other two fail with the read's message;
    every request is counted once and the admitted-state bytes return to zero
    (a request retired before the failure is not released a second time)."""
    from paper_2101_05356_gb300 import facert, optim, serve
    sc = synth.make_scene("c1")
    specs = [(32, 32, 2)] * 3
    sched = optim.Schedule(2, 1)
    reqs = _requests(sc, specs, sched)
    ns = serve.NativeServer(sc, max_slots=3, **KW)
    try:
        # reads of a retiring request: its final loss, then its parameters
        facert.fr_server_inject_read_failure(ns.srv, 2)
        ids = [facert.fr_submit(ns.srv, q.target, q.init, q.spp, q.schedule.stage1, q.schedule.stage2)
               for q in reqs]
        assert facert.fr_server_wait(ns.srv, 600.0)
        res = [facert.fr_poll(ns.srv, i, ns._shapes(q.init)) for i, q in zip(ids, reqs)]
        stats = facert.fr_server_get_stats(ns.srv)
    finally:
        ns.close()
    assert res[0][1]["state"] == facert.REQ_DONE
    for k in (1, 2):
        assert res[k][1]["state"] == facert.REQ_FAILED
        assert res[k][1]["error"] == "reading a final loss failed"
    assert stats["finished"] == 3
    assert stats["used_bytes"] == 0
    assert stats["active"] == 0 and stats["queued"] == 0
    ref = serve.Server(sc, max_slots=3, **KW).run(_requests(sc, specs, sched))
    assert res[0][1]["final_loss"] == pytest.approx(ref[0].final_loss, rel=1e-12)
    for n in ("coef", "rot", "trans", "light_i", "diffuse"):
        assert np.array_equal(res[0][2][n], np.asarray(ref[0].params[n]).reshape(res[0][2][n].shape)), n
