"""Serving (gdpm_request_submit / gdpm_request_poll): requests run side by
side with continuous admission; a request's result does not depend on what
else runs (its Philox stream is its own), and equals gdpm_simulate's."""
import time

import numpy as np
import pytest

from paper_1107_3355_gb300 import gdpm as G
from paper_1107_3355_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def wait(ctx, rid, V, timeout=120.0):
    d = torch.empty(V, dtype=torch.float64, device="cuda")
    s = torch.empty(V, dtype=torch.float64, device="cuda")
    t0 = time.time()
    while True:
        done, st = G.gdpm_request_poll(ctx, rid, d, s)
        if done:
            return d.cpu().numpy(), s.cpu().numpy(), st
        assert time.time() - t0 < timeout
        time.sleep(0.001)


def test_request_alone_equals_in_mix_and_simulate():
    prob = W.slab_photon_problem(n_histories=200_000, n_batches=10, shape=(64, 64, 128))
    eng = G.Engine(prob)
    V = prob.phantom.n_voxels
    try:
        # the same calculation through gdpm_simulate with the same stream id
        G.gdpm_set_param(eng.ctx, G.GDPM_PARAM_REQUEST_ID, 77)
        d_sim, s_sim, st_sim = eng.run()
        d_sim = d_sim.cpu().numpy()
        # alone
        rid = G.gdpm_request_submit(eng.ctx, eng.phantom, eng.tables, prob.source, 200_000, 10,
                                    stream_id=77)
        d_alone, s_alone, st_alone = wait(eng.ctx, rid, V)
        # in a mix with other requests submitted around it
        others = []
        ph = prob.phantom
        for k in range(6):
            src = W.single_beamlet(ph, 45.0 * k, -1.0, -1.0, 2.0) if k % 2 else prob.source
            others.append(G.gdpm_request_submit(eng.ctx, eng.phantom, eng.tables, src,
                                                100_000 * (k + 1), 10))
        rid2 = G.gdpm_request_submit(eng.ctx, eng.phantom, eng.tables, prob.source, 200_000, 10,
                                     stream_id=77)
        others.append(G.gdpm_request_submit(eng.ctx, eng.phantom, eng.tables, prob.source,
                                            300_000, 10))
        d_mix, s_mix, st_mix = wait(eng.ctx, rid2, V)
        for r in others:
            wait(eng.ctx, r, V)
    finally:
        eng.close()
    tol = dict(rtol=1e-9, atol=1e-12 * d_sim.max())
    np.testing.assert_allclose(d_alone, d_sim, **tol)
    np.testing.assert_allclose(d_mix, d_alone, **tol)
    np.testing.assert_allclose(s_mix, s_alone, rtol=1e-6, atol=1e-9 * s_alone.max())
    for k in ("compton", "el_steps", "moller", "brems", "n_primary"):
        assert st_mix[k] == st_alone[k] == st_sim[k], k


def test_many_requests_complete_with_few_slots():
    prob = W.tiny_problem(n_histories=20_000, n_batches=4)
    eng = G.Engine(prob)
    try:
        G.gdpm_set_param(eng.ctx, G.GDPM_PARAM_SERVE_SLOTS, 2)
        ids = [G.gdpm_request_submit(eng.ctx, eng.phantom, eng.tables, prob.source, 5_000 + 1000 * k, 4)
               for k in range(12)]
        V = prob.phantom.n_voxels
        for k, rid in enumerate(ids):
            d, s, st = wait(eng.ctx, rid, V)
            assert st["n_primary"] == 5_000 + 1000 * k
            bal = st["deposited"] + st["escaped"] + st["discarded"]
            assert abs(bal - st["source_energy"]) <= 1e-6 * st["source_energy"]
        with pytest.raises(G.GdpmError):
            G.gdpm_request_poll(eng.ctx, ids[0])          # already released
    finally:
        eng.close()


def test_request_that_can_never_fit_is_refused():
    """Admission: a request whose workspace plus the reserve exceeds the
    device's memory is refused with GDPM_E_NOMEM instead of waiting."""
    prob = W.tiny_problem(n_histories=20_000, n_batches=10)
    eng = G.Engine(prob)
    V = prob.phantom.n_voxels
    try:
        G.gdpm_set_param(eng.ctx, G.GDPM_PARAM_SERVE_RESERVE_MB, 1e7)   # 10 TB kept free
        rid = G.gdpm_request_submit(eng.ctx, eng.phantom, eng.tables, prob.source, 20_000, 10)
        with pytest.raises(G.GdpmError) as e:
            wait(eng.ctx, rid, V)
        assert e.value.code == G.GDPM_E_NOMEM
        # the context still serves once the reserve is sane again
        G.gdpm_set_param(eng.ctx, G.GDPM_PARAM_SERVE_RESERVE_MB, 1024)
        rid = G.gdpm_request_submit(eng.ctx, eng.phantom, eng.tables, prob.source, 20_000, 10)
        d, _, st = wait(eng.ctx, rid, V)
        assert st["n_primary"] == 20_000 and d.max() > 0
    finally:
        eng.close()


def test_submit_and_poll_from_several_threads():
    """gdpm_request_submit / gdpm_request_poll are the thread-safe calls of a
    context: four host threads each submit and poll three requests at once,
    and every result equals gdpm_simulate with the same stream id."""
    import threading
    prob = W.tiny_problem(n_histories=50_000, n_batches=10)
    eng = G.Engine(prob)
    V = prob.phantom.n_voxels
    ids = [100 + 10 * t + j for t in range(4) for j in range(3)]
    try:
        ref = {}
        for sid in ids:
            G.gdpm_set_param(eng.ctx, G.GDPM_PARAM_REQUEST_ID, sid)
            d, _, _ = eng.run()
            ref[sid] = d.cpu().numpy()
        G.gdpm_set_param(eng.ctx, G.GDPM_PARAM_REQUEST_ID, 0)
        results, errors = {}, []

        def worker(t):
            try:
                for j in range(3):
                    sid = 100 + 10 * t + j
                    rid = G.gdpm_request_submit(eng.ctx, eng.phantom, eng.tables, prob.source, 50_000,
                                                10, stream_id=sid)
                    d, s = np.empty(V), np.empty(V)
                    t0 = time.time()
                    while True:
                        done, _ = G.gdpm_request_poll(eng.ctx, rid, d, s)
                        if done:
                            break
                        if time.time() - t0 > 120:
                            raise TimeoutError(sid)
                        time.sleep(0.0005)
                    results[sid] = d
            except Exception as e:                      # reported below, on the main thread
                errors.append(e)

        threads = [threading.Thread(target=worker, args=(t,)) for t in range(4)]
        for th in threads:
            th.start()
        for th in threads:
            th.join(timeout=300)
        assert not any(th.is_alive() for th in threads)
    finally:
        eng.close()
    assert not errors, errors
    assert sorted(results) == sorted(ids)
    for sid in ids:
        np.testing.assert_allclose(results[sid], ref[sid], rtol=1e-9, atol=1e-12 * ref[sid].max())


def test_served_vmat_arc_matches_the_oracle_history_by_history():
    """A short VMAT arc (6 control points 2 degrees apart, MLC apertures from
    seeded leaf positions, Sec. 2.3 and Sec. 3.2) served through
    gdpm_request_submit among other requests, on the patient-like phantom:
    with its stream id as the oracle's request id, the same histories on both
    sides -- per-history event records, the Sec. 3.1 t-test and the signed
    bias over tissue-like voxels."""
    from oracle import oracle as O
    from tests._stats import BIAS_GATE, t_test
    ph = W.ct_phantom(shape=(64, 64, 32), voxel=(1.0, 1.0, 1.0))
    arc = W.vmat_arc(ph, n_points=6, seed=5)
    prob = W.Problem(ph, arc, 30_000, 10, eabs_photon=0.05, eabs_electron=0.2, e_min=0.005,
                     e_max=6.5, request_id=4242)
    d_o, s_o, led_o, rec_o, _ = O.run(prob, per_history=True)
    eng = G.Engine(prob.with_(request_id=0))
    V = ph.n_voxels
    try:
        rec = torch.zeros(prob.n_histories * 4, dtype=torch.int32, device="cuda")
        recd = torch.zeros(prob.n_histories * 2, dtype=torch.float64, device="cuda")
        others = [G.gdpm_request_submit(eng.ctx, eng.phantom, eng.tables,
                                        W.single_beamlet(ph, 90.0 * k, -2.0, 1.0, 1.0), 50_000, 10)
                  for k in range(3)]
        rid = G.gdpm_request_submit(eng.ctx, eng.phantom, eng.tables, arc, prob.n_histories, 10,
                                    stream_id=4242)
        d_g, s_g, st = wait(eng.ctx, rid, V)
        for r in others:
            wait(eng.ctx, r, V)
        # the same request through gdpm_simulate with per-history records
        G.gdpm_set_param(eng.ctx, G.GDPM_PARAM_REQUEST_ID, 4242)
        G.gdpm_set_history_records(eng.ctx, rec, recd, prob.n_histories)
        d_r, _, _ = eng.run()
        G.gdpm_set_history_records(eng.ctx, None, None, 0)
        rec_g = rec.cpu().numpy().reshape(-1, 4)
        d_r = d_r.cpu().numpy()
    finally:
        eng.close()
    np.testing.assert_allclose(d_g, d_r, rtol=1e-9, atol=1e-12 * d_r.max())   # served = simulate
    same = np.all(rec_o == rec_g, axis=1)
    print("served VMAT arc identical records: %.5f" % same.mean())
    assert same.mean() > 0.97
    assert st["n_primary"] == prob.n_histories
    assert st["source_energy"] == pytest.approx(led_o["source_energy"], rel=1e-6)
    r = t_test(d_o, s_o, d_g, s_g, high_frac=0.1, mask=ph.rho >= 0.05)
    print("served VMAT arc t-test", r)
    assert r["P_high"] >= 0.95 and r["P_all"] >= 0.97
    assert abs(r["bias"]) <= BIAS_GATE


@pytest.mark.parametrize("big,share,cap", [(2, 6, 0), (1, 8, 1 << 20)])
def test_serving_layouts_keep_results(big, share, cap):
    """Two slots for large requests, another SM share while small requests
    run, a phase cap for served requests: each changes when the work runs,
    never what it computes -- a request equals gdpm_simulate with its stream
    id, in a mix of large and small requests."""
    prob = W.slab_photon_problem(n_histories=300_000, n_batches=10, shape=(64, 64, 128))
    eng = G.Engine(prob)
    V = prob.phantom.n_voxels
    try:
        G.gdpm_set_param(eng.ctx, G.GDPM_PARAM_REQUEST_ID, 91)
        d_sim, _, st_sim = eng.run()
        d_sim = d_sim.cpu().numpy()
        G.gdpm_set_param(eng.ctx, G.GDPM_PARAM_SERVE_SMALL_HIST, 200_000)
        G.gdpm_set_param(eng.ctx, G.GDPM_PARAM_SERVE_BIG_SLOTS, big)
        G.gdpm_set_param(eng.ctx, G.GDPM_PARAM_SERVE_SHARE, share)
        G.gdpm_set_param(eng.ctx, G.GDPM_PARAM_SERVE_PHASE_CAP, cap)
        ph = prob.phantom
        ids = [G.gdpm_request_submit(eng.ctx, eng.phantom, eng.tables, prob.source, 400_000, 10)]
        rid = G.gdpm_request_submit(eng.ctx, eng.phantom, eng.tables, prob.source, 300_000, 10,
                                    stream_id=91)
        ids += [G.gdpm_request_submit(eng.ctx, eng.phantom, eng.tables,
                                      W.single_beamlet(ph, 30.0 * k, -1.0, 0.0, 1.0), 50_000, 10)
                for k in range(4)]
        d, _, st = wait(eng.ctx, rid, V)
        for r in ids:
            wait(eng.ctx, r, V)
        with pytest.raises(G.GdpmError) as e:        # the slots are running now
            G.gdpm_set_param(eng.ctx, G.GDPM_PARAM_SERVE_BIG_SLOTS, 1)
        assert e.value.code == G.GDPM_E_STATE
        for param, bad in ((G.GDPM_PARAM_SERVE_SHARE, 0), (G.GDPM_PARAM_SERVE_SHARE, 9),
                           (G.GDPM_PARAM_SERVE_SHARE, 6.5), (G.GDPM_PARAM_SERVE_PHASE_CAP, -1)):
            with pytest.raises(G.GdpmError) as e:
                G.gdpm_set_param(eng.ctx, param, bad)
            assert e.value.code == G.GDPM_E_ARG
    finally:
        eng.close()
    np.testing.assert_allclose(d, d_sim, rtol=1e-9, atol=1e-12 * d_sim.max())
    for k in ("compton", "el_steps", "crossings"):
        assert st[k] == st_sim[k], k
