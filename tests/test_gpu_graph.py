"""The device-driven phase loop (GDPM_PARAM_GRAPH = 1): one CUDA graph launch
whose conditional WHILE node repeats photon phase, electron phase and a
control kernel until no primaries or particles are left.

It transports the same histories as the host loop (same random streams);
its phase kernel is a separate compilation of the same transport code, so
a few histories may take another FP32 branch.  Checked: per-history
records, the Sec. 3.1 t-test, ledger closure, the phase cap, and a
Metropolis-sampled fluence map (the chains advance inside the loop).
"""
import numpy as np
import pytest

from paper_1107_3355_gb300 import gdpm as G
from paper_1107_3355_gb300 import workloads as W
from tests._stats import BIAS_GATE, t_test

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def run(prob, graph, records=True, params=None):
    p = {G.GDPM_PARAM_GRAPH: graph}
    p.update(params or {})
    eng = G.Engine(prob, params=p)
    try:
        rec = torch.zeros(prob.n_histories * 4, dtype=torch.int32, device="cuda")
        recd = torch.zeros(prob.n_histories * 2, dtype=torch.float64, device="cuda")
        if records:
            G.gdpm_set_history_records(eng.ctx, rec, recd, prob.n_histories)
        d, s, st = eng.run()
        return d.cpu().numpy(), s.cpu().numpy(), st, rec.cpu().numpy().reshape(-1, 4)
    finally:
        eng.close()


@pytest.mark.parametrize("case", ["slab_photon", "slab_electron", "ct_metropolis"])
def test_graph_loop_matches_host_loop(case):
    if case == "slab_photon":
        prob = W.slab_photon_problem(n_histories=200_000, n_batches=10, shape=(64, 64, 128))
    elif case == "slab_electron":
        prob = W.slab_electron_problem(n_histories=20_000, n_batches=10, shape=(64, 64, 128))
    else:
        ph = W.ct_phantom(shape=(64, 64, 32), voxel=(1.0, 1.0, 1.0))
        src = W.imrt_plan(ph)
        src.sampler = "metropolis"
        src.chains = 512
        prob = W.Problem(ph, src, 100_000, 10, eabs_photon=0.05, eabs_electron=0.2,
                         e_min=0.005, e_max=6.5)
    d_h, s_h, st_h, r_h = run(prob, 0)
    d_g, s_g, st_g, r_g = run(prob, 1)
    same = np.all(r_h == r_g, axis=1).mean()
    print(case, "graph vs host identical records: %.5f" % same, "phases", st_h["phases"], st_g["phases"])
    assert same > 0.999
    r = t_test(d_h, s_h, d_g, s_g, high_frac=0.1)
    assert r["P_high"] >= 0.99, r
    assert abs(r["bias"]) <= BIAS_GATE, r
    assert st_g["n_primary"] == prob.n_histories
    bal = st_g["deposited"] + st_g["escaped"] + st_g["discarded"]
    assert bal == pytest.approx(st_g["source_energy"], rel=1e-5)
    assert st_g["pushes"] == st_g["pops"]


def test_graph_loop_phase_cap():
    # 20 MeV electrons need more than 8 phases (bremsstrahlung photons,
    # their electrons, annihilation photons, ...)
    prob = W.slab_electron_problem(n_histories=2000, n_batches=2, shape=(32, 32, 128))
    eng = G.Engine(prob, params={G.GDPM_PARAM_GRAPH: 1, G.GDPM_PARAM_MAX_PHASES: 8})
    try:
        with pytest.raises(G.GdpmError) as e:
            eng.run()
        assert e.value.code == G.GDPM_E_TIMEOUT
    finally:
        eng.close()


def test_graph_loop_reused_across_calls():
    """The instantiated graph is kept and relaunched: equal results twice."""
    prob = W.tiny_problem(n_histories=50_000, n_batches=10)
    eng = G.Engine(prob, params={G.GDPM_PARAM_GRAPH: 1})
    try:
        d1, _, st1 = eng.run()
        d1 = d1.cpu().numpy()
        d2, _, st2 = eng.run()
        assert st1["compton"] == st2["compton"] and st1["el_steps"] == st2["el_steps"]
        np.testing.assert_allclose(d2.cpu().numpy(), d1, rtol=1e-12, atol=1e-15)
    finally:
        eng.close()
