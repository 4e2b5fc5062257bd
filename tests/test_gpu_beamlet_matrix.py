"""Beamlet dose matrix (gdpm_simulate_beamlets) against the oracle.

Every fluence-map row is its own calculation with its own range of history
ids, so beamlet k on the GPU must reproduce, history by history, the oracle
run of that beamlet alone (Problem.sub_problem(k)): same per-history event
records (up to FP32/FP64 branch flips), doses that pass the Sec. 3.1 t-test,
and an energy ledger that sums over the beamlets.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1107_3355_gb300 import gdpm as G
from paper_1107_3355_gb300 import workloads as W
from tests._stats import BIAS_GATE, t_test

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def small_matrix(n_batches=10):
    return W.beamlet_matrix_problem(n_beamlets=6, seed=7, n_batches=n_batches,
                                    hist_range=(3000, 20000), shape=(32, 32, 32),
                                    voxel=(0.5, 0.5, 0.5))


def test_dose_matrix_matches_oracle_per_beamlet():
    prob = small_matrix()
    K, V, total = len(prob.sub_histories), prob.phantom.n_voxels, prob.n_histories
    eng = G.Engine(prob)
    try:
        rec = torch.zeros(total * 4, dtype=torch.int32, device="cuda")
        recd = torch.zeros(total * 2, dtype=torch.float64, device="cuda")
        G.gdpm_set_history_records(eng.ctx, rec, recd, total)
        dose, sigma, st = eng.run_beamlets()
        dose, sigma = dose.cpu().numpy(), sigma.cpu().numpy()
        rec = rec.cpu().numpy().reshape(-1, 4)
    finally:
        eng.close()
    recs, dep, src_e = [], 0.0, 0.0
    for k in range(K):
        sub = prob.sub_problem(k)
        d_o, s_o, led, r_o, _ = O.run(sub, per_history=True)
        recs.append(r_o)
        dep += led["deposited"]
        src_e += led["source_energy"]
        r = t_test(d_o, s_o, dose[k], sigma[k], high_frac=0.1)
        print("beamlet", k, sub.n_histories, r)
        assert r["P_high"] >= 0.95, (k, r)
        assert abs(r["bias"]) <= BIAS_GATE, (k, r)
    same = np.all(np.concatenate(recs) == rec, axis=1)
    print("dose matrix identical records: %.5f" % same.mean())
    assert same.mean() > 0.999
    assert st["n_primary"] == total
    assert st["source_energy"] == pytest.approx(src_e, rel=1e-6)
    assert st["deposited"] == pytest.approx(dep, rel=2e-3)
    bal = st["deposited"] + st["escaped"] + st["discarded"]
    assert bal == pytest.approx(st["source_energy"], rel=1e-6)


def test_dose_only_matrix_host_outputs():
    """One batch and no sigma, host outputs: the same per-beamlet doses as a
    ten-batch run within its statistical error."""
    prob = small_matrix()
    K, V = len(prob.sub_histories), prob.phantom.n_voxels
    eng = G.Engine(prob)
    try:
        d10, s10, _ = eng.run_beamlets()
        d10, s10 = d10.cpu().numpy(), s10.cpu().numpy()
        host = np.full((K, V), -1.0)
        st = G.gdpm_simulate_beamlets(eng.ctx, eng.phantom, eng.tables, prob.sub_histories, 1, host)
    finally:
        eng.close()
    assert np.all(host >= 0.0)
    for k in range(K):
        # the one-batch run orders its histories' energy intervals differently,
        # so it is an independent estimate with about the same error
        r = t_test(d10[k], s10[k], host[k], s10[k], high_frac=0.1)
        assert r["P_high"] >= 0.9, (k, r)
    assert st["n_primary"] == prob.n_histories


def test_dose_matrix_bad_inputs():
    prob = small_matrix()
    eng = G.Engine(prob)
    try:
        K, V = len(prob.sub_histories), prob.phantom.n_voxels
        d = torch.empty((K, V), dtype=torch.float64, device="cuda")
        with pytest.raises(G.GdpmError) as e:        # fewer histories than batches
            G.gdpm_simulate_beamlets(eng.ctx, eng.phantom, eng.tables, [5] * K, 10, d, d)
        assert e.value.code == G.GDPM_E_ARG
        with pytest.raises(G.GdpmError) as e:        # too many tally slots
            G.gdpm_simulate_beamlets(eng.ctx, eng.phantom, eng.tables, [100000] * K, 6000, d)
        assert e.value.code == G.GDPM_E_ARG
        with pytest.raises(G.GdpmError) as e:        # sigma needs two batches
            G.gdpm_simulate_beamlets(eng.ctx, eng.phantom, eng.tables, prob.sub_histories, 1, d, d)
        assert e.value.code == G.GDPM_E_ARG
        G.gdpm_source_set(eng.ctx, W.pencil_source(prob.phantom, 1.0))
        with pytest.raises(G.GdpmError) as e:        # not a fluence map
            G.gdpm_simulate_beamlets(eng.ctx, eng.phantom, eng.tables, prob.sub_histories, 10, d)
        assert e.value.code == G.GDPM_E_ARG
    finally:
        eng.close()
