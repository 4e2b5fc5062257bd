"""Checkpoint / resume: a calculation run as parts (gdpm_simulate_part),
with the per-voxel batch sums as the carried state, then gdpm_finalize,
equals the uninterrupted gdpm_simulate -- histories keep their ids, so
only the order of FP64 additions differs."""
import numpy as np
import pytest

from paper_1107_3355_gb300 import gdpm as G
from paper_1107_3355_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

KEYS = ("n_primary", "compton", "photoelectric", "pair", "el_steps", "moller", "brems",
        "ph_flights", "crossings", "annihilations")


@pytest.mark.parametrize("host_state", [False, True])
def test_parts_equal_uninterrupted_run(host_state):
    prob = W.slab_photon_problem(n_histories=100_003, n_batches=10, shape=(32, 32, 64))
    eng = G.Engine(prob, params={G.GDPM_PARAM_BATCH_MODE: 2})
    V = prob.phantom.n_voxels
    try:
        d_ref, s_ref, st_ref = eng.run()
        d_ref, s_ref = d_ref.cpu().numpy(), s_ref.cpu().numpy()
        if host_state:
            s1, s2 = np.zeros(V), np.zeros(V)
        else:
            s1 = torch.zeros(V, dtype=torch.float64, device="cuda")
            s2 = torch.zeros(V, dtype=torch.float64, device="cuda")
        parts = [(0, 3), (3, 4), (7, 3)]            # resumed twice
        tot = {k: 0 for k in KEYS}
        dep = 0.0
        for b0, n in parts:
            st = G.gdpm_simulate_part(eng.ctx, eng.phantom, eng.tables, prob.n_histories,
                                      prob.n_batches, b0, n, s1, s2)
            for k in KEYS:
                tot[k] += st[k]
            dep += st["deposited"]
        dose = torch.empty(V, dtype=torch.float64, device="cuda")
        sig = torch.empty(V, dtype=torch.float64, device="cuda")
        stf = G.gdpm_finalize(eng.ctx, eng.phantom, prob.n_batches, s1, s2, dose, sig)
    finally:
        eng.close()
    np.testing.assert_allclose(dose.cpu().numpy(), d_ref, rtol=1e-9, atol=1e-12 * d_ref.max())
    np.testing.assert_allclose(sig.cpu().numpy(), s_ref, rtol=1e-6, atol=1e-9 * s_ref.max())
    for k in KEYS:
        assert tot[k] == st_ref[k], k
    assert dep == pytest.approx(st_ref["deposited"], rel=1e-9)
    assert stf["sigma_over_dmax"] == pytest.approx(st_ref["sigma_over_dmax"], rel=1e-6)


def test_part_bad_ranges():
    prob = W.tiny_problem(n_histories=10_000, n_batches=10)
    eng = G.Engine(prob)
    V = prob.phantom.n_voxels
    try:
        s1 = torch.zeros(V, dtype=torch.float64, device="cuda")
        for b0, n in ((-1, 2), (8, 3), (0, 0)):
            with pytest.raises(G.GdpmError) as e:
                G.gdpm_simulate_part(eng.ctx, eng.phantom, eng.tables, 10_000, 10, b0, n, s1, s1)
            assert e.value.code == G.GDPM_E_ARG
    finally:
        eng.close()
