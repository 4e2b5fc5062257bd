"""Runs to a target precision (gdpm_simulate_to_precision, Sec. 3.1 metric).

sigma/Dmax over D > 0.5 Dmax falls as N^(-1/2), so one pilot run predicts
the histories that reach a target; the call reruns until a run meets it.
"""
import pytest

from paper_1107_3355_gb300 import gdpm as G
from paper_1107_3355_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def eng():
    e = G.Engine(W.tiny_problem(n_histories=20_000, n_batches=10))
    yield e
    e.close()


def test_reaches_the_target_from_a_pilot(eng):
    V = eng.prob.phantom.n_voxels
    dose = torch.empty(V, dtype=torch.float64, device="cuda")
    sigma = torch.empty(V, dtype=torch.float64, device="cuda")
    pilot = G.gdpm_simulate(eng.ctx, eng.phantom, eng.tables, 20_000, 10)
    target = pilot["sigma_over_dmax"] / 4                  # about 16x the pilot's histories
    st, total = G.gdpm_simulate_to_precision(eng.ctx, eng.phantom, eng.tables, target, 20_000,
                                             2 ** 32 - 1, 10, dose, sigma)
    assert st["sigma_over_dmax"] <= target
    predicted = 20_000 * (pilot["sigma_over_dmax"] / target) ** 2
    assert 0.8 * predicted < st["n_primary"] < 2.5 * predicted
    assert total >= 20_000 + st["n_primary"]
    assert float(dose.max()) > 0 and float(sigma.max()) > 0


def test_pilot_that_already_meets_the_target(eng):
    st, total = G.gdpm_simulate_to_precision(eng.ctx, eng.phantom, eng.tables, 0.9, 20_000, 10 ** 6, 10)
    assert total == 20_000 and st["n_primary"] == 20_000


def test_cap_on_histories(eng):
    st, total = G.gdpm_simulate_to_precision(eng.ctx, eng.phantom, eng.tables, 1e-6, 20_000, 50_000, 10)
    assert st["n_primary"] == 50_000 and st["sigma_over_dmax"] > 1e-6
    assert total == 20_000 + 50_000


def test_bad_arguments(eng):
    for args in ((0.0, 20_000, 10 ** 6, 10), (0.01, 5, 10 ** 6, 10), (0.01, 20_000, 10_000, 10),
                 (0.01, 20_000, 2 ** 32, 10)):
        with pytest.raises(G.GdpmError) as e:
            G.gdpm_simulate_to_precision(eng.ctx, eng.phantom, eng.tables, *args)
        assert e.value.code == G.GDPM_E_ARG
    rec = torch.zeros(4 * 10 ** 6, dtype=torch.int32, device="cuda")
    recd = torch.zeros(2 * 10 ** 6, dtype=torch.float64, device="cuda")
    G.gdpm_set_history_records(eng.ctx, rec, recd, 10 ** 6)
    try:
        with pytest.raises(G.GdpmError) as e:
            G.gdpm_simulate_to_precision(eng.ctx, eng.phantom, eng.tables, 0.5, 20_000, 10 ** 6, 10)
        assert e.value.code == G.GDPM_E_STATE
    finally:
        G.gdpm_set_history_records(eng.ctx, None, None, 0)
