"""gdpm_autotune: tries launch configurations, keeps the fastest, sets it.

The per-history random streams make results independent of the launch
configuration, so a run under the tuned configuration must give the same
integer event counts as a run under the defaults.
"""
import pytest

from paper_1107_3355_gb300 import gdpm as G
from paper_1107_3355_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

KEYS = ("n_primary", "compton", "photoelectric", "pair", "el_steps", "moller", "brems",
        "crossings", "ph_flights", "annihilations", "local_deposits")


def test_autotune_sets_a_valid_configuration_and_keeps_results():
    prob = W.slab_photon_problem(n_histories=3_000_000, n_batches=10)
    eng = G.Engine(prob)
    try:
        _, _, ref = eng.run()
        r = G.gdpm_autotune(eng.ctx, eng.phantom, eng.tables, prob.n_histories, prob.n_batches,
                            budget_ms=5000.0)
        print("tuned", r)
        assert r["batch_mode"] in (1, 2)
        assert r["speculative"] in (1, 2, 4)
        assert 1 <= r["source_chunk"] <= prob.n_histories
        assert r["candidates_tried"] >= 1 and r["histories_per_s"] > 0
        assert r["electron_walk"] in (0, 1)
        assert r["block_threads"] in (0, 128, 192, 256)
        assert r["queue_capacity"] in (0, 4 * r["source_chunk"] + 65536)
        assert r["graph"] in (0, 1) and (r["graph"] == 0 or r["batch_mode"] == 2)
        _, _, st = eng.run()
        for k in KEYS:
            assert st[k] == ref[k], k
        assert st["deposited"] == pytest.approx(ref["deposited"], rel=1e-9)
    finally:
        eng.close()


@pytest.mark.parametrize("walk,threads,cap", [(0, 128, 0), (1, 192, 4 * 300_000 + 65536),
                                              (1, 256, 0)])
def test_tuned_dimensions_keep_results(walk, threads, cap):
    """Each dimension the autotuner sets beyond the phase layout -- electron
    phase form, block shape, queue capacity -- changes only the launch: the
    integer event counts and the energy ledger equal the defaults'."""
    prob = W.slab_electron_problem(n_histories=300_000, n_batches=10, shape=(64, 64, 128))
    eng = G.Engine(prob)
    try:
        _, _, ref = eng.run()
        G.gdpm_set_param(eng.ctx, G.GDPM_PARAM_ELECTRON_WALK, walk)
        G.gdpm_set_param(eng.ctx, G.GDPM_PARAM_BLOCK_THREADS, threads)
        G.gdpm_set_param(eng.ctx, G.GDPM_PARAM_QUEUE_CAPACITY, cap)
        _, _, st = eng.run()
        for k in KEYS:
            assert st[k] == ref[k], k
        assert st["deposited"] == pytest.approx(ref["deposited"], rel=1e-9)
    finally:
        eng.close()


def test_autotune_rejects_bad_budget():
    prob = W.tiny_problem(n_histories=10_000, n_batches=10)
    eng = G.Engine(prob)
    try:
        with pytest.raises(G.GdpmError) as e:
            G.gdpm_autotune(eng.ctx, eng.phantom, eng.tables, prob.n_histories, prob.n_batches,
                            budget_ms=0.0)
        assert e.value.code == G.GDPM_E_ARG
    finally:
        eng.close()
