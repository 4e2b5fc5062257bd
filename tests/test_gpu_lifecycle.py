"""Handles and contexts: repeated create / run / destroy cycles return
every byte of device memory (workspaces, tables, phantoms, sampler
buffers, serving slots and pooled results)."""
import gc

import pytest

from paper_1107_3355_gb300 import gdpm as G
from paper_1107_3355_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def cycle(prob):
    eng = G.Engine(prob)
    try:
        eng.run()
        if prob.source.kind == "beamlets":
            eng.run_beamlets() if prob.sub_histories else None
        rid = G.gdpm_request_submit(eng.ctx, eng.phantom, eng.tables, prob.source, 20_000, 10)
        d = torch.empty(prob.phantom.n_voxels, dtype=torch.float64, device="cuda")
        while not G.gdpm_request_poll(eng.ctx, rid, d, d)[0]:
            pass
    finally:
        eng.close()


def test_no_device_memory_leaks():
    torch.cuda.synchronize()
    probs = [W.tiny_problem(n_histories=50_000, n_batches=10),
             W.beamlet_matrix_problem(n_beamlets=4, n_batches=2, hist_range=(2000, 5000),
                                      shape=(32, 32, 32), voxel=(0.5, 0.5, 0.5))]
    probs[1].source.sampler = "metropolis"
    for p in probs:            # the first cycle loads modules and sizes pools
        cycle(p)
    gc.collect()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        for p in probs:
            cycle(p)
    gc.collect()
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    # allow for allocator granularity, nothing more
    assert free0 - free1 <= (4 << 20), (free0, free1)


def test_tally_grids_cleared_between_calculations():
    """The batch fold zeroes each per-batch grid as it reads it, and the
    next calculation on the context skips the grids' memset.  Whatever ran
    before -- the same calculation, fewer batches, a calculation stopped
    by its phase cap before the fold, the FP32-pair tally -- a calculation
    must give the fresh context's events and dose."""
    # 20 MeV electrons: more than 8 phases (bremsstrahlung photons, their
    # electrons, ...), so a phase cap of 8 stops the calculation midway
    prob = W.slab_electron_problem(n_histories=200_000, n_batches=10, shape=(32, 32, 128))
    keys = ("n_primary", "compton", "photoelectric", "pair", "el_steps", "moller", "brems",
            "crossings", "ph_flights")

    def run(eng):
        d, s, st = eng.run()
        return d.cpu().numpy(), s.cpu().numpy(), st

    fresh = G.Engine(prob, params={G.GDPM_PARAM_BATCH_MODE: 2})
    try:
        d0, s0, st0 = run(fresh)
    finally:
        fresh.close()

    def same(res, what):
        d, s, st = res
        for k in keys:
            assert st[k] == st0[k], (what, k)
        assert d == pytest.approx(d0, rel=1e-12, abs=1e-300), what
        assert s == pytest.approx(s0, rel=1e-6, abs=1e-300), what

    eng = G.Engine(prob, params={G.GDPM_PARAM_BATCH_MODE: 2})
    try:
        same(run(eng), "first calculation")
        same(run(eng), "grids cleared by the previous fold")
        eng.run(n_batches=5)
        same(run(eng), "after a calculation of fewer batches")
        G.gdpm_set_param(eng.ctx, G.GDPM_PARAM_MAX_PHASES, 8)
        with pytest.raises(G.GdpmError) as e:
            eng.run()                       # stopped after five phases, never folded
        assert e.value.code == G.GDPM_E_TIMEOUT
        G.gdpm_set_param(eng.ctx, G.GDPM_PARAM_MAX_PHASES, 512)
        same(run(eng), "after a calculation stopped before its fold")
        G.gdpm_set_param(eng.ctx, G.GDPM_PARAM_TALLY_MODE, 1)
        eng.run()
        G.gdpm_set_param(eng.ctx, G.GDPM_PARAM_TALLY_MODE, 0)
        same(run(eng), "after an FP32-pair calculation")
    finally:
        eng.close()
