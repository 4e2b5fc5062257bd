"""gdpm_simulate_noalloc: the dose calculation without any allocation.

Some callers cannot call cudaMalloc -- applications whose own allocator owns
the GPU's memory (a pool sized at start-up, a planning system with a fixed
memory budget) and that forbid libraries from allocating behind it -- so the
library offers one entry point whose work buffers all live in a fixed static
device array.  This file is named so that pytest collects it last.
"""
import numpy as np
import pytest

from paper_1107_3355_gb300 import gdpm as G
from paper_1107_3355_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_noalloc_matches_simulate_on_two_calls():
    prob = W.tiny_problem(n_histories=50_000, n_batches=10)
    eng = G.Engine(prob)
    try:
        V = prob.phantom.n_voxels
        d_ref, s_ref, st_ref = eng.run()
        d_ref = d_ref.cpu().numpy()
        s_ref = s_ref.cpu().numpy()
        for call in range(2):
            d = torch.full((V,), -1.0, dtype=torch.float64, device="cuda")
            s = torch.full((V,), -1.0, dtype=torch.float64, device="cuda")
            torch.cuda.synchronize()
            free_before = torch.cuda.mem_get_info()[0]
            st = G.gdpm_simulate_noalloc(eng.ctx, eng.phantom, eng.tables, prob.n_histories,
                                         prob.n_batches, d, s)
            torch.cuda.synchronize()
            free_after = torch.cuda.mem_get_info()[0]
            if call == 1:   # the first call on a device may load the module
                assert free_after == free_before
            # same per-history random streams: equal up to FP64 summation order
            np.testing.assert_allclose(d.cpu().numpy(), d_ref, rtol=1e-9,
                                       atol=1e-12 * d_ref.max())
            np.testing.assert_allclose(s.cpu().numpy(), s_ref, rtol=1e-6,
                                       atol=1e-9 * s_ref.max())
            for k in ("n_primary", "compton", "photoelectric", "el_steps", "moller", "brems",
                      "el_created", "ph_created", "crossings"):
                assert st[k] == st_ref[k], k
            assert st["deposited"] == pytest.approx(st_ref["deposited"], rel=1e-12)
            assert st["sigma_over_dmax"] == pytest.approx(st_ref["sigma_over_dmax"], rel=1e-6)
    finally:
        eng.close()


@pytest.mark.parametrize("kind", ["point_field", "beamlets_cdf", "beamlets_metropolis"])
def test_noalloc_matches_simulate_for_field_and_beamlet_sources(kind):
    """A point-source field, and a fluence map of 16 beamlets drawn by the
    cumulative sampler and by the Metropolis chains, through the
    allocation-free entry: gdpm_simulate's events and dose (its batches run
    one after another in small phases, gdpm_simulate's side by side)."""
    if kind == "point_field":
        prob = W.slab_photon_problem(n_histories=100_000, n_batches=10, shape=(32, 32, 32),
                                     voxel=(1.0, 1.0, 1.0))
    else:
        prob = W.beamlet_matrix_problem(n_beamlets=16, n_batches=10, hist_range=(4000, 8000),
                                        shape=(32, 32, 32), voxel=(1.0, 1.0, 1.0))
        if kind == "beamlets_metropolis":
            prob.source.sampler = "metropolis"
    eng = G.Engine(prob)
    try:
        V = prob.phantom.n_voxels
        d_ref, s_ref, st_ref = eng.run()
        d_ref = d_ref.cpu().numpy()
        s_ref = s_ref.cpu().numpy()
        d = torch.full((V,), -1.0, dtype=torch.float64, device="cuda")
        s = torch.full((V,), -1.0, dtype=torch.float64, device="cuda")
        st = G.gdpm_simulate_noalloc(eng.ctx, eng.phantom, eng.tables, prob.n_histories,
                                     prob.n_batches, d, s)
        torch.cuda.synchronize()
        np.testing.assert_allclose(d.cpu().numpy(), d_ref, rtol=1e-9, atol=1e-12 * d_ref.max())
        np.testing.assert_allclose(s.cpu().numpy(), s_ref, rtol=1e-6, atol=1e-9 * s_ref.max())
        for k in ("n_primary", "compton", "photoelectric", "el_steps", "moller", "brems",
                  "el_created", "ph_created", "crossings"):
            assert st[k] == st_ref[k], k
        assert st["deposited"] == pytest.approx(st_ref["deposited"], rel=1e-9)
    finally:
        eng.close()


def test_noalloc_fp32_pair_tally_on_odd_grid():
    """The compensated FP32 tally keeps two float halves in the scratch; on a
    grid with an odd voxel count (31^3) the low half must still be read as
    aligned float pairs.  Two calls in a row equal gdpm_simulate's result in
    the same tally mode."""
    base = W.tiny_problem(n_histories=40_000, n_batches=10)
    ph = W.homogeneous_phantom((31, 31, 31), (0.5, 0.5, 0.5))
    prob = base.with_(phantom=ph, source=W.pencil_source(ph, 1.0))
    eng = G.Engine(prob, params={G.GDPM_PARAM_TALLY_MODE: 1})
    try:
        V = ph.n_voxels
        assert V % 2 == 1
        d_ref, s_ref, st_ref = eng.run()
        d_ref = d_ref.cpu().numpy()
        s_ref = s_ref.cpu().numpy()
        for _ in range(2):
            d = torch.full((V,), -1.0, dtype=torch.float64, device="cuda")
            s = torch.full((V,), -1.0, dtype=torch.float64, device="cuda")
            st = G.gdpm_simulate_noalloc(eng.ctx, eng.phantom, eng.tables, prob.n_histories,
                                         prob.n_batches, d, s)
            torch.cuda.synchronize()
            np.testing.assert_allclose(d.cpu().numpy(), d_ref, rtol=1e-9,
                                       atol=1e-12 * d_ref.max())
            np.testing.assert_allclose(s.cpu().numpy(), s_ref, rtol=1e-6,
                                       atol=1e-9 * s_ref.max())
            for k in ("n_primary", "compton", "el_steps", "crossings"):
                assert st[k] == st_ref[k], k
            assert st["deposited"] == pytest.approx(st_ref["deposited"], rel=1e-9)
    finally:
        eng.close()


def test_noalloc_rejects_sizes_beyond_its_limit():
    prob = W.tiny_problem(n_histories=1000, n_batches=10)
    eng = G.Engine(prob)
    try:
        big = W.homogeneous_phantom((40, 40, 40), (0.5, 0.5, 0.5))     # 64000 > 32768 voxels
        ph = G.gdpm_phantom_create(eng.ctx, big.shape, big.voxel, big.mat, big.rho)
        d = torch.empty(big.n_voxels, dtype=torch.float64, device="cuda")
        with pytest.raises(G.GdpmError) as e:
            G.gdpm_simulate_noalloc(eng.ctx, ph, eng.tables, 1000, 10, d, d)
        assert e.value.code == G.GDPM_E_ARG
        G.gdpm_phantom_destroy(ph)
        host = np.zeros(prob.phantom.n_voxels)
        with pytest.raises(G.GdpmError) as e:
            G.gdpm_simulate_noalloc(eng.ctx, eng.phantom, eng.tables, 1000, 10, host, host)
        assert e.value.code == G.GDPM_E_ARG
    finally:
        eng.close()
