"""GPU parity of the fluence-map beamlet samplers (Sec. 2.3.1).

The alias and Metropolis (Algorithm A1) samplers take every decision from
integer Philox words and FP64 comparisons that both sides evaluate in the
same precision, so the beamlet of every history must match the oracle's
exactly; the cumulative search compares the primary's FP32 uniform (FP64 in
the oracle) with the cumulative fluence, so a few histories near interval
edges may differ.  The fluence error e(N) of Fig. 2(c) is checked on the
GPU's own picks.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1107_3355_gb300 import gdpm as G
from paper_1107_3355_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def plan_problem(sampler, chains=4096, n_hist=400_000, n_batches=2):
    ph = W.ct_phantom(shape=(64, 64, 32), voxel=(1.0, 1.0, 1.0))
    src = W.imrt_plan(ph)
    src.sampler = sampler
    src.chains = chains
    return W.Problem(ph, src, n_hist, n_batches, eabs_photon=0.05, eabs_electron=0.2,
                     e_min=0.005, e_max=6.5)


def gpu_picks(prob, first, n):
    eng = G.Engine(prob)
    try:
        out = torch.full((n,), -1, dtype=torch.int32, device="cuda")
        G.gdpm_debug_beamlets(eng.ctx, first, n, out)
        return out.cpu().numpy()
    finally:
        eng.close()


def fluence_error(picks, w):
    p_star = w / w.sum()
    p = np.bincount(picks, minlength=w.size) / picks.size
    return float(np.linalg.norm(p - p_star))


@pytest.mark.parametrize("sampler", ["alias", "metropolis"])
@pytest.mark.parametrize("first", [0, 123_457])
def test_beamlet_picks_bitwise(sampler, first):
    prob = plan_problem(sampler)
    n = 200_000
    g = gpu_picks(prob, first, n)
    o = O.beamlet_picks(prob, first, n)
    assert np.array_equal(g, o), np.flatnonzero(g != o)[:10]


def test_cdf_picks_agree_up_to_uniform_precision():
    prob = plan_problem("cdf")
    g = gpu_picks(prob, 0, 200_000)
    o = O.beamlet_picks(prob, 0, 200_000)
    w = prob.source.beamlets[:, 16]
    assert np.all(w[g] > 0)
    assert (g == o).mean() > 0.999


def test_metropolis_few_chains_and_many_chains():
    """Chain counts at both ends: one chain (strictly sequential) and more
    chains than histories (every history the first step of its chain)."""
    for chains in (1, 1 << 20):
        prob = plan_problem("metropolis", chains=chains)
        g = gpu_picks(prob, 0, 50_000)
        assert np.array_equal(g, O.beamlet_picks(prob, 0, 50_000))


def test_fluence_error_falls_with_particles():
    """Fig. 2(c) on the GPU's picks: 10^7 particles of the 7-beam plan."""
    prob = plan_problem("metropolis", n_hist=10_000_000)
    w = prob.source.beamlets[:, 16]
    g = gpu_picks(prob, 0, 10_000_000)
    Ns = [10_000, 100_000, 1_000_000, 10_000_000]
    e = [fluence_error(g[:n], w) for n in Ns]
    print("e(N):", dict(zip(Ns, e)))
    assert all(a > b for a, b in zip(e, e[1:]))
    slope = np.log(e[-1] / e[-2]) / np.log(10.0)
    assert -0.75 < slope < -0.3
    # the first million equal the oracle's, pick for pick
    assert np.array_equal(g[:1_000_000], O.beamlet_picks(prob, 0, 1_000_000))


def test_metropolis_primaries_elementwise():
    prob = plan_problem("metropolis", chains=512, n_hist=20_000, n_batches=10)
    eng = G.Engine(prob)
    try:
        n = 2000
        out = torch.zeros(n * 8, dtype=torch.float64, device="cuda")
        G.gdpm_debug_sources(eng.ctx, eng.phantom, eng.tables, prob.n_histories,
                             prob.n_batches, 0, n, out)
        g = out.cpu().numpy().reshape(n, 8)
    finally:
        eng.close()
    o = O.sources(prob, 0, n)
    assert np.array_equal(g[:, 7], o[:, 7])
    hit = o[:, 7] > 0
    np.testing.assert_allclose(g[hit, :6], o[hit, :6], atol=2e-4)
    np.testing.assert_allclose(g[:, 6], o[:, 6], rtol=1e-6)
