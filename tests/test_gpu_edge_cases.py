"""Degenerate and limiting cases of the transport, against the oracle.

Beams that never reach the phantom, sources below the absorption energies,
a one-voxel phantom, an air-filled phantom, a phantom at the largest
extent per axis and at the largest volume, one history per batch, and a
ragged history count.  Same
seed on both sides, so each history's event record must agree (Sec. 2.2.1
transport; records differ only where FP32 and FP64 arithmetic part ways),
and the energy ledger must balance.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1107_3355_gb300 import gdpm as G
from paper_1107_3355_gb300 import workloads as W
from tests._stats import BIAS_GATE, signed_bias
from tests.test_gpu_parity import LEDGER_TOL, check_ledger, run_gpu

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def problem(phantom, source, n=20_000, nb=10, eabs_photon=0.01, eabs_electron=0.2, e_max=1.5):
    return W.Problem(phantom, source, n, nb, eabs_photon=eabs_photon, eabs_electron=eabs_electron,
                     e_min=0.005, e_max=e_max)


def same_seed(prob, min_identical=0.99):
    d_o, s_o, led_o, rec_o, _ = O.run(prob, per_history=True)
    d_g, s_g, st, rec_g, _ = run_gpu(prob, records=True)
    check_ledger(st, prob.n_histories, LEDGER_TOL)
    same = np.all(rec_o == rec_g, axis=1).mean()
    assert same >= min_identical, same
    assert st["source_energy"] == pytest.approx(led_o["source_energy"], rel=1e-6)
    assert abs(signed_bias(d_o, d_g)) <= BIAS_GATE
    return d_o, d_g, st, led_o


def test_beam_that_misses_the_phantom():
    ph = W.homogeneous_phantom((16, 16, 16), (0.5, 0.5, 0.5), W.WATER, 1.0)
    src = W.Source(W.PHOTON, W.mono_spectrum(1.0), "pencil", (-5.0, 4.0, 0.0), (0.0, 0.0, 1.0))
    d_o, d_g, st, led_o = same_seed(problem(ph, src))
    assert np.all(d_g == 0.0) and np.all(d_o == 0.0)
    assert st["deposited"] == 0.0
    assert st["escaped"] == pytest.approx(st["source_energy"], rel=1e-12)
    assert st["compton"] == 0 and st["el_steps"] == 0


@pytest.mark.parametrize("particle,energy", [(W.PHOTON, 0.008), (W.ELECTRON, 0.1)])
def test_source_below_its_absorption_energy(particle, energy):
    """Every primary is absorbed where it enters: all energy in the entry
    voxel of the pencil (central voxel of the z=0 face)."""
    ph = W.homogeneous_phantom((16, 16, 16), (0.5, 0.5, 0.5), W.WATER, 1.0)
    src = W.Source(particle, W.mono_spectrum(energy), "pencil", (4.25, 4.25, 0.0), (0.0, 0.0, 1.0))
    d_o, d_g, st, _ = same_seed(problem(ph, src))
    entry = 8 + 16 * 8                     # ix = iy = 8, iz = 0
    assert np.count_nonzero(d_g) == 1 and d_g[entry] > 0
    assert d_g[entry] == pytest.approx(d_o[entry], rel=1e-6)
    assert st["deposited"] == pytest.approx(st["source_energy"], rel=1e-6)


def test_one_voxel_phantom():
    ph = W.homogeneous_phantom((1, 1, 1), (1.0, 1.0, 1.0), W.WATER, 1.0)
    src = W.Source(W.PHOTON, W.mono_spectrum(1.0), "pencil", (0.5, 0.5, 0.0), (0.0, 0.0, 1.0))
    d_o, d_g, st, led_o = same_seed(problem(ph, src, n=50_000))
    assert 0 < st["deposited"] < st["source_energy"]
    assert st["deposited"] == pytest.approx(led_o["deposited"], rel=0.02)


def test_air_filled_phantom():
    ph = W.homogeneous_phantom((32, 32, 32), (0.5, 0.5, 0.5), W.AIR, 0.0012)
    src = W.pencil_source(ph, 1.0)
    d_o, d_g, st, led_o = same_seed(problem(ph, src, n=50_000))
    assert st["escaped"] > 0.99 * st["source_energy"]
    assert st["compton"] == pytest.approx(led_o["compton"], abs=10)


def test_largest_extent_along_an_axis():
    """nx = 1024 voxels (the per-axis limit), a beam along +x through all of
    them; 1025 is refused."""
    ph = W.homogeneous_phantom((1024, 2, 2), (0.1, 0.5, 0.5), W.WATER, 1.0)
    src = W.Source(W.PHOTON, W.mono_spectrum(1.0), "pencil", (0.0, 0.5, 0.5), (1.0, 0.0, 0.0))
    d_o, d_g, st, led_o = same_seed(problem(ph, src, n=20_000))
    along_x = d_g.reshape(2, 2, 1024).sum(axis=(0, 1))
    assert along_x[:100].sum() > 0 and along_x[512:].sum() > 0    # dose past the middle
    ctx = G.gdpm_context_create(0)
    try:
        big = W.homogeneous_phantom((1025, 1, 1), (0.1, 0.1, 0.1), W.WATER, 1.0)
        with pytest.raises(G.GdpmError) as e:
            G.gdpm_phantom_create(ctx, big.shape, big.voxel, big.mat, big.rho)
        assert e.value.code == G.GDPM_E_ARG
    finally:
        G.gdpm_context_destroy(ctx)


@pytest.mark.parametrize("n,nb", [(10, 10), (10_007, 10), (2, 2)])
def test_few_and_ragged_histories_per_batch(n, nb):
    prob = W.tiny_problem(n_histories=n, n_batches=nb)
    d_o, d_g, st, _ = same_seed(prob, min_identical=0.95)
    assert st["n_primary"] == n


@pytest.mark.parametrize("bad", [0.0, -1.0, float("nan"), float("inf")])
def test_phantom_rejects_densities_that_are_not_positive_and_finite(bad):
    """A voxel of zero mass has no dose (its dose would be energy / 0), and a
    negative, NaN or infinite density has no meaning: the phantom is refused."""
    ph = W.homogeneous_phantom((8, 8, 8), (0.5, 0.5, 0.5), W.WATER, 1.0)
    rho = ph.rho.copy()
    rho[137] = bad
    ctx = G.gdpm_context_create(0)
    try:
        with pytest.raises(G.GdpmError) as e:
            G.gdpm_phantom_create(ctx, ph.shape, ph.voxel, ph.mat, rho)
        assert e.value.code == G.GDPM_E_ARG
    finally:
        G.gdpm_context_destroy(ctx)


def test_largest_phantom_volume():
    """1024^3 voxels, the largest grid (2^30 voxels: 5.4 GB of phantom and
    8.6 GB per tally grid, so batches run one after another).  A 64^3 water
    cube in the far corner of a near-vacuum phantom (1e-9 g/cm3) must get the
    dose that a 64^3 water phantom alone gets from the same pencil beam,
    which starts on the cube's face at a voxel centre.  A particle that
    leaves the convex cube never comes back, so each history is the same in
    both geometries up to the FP32 rounding of larger coordinates; a tally
    or index that goes wrong beyond 2^31 bytes or voxels moves dose out of
    the cube."""
    n, m, dx = 1024, 64, 0.0625                    # dx a power of two: exact voxel edges
    c0 = n - m
    rho = np.full((n, n, n), 1e-9, np.float32)
    rho[c0:, c0:, c0:] = 1.0
    big = W.Phantom((n, n, n), (dx, dx, dx), np.zeros(n ** 3, np.uint8), rho.reshape(-1), [W.WATER])
    del rho
    small = W.homogeneous_phantom((m, m, m), (dx, dx, dx), W.WATER, 1.0)
    spec = W.mono_spectrum(1.0)
    off = (m // 2 + 0.5) * dx
    src_big = W.Source(W.PHOTON, spec, "pencil", (c0 * dx + off, c0 * dx + off, c0 * dx), (0.0, 0.0, 1.0))
    src_small = W.Source(W.PHOTON, spec, "pencil", (off, off, 0.0), (0.0, 0.0, 1.0))
    res = {}
    for name, ph, src in (("big", big, src_big), ("small", small, src_small)):
        prob = problem(ph, src, n=100_000, nb=10, e_max=1.5)
        eng = G.Engine(prob)
        try:
            d, s, st = eng.run()
            if name == "big":
                d = d.view(n, n, n)[c0:, c0:, c0:].contiguous()
                assert bool(torch.isfinite(s).all())
            res[name] = (d.cpu().numpy().reshape(-1), st)
        finally:
            eng.close()
        del d, s
        torch.cuda.empty_cache()
        check_ledger(st, prob.n_histories, LEDGER_TOL)
    (d_b, st_b), (d_s, st_s) = res["big"], res["small"]
    for k in ("compton", "el_steps"):
        assert st_b[k] == pytest.approx(st_s[k], rel=5e-3), k
    assert abs(signed_bias(d_s, d_b)) <= BIAS_GATE
    # all of the cube's energy is in the cube: the rest of the big grid holds
    # only the near-vacuum's share
    e_cube = float((d_b.astype(np.float64) * 1.0 * dx ** 3).sum())
    assert e_cube == pytest.approx(st_b["deposited"] / st_b["n_primary"], rel=1e-3)
