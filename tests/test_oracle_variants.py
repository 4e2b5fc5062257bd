"""Pins for the oracle's physics variants (paper Sec. 4).

* Sauter photoelectron angles: the sampler against the density it reads,
  p(mu) ~ (1-mu^2)/(1-beta mu)^4 [1 + gamma(gamma-1)(gamma-2)(1-beta mu)/2],
  by chi-square on binned mu (bin probabilities by numerical integration),
  on both sides of gamma = 2 where the bracket changes sign; its mean moves
  forward with energy; and in transport the photon history is untouched
  (the variant only turns the photoelectron).
* ICRU-44 lung tissue: the composition-dependent coefficients follow the
  closed forms (electron density and Z^4 sums) for that composition.
"""
import numpy as np
import pytest
from scipy import integrate

from oracle import oracle as O
from paper_1107_3355_gb300 import workloads as W
from tests._stats import chi2_pvalue

MC2 = 0.51099895


def sauter_density(mu, T):
    g = 1.0 + T / MC2
    beta = np.sqrt(1.0 - 1.0 / g ** 2)
    b = 0.5 * g * (g - 1.0) * (g - 2.0)
    d = 1.0 - beta * mu
    return (1.0 - mu ** 2) / d ** 4 * (1.0 + b * d)


@pytest.mark.parametrize("T", [0.02, 0.15, 0.6, 3.0])
def test_sauter_sampler_matches_its_density(T):
    mu, phi = O.sample(O.OS_SAUTER, T, 0.0, 200_000, seed=7)
    assert np.all(np.abs(mu) <= 1.0)
    edges = np.linspace(-1.0, 1.0, 41)
    probs = np.array([integrate.quad(sauter_density, a, b, args=(T,))[0]
                      for a, b in zip(edges[:-1], edges[1:])])
    probs /= probs.sum()
    h, _ = np.histogram(mu, bins=edges)
    p, _ = chi2_pvalue(h, probs * mu.size)
    assert p > 1e-3, (T, p)
    # azimuth uniform
    hp, _ = np.histogram(phi, bins=16, range=(0, 2 * np.pi))
    assert chi2_pvalue(hp, np.full(16, mu.size / 16))[0] > 1e-3


def test_sauter_forward_peaking_grows_with_energy():
    means = [O.sample(O.OS_SAUTER, T, 0.0, 50_000, seed=3)[0].mean() for T in (0.01, 0.1, 1.0, 5.0)]
    assert all(a < b for a, b in zip(means, means[1:]))
    assert abs(means[0]) < 0.2               # nearly the dipole (1 - mu^2) at 10 keV


def test_sauter_variant_leaves_photon_histories_alone():
    """Low-energy photons with a low electron cutoff, so photoelectrons are
    transported: photon counts identical with and without the variant; the
    electrons (and so the dose) differ; energy still balances."""
    ph = W.homogeneous_phantom((16, 16, 16), (0.2, 0.2, 0.2), W.WATER, 1.0)
    base = W.Problem(ph, W.pencil_source(ph, 0.08), 20_000, 10, eabs_photon=0.005,
                     eabs_electron=0.01, e_min=0.002, e_max=0.1)
    d0, _, l0 = O.run(base)
    d1, _, l1 = O.run(base.with_(flags=W.FLAG_SAUTER))
    for k in ("ph_flights", "compton", "photoelectric", "n_primary"):
        assert l0[k] == l1[k], k
    assert l1["photoelectric"] > 500
    assert not np.array_equal(d0, d1)
    for led in (l0, l1):
        bal = led["deposited"] + led["escaped"] + led["discarded"]
        assert bal == pytest.approx(led["source_energy"], rel=1e-9)


def test_icru_lung_coefficients_follow_its_composition():
    """Electron density per gram and the photoelectric Z^4 sum of ICRU lung
    against sums written out from its mass fractions."""
    NA = 6.02214076e23
    ph = W.slab_phantom((8, 8, 32), (0.5, 0.5, 0.5),
                        layers=((3.0, W.WATER, 1.0), (10.0, W.LUNG_ICRU, 0.26), (1e30, W.WATER, 1.0)))
    prob = W.Problem(ph, W.pencil_source(ph, 1.0), 100, 10, eabs_photon=0.05, eabs_electron=0.2,
                     e_min=0.005, e_max=1.5)
    m = ph.materials.index(W.LUNG_ICRU)
    ne = sum(w * z / a for z, a, w in W.LUNG_ICRU.elements) * NA
    assert O.evaluate(prob, m, O.OF_NE, 0.0)[0] == pytest.approx(ne, rel=1e-12)
    # mu_C scales with n_e: lung/water ratio equals the electron-density ratio
    w = ph.materials.index(W.WATER)
    ne_w = sum(wf * z / a for z, a, wf in W.WATER.elements) * NA
    r = O.evaluate(prob, m, O.OF_MU_C, 1.0)[0] / O.evaluate(prob, w, O.OF_MU_C, 1.0)[0]
    assert r == pytest.approx(ne / ne_w, rel=1e-12)
    # photoelectric: C_PE sum_i (w_i N_A / A_i) Z_i^4 / E^3
    z4 = sum(wf * NA / a * z ** 4 for z, a, wf in W.LUNG_ICRU.elements)
    E = 0.05
    assert O.evaluate(prob, m, O.OF_MU_PE, E)[0] == pytest.approx(3.9365358876e-32 * z4 / E ** 3, rel=1e-12)
