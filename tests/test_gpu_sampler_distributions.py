"""Interaction samplers on the GPU against their analytic densities.

10^7 draws of each device sampler (gdpm_debug_sample, the same code the
transport kernels inline) are histogrammed and chi-square tested against
bin probabilities integrated from the density the sampler reads: the
Klein-Nishina energy distribution (Sec. 2.1 photon transport), the Moller
delta-ray energy, the 1/k bremsstrahlung spectrum above W_cb, the screened
Rutherford deflection of the hinge, isotropic directions and the Sauter
photoelectron angle.  Two-body kinematics are checked sample by sample.
The oracle samplers are pinned to the same densities on the CPU; here the
FP32 device code is.
"""
import math

import numpy as np
import pytest
from scipy import integrate

from paper_1107_3355_gb300 import gdpm as G
from tests._stats import chi2_pvalue
from tests.test_oracle_pins import kn_dsigma_domega
from tests.test_oracle_variants import sauter_density

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MC2 = 0.51099895
N = 10_000_000
P_MIN = 1e-4


@pytest.fixture(scope="module")
def ctx():
    c = G.gdpm_context_create(0)
    yield c
    G.gdpm_context_destroy(c)


def draw(ctx, kind, a, b, seed):
    o1 = torch.empty(N, dtype=torch.float64, device="cuda")
    o2 = torch.empty(N, dtype=torch.float64, device="cuda")
    G.gdpm_debug_sample(ctx, kind, a, b, N, seed, o1, o2)
    return o1.cpu().numpy(), o2.cpu().numpy()


def chi2_against(x, edges, dens):
    # the support, up to FP32 rounding of its end points
    lo, hi = edges[0], edges[-1]
    tol = 1e-6 * max(abs(lo), abs(hi), 1.0)
    assert x.min() >= lo - tol and x.max() <= hi + tol, (x.min(), x.max(), lo, hi)
    expect = np.array([integrate.quad(dens, a, b, limit=200)[0] for a, b in zip(edges[:-1], edges[1:])])
    h, _ = np.histogram(np.clip(x, lo, hi), edges)
    return chi2_pvalue(h, expect * x.size / expect.sum())[0]


@pytest.mark.parametrize("E", [0.1, 1.0, 6.0])
def test_klein_nishina(ctx, E):
    eps, cost = draw(ctx, 0, E, 0.0, 101)
    k = E / MC2
    e0 = 1 / (1 + 2 * k)

    def dens(e):
        c = 1 - (1 / e - 1) / k
        return 2 * math.pi * kn_dsigma_domega(E, c) / (k * e * e)

    p = chi2_against(eps, np.linspace(e0, 1, 41), dens)
    print("KN", E, p)
    assert p > P_MIN
    np.testing.assert_allclose(cost, 1 - (1 / eps - 1) / k, atol=2e-5)


@pytest.mark.parametrize("T", [1.0, 10.0])
def test_moller(ctx, T):
    wcc = 0.2
    eps, cosd = draw(ctx, 1, T, wcc, 102)
    ec = wcc / T
    tau = T / MC2
    c1 = (tau / (tau + 1)) ** 2
    c2 = (2 * tau + 1) / (tau + 1) ** 2

    def dens(e):
        return 1 / e ** 2 + 1 / (1 - e) ** 2 + c1 - c2 / (e * (1 - e))

    p = chi2_against(eps, np.geomspace(ec, 0.5, 41), dens)
    print("Moller", T, p)
    assert p > P_MIN
    W = eps * T
    np.testing.assert_allclose(cosd, np.sqrt(W * (T + 2 * MC2) / (T * (W + 2 * MC2))), atol=2e-5)


def test_bremsstrahlung_one_over_k(ctx):
    T, wcb = 5.0, 0.05
    k, _ = draw(ctx, 2, T, wcb, 103)
    p = chi2_against(k, np.geomspace(wcb, T, 41), lambda x: 1.0 / x)
    print("brems", p)
    assert p > P_MIN


@pytest.mark.parametrize("A", [1e-3, 0.05, 1.0])
def test_screened_rutherford(ctx, A):
    """Bins reach down to 1 - mu = 1e-4: the device returns mu in FP32,
    whose spacing near 1 (6e-8) would show in narrower bins.  The first
    moment, which FP32 rounding leaves unbiased, is checked exactly:
    E[1 - mu] = 2A(1+A)[ln((1+A)/A) - 1/(1+A)]."""
    mu, _ = draw(ctx, 3, A, 0.0, 104)
    edges = np.sort(np.concatenate([[1.0], 1 - np.geomspace(1e-4, 2, 40)]))   # -1 ... 1 - 1e-4, 1
    p = chi2_against(mu, edges, lambda m: 1.0 / (1 - m + 2 * A) ** 2)
    t = 1.0 - mu
    m1 = 2 * A * (1 + A) * (math.log((1 + A) / A) - 1 / (1 + A))
    z = (t.mean() - m1) / (t.std() / math.sqrt(t.size))
    print("SR", A, p, "first moment z", z)
    assert p > P_MIN
    assert abs(z) < 5


def test_isotropic(ctx):
    cost, phi = draw(ctx, 4, 0.0, 0.0, 105)
    assert chi2_against(cost, np.linspace(-1, 1, 41), lambda c: 1.0) > P_MIN
    assert chi2_against(phi, np.linspace(0, 2 * math.pi, 33), lambda c: 1.0) > P_MIN


@pytest.mark.parametrize("T", [0.02, 0.6, 3.0])
def test_sauter(ctx, T):
    mu, phi = draw(ctx, 5, T, 0.0, 106)
    p = chi2_against(mu, np.linspace(-1, 1, 41), lambda m: sauter_density(m, T))
    print("Sauter", T, p)
    assert p > P_MIN
    assert chi2_against(phi, np.linspace(0, 2 * math.pi, 17), lambda c: 1.0) > P_MIN
