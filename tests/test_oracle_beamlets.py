"""Pins for the oracle's beamlet samplers (Sec. 2.3.1).

All three samplers must draw beamlet I with probability f_I / sum f over the
beamlets of positive fluence.  The checks use what the mathematics fixes:
the exact probability mass held by an alias table, chi-square tests of
sampled histograms against f, and -- for the Metropolis chain of
Algorithm A1 -- its one-step transition law min(1, f_J/f_I)/n_f, the
distribution of independent chains after k steps (the uniform start
multiplied by the transition matrix k times), and the convergence of the
fluence error e(N) = ||p_f - p_f*||_2 with the number of particles
(Fig. 2(c)).
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1107_3355_gb300 import workloads as W
from tests._stats import chi2_pvalue


def beamlet_problem(weights, sampler="cdf", chains=4096, n=1000):
    base = W.tiny_problem(n_histories=n, n_batches=10)
    iso = tuple(e / 2 for e in base.phantom.extent)
    fr = W.beam_frame(0.0, iso, 100.0)
    rows = [W.beamlet_row(fr, 0.5 * k - 4, 0.5 * k - 3.5, -1, 1, float(w))
            for k, w in enumerate(weights)]
    src = W.beamlet_source(rows, W.mono_spectrum(1.0))
    src.sampler = sampler
    src.chains = chains
    return base.with_(source=src)


def transition_matrix(f):
    """Algorithm A1 as a Markov matrix: propose J uniformly among the n
    beamlets, accept with probability min(1, f_J/f_I)."""
    f = np.asarray(f, np.float64)
    n = f.size
    T = np.minimum(1.0, f[None, :] / f[:, None]) / n
    np.fill_diagonal(T, 0.0)
    T[np.arange(n), np.arange(n)] = 1.0 - T.sum(axis=1)
    return T


def fluence_error(picks, f_rows):
    f = np.asarray(f_rows, np.float64)
    p_star = f / f.sum()
    p = np.bincount(picks, minlength=f.size) / picks.size
    return float(np.linalg.norm(p - p_star))


def test_alias_table_holds_the_exact_probabilities():
    rng = np.random.default_rng(5)
    w = rng.uniform(0, 1, 300)
    w[rng.choice(300, 40, replace=False)] = 0.0          # zero-fluence beamlets are dropped
    w[7] = 50.0                                           # one heavy beamlet
    index, cut, alias = O.beamlet_tables(beamlet_problem(w))
    assert np.array_equal(index, np.flatnonzero(w > 0))
    nf = index.size
    assert np.all((cut > 0) & (cut <= 1.0))
    mass = cut.copy()
    np.add.at(mass, alias, 1.0 - cut)                     # what each column donates
    f = w[index]
    np.testing.assert_allclose(mass / nf, f / f.sum(), rtol=1e-12, atol=1e-15)


@pytest.mark.parametrize("sampler", ["cdf", "alias", "metropolis"])
def test_sampler_histogram_matches_fluence(sampler):
    w = np.array([0.0, 1.0, 2.0, 0.5, 0.0, 4.0, 3.0, 0.25])
    prob = beamlet_problem(w, sampler, chains=64)
    picks = O.beamlet_picks(prob, 0, 200_000)
    assert set(np.unique(picks)) <= set(np.flatnonzero(w > 0))
    counts = np.bincount(picks, minlength=w.size)[w > 0]
    p, _ = chi2_pvalue(counts, w[w > 0] / w.sum() * picks.size)
    # Metropolis draws are correlated along a chain: allow a looser level
    assert p > (1e-6 if sampler == "metropolis" else 1e-3)


def test_metropolis_one_step_transitions():
    f = np.array([1.0, 2.0, 5.0])
    picks = O.beamlet_picks(beamlet_problem(f, "metropolis", chains=1), 0, 300_000)
    T = transition_matrix(f)
    for i in range(3):
        nxt = picks[1:][picks[:-1] == i]
        p, _ = chi2_pvalue(np.bincount(nxt, minlength=3), T[i] * nxt.size)
        assert p > 1e-3, (i, np.bincount(nxt, minlength=3) / nxt.size, T[i])


def test_metropolis_independent_chains_follow_matrix_powers():
    """C chains start uniform; after k + 1 steps (history h = c + k C) each
    chain's beamlet is distributed as uniform @ T^(k+1)."""
    f = np.array([0.2, 1.0, 3.0, 0.6])
    C = 50_000
    prob = beamlet_problem(f, "metropolis", chains=C)
    picks = O.beamlet_picks(prob, 0, 4 * C).reshape(4, C)
    T = transition_matrix(f)
    pi = np.full(4, 0.25)
    for k in range(4):
        pi = pi @ T
        p, _ = chi2_pvalue(np.bincount(picks[k], minlength=4), pi * C)
        assert p > 1e-3, (k, np.bincount(picks[k], minlength=4) / C, pi)


def test_metropolis_chain_is_fixed_by_history_not_by_range():
    f = np.random.default_rng(2).uniform(0.1, 1, 50)
    prob = beamlet_problem(f, "metropolis", chains=16)
    whole = O.beamlet_picks(prob, 0, 4000)
    tail = O.beamlet_picks(prob, 2500, 1500)
    assert np.array_equal(whole[2500:], tail)


def test_fluence_error_decreases_with_particles():
    """Fig. 2(c): e(N) falls with N for the Metropolis sampler, like
    N^(-1/2) once the chains have mixed, and is close to the error of the
    direct samplers at large N."""
    rng = np.random.default_rng(11)
    w = rng.uniform(0, 1, 400)                            # one 20x20 map of intensities
    Ns = [10_000, 100_000, 1_000_000]
    errs = {}
    for sampler in ("metropolis", "alias", "cdf"):
        picks = O.beamlet_picks(beamlet_problem(w, sampler, chains=4096), 0, Ns[-1])
        errs[sampler] = [fluence_error(picks[:n], w) for n in Ns]
    e = errs["metropolis"]
    assert e[0] > e[1] > e[2]
    slope = np.log(e[2] / e[1]) / np.log(Ns[2] / Ns[1])
    assert -0.75 < slope < -0.3
    iid = np.sqrt((1 - np.sum((w / w.sum()) ** 2)) / Ns[-1])   # expected e for independent draws
    assert errs["alias"][2] < 2 * iid and errs["cdf"][2] < 2 * iid
    assert e[2] < 3 * iid
