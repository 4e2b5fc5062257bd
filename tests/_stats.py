"""Comparison statistics used by the tests (paper Sec. 3.1)."""
import numpy as np


def sigma_over_dmax(dose, sigma, frac=0.5):
    """Mean of sigma/Dmax over voxels with D > frac*Dmax (Sec. 3.1)."""
    dose = np.asarray(dose); sigma = np.asarray(sigma)
    dmax = float(dose.max())
    sel = dose > frac * dmax
    return float(np.mean(sigma[sel]) / dmax)


def t_test(d1, s1, d2, s2, high_frac=0.1, threshold=2.0, mask=None):
    """Per-voxel two-sample test t = (D1-D2)/sqrt(s1^2+s2^2) (Sec. 3.1).
    Returns dict(P_high, P_all, bias, mean_abs_rel).  P_high is over voxels
    with D1 > high_frac*Dmax; zero-variance voxels pass iff D1 == D2.  With
    `mask` (booleans per voxel) only those voxels count, Dmax included: in a
    phantom with air, tissue-like voxels (density >= 0.05 g/cm3), as for the
    Sec. 3.1 metric, since an air voxel's tiny mass turns one deposit into a
    huge dose."""
    d1 = np.asarray(d1, np.float64); d2 = np.asarray(d2, np.float64)
    s1 = np.asarray(s1, np.float64); s2 = np.asarray(s2, np.float64)
    if mask is not None:
        mask = np.asarray(mask, bool)
        d1, d2, s1, s2 = d1[mask], d2[mask], s1[mask], s2[mask]
    s = np.sqrt(s1 ** 2 + s2 ** 2)
    diff = d1 - d2
    ok = np.where(s > 0, np.abs(diff) <= threshold * s, diff == 0)
    dmax = max(float(d1.max()), float(d2.max()))
    high = d1 > high_frac * dmax
    return dict(P_high=float(ok[high].mean()), P_all=float(ok.mean()),
                bias=float(diff[high].sum() / d1[high].sum()),
                mean_abs_rel=float(np.mean(np.abs(diff[high]) / d1[high])),
                n_high=int(high.sum()))


# Gate 1 of the dose comparison: the signed bias |sum dD| / sum D over the
# voxels above 10 % of Dmax stays within 0.5 %.
BIAS_GATE = 0.005


def signed_bias(d_ref, d, high_frac=0.1):
    """sum(d_ref - d) / sum(d_ref) over voxels with d_ref > high_frac * Dmax
    (0 when no voxel holds dose)."""
    d_ref = np.asarray(d_ref, np.float64); d = np.asarray(d, np.float64)
    dmax = max(float(d_ref.max()), float(d.max()))
    if dmax <= 0:
        return 0.0
    high = d_ref > high_frac * dmax
    return float((d_ref - d)[high].sum() / d_ref[high].sum())


def chi2_pvalue(observed, expected, ddof=0):
    from scipy import stats
    observed = np.asarray(observed, np.float64); expected = np.asarray(expected, np.float64)
    keep = expected > 5
    o, e = observed[keep], expected[keep]
    e = e * o.sum() / e.sum()
    chi2 = float(((o - e) ** 2 / e).sum())
    return float(stats.chi2.sf(chi2, len(o) - 1 - ddof)), chi2
