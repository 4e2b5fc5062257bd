"""The oracle against the precision the paper prints for its phantom cases.

Table 1 (Sec. 3.1) gives sigma/Dmax for 2.5e6 histories of a 20 MeV
electron beam on the water-lung-water and water-bone-water slabs of Sec.
3.1.  Batch estimates of sigma fall as N^(-1/2), so the oracle, run on the
same geometry with N histories, must give sigma/Dmax * sqrt(N / 2.5e6)
close to the printed value.  The physics data are this build's readings of
DPM's (different material densities, no DPM tables), so "close" is a band
of a factor 1.5 either way: wide enough for those differences, narrow
enough to catch a wrong power of N, a variance in place of a standard
deviation or a missing batch factor.
"""
import math

import pytest

from oracle import oracle as O
from paper_1107_3355_gb300 import workloads as W
from tests._stats import sigma_over_dmax
from tests.paper_values import table1

N = 15_000


@pytest.mark.parametrize("row", [r for r in table1() if r["source"] == "electron"],
                         ids=lambda r: r["middle"])
def test_electron_precision_scales_to_table1(row):
    prob = W.paper_slab_problem(row["middle"], W.ELECTRON, n_histories=N)
    d, s, led = O.run(prob)
    scaled = sigma_over_dmax(d, s) * math.sqrt(N / row["histories"])
    print(row["middle"], "oracle %.3f %%  paper %.2f %%" % (100 * scaled, 100 * row["sigma_cpu"]))
    assert row["sigma_cpu"] / 1.5 < scaled < row["sigma_cpu"] * 1.5
    assert led["sigma_over_dmax"] == pytest.approx(sigma_over_dmax(d, s), rel=1e-9)
