"""The four phantom cases of Table 1 (Sec. 3.1) at the paper's history
counts on the GPU: 2.5e6 electrons and 2.5e8 photons in 10 batches.

The paper reports sigma/Dmax below 1 % in every case; this build's physics
readings (densities, spectrum, cross sections written from closed forms)
differ from DPM's data, so each case must land within a factor 1.25 of the
printed GPU value and below 1.5 %.
"""
import pytest

from paper_1107_3355_gb300 import gdpm as G
from paper_1107_3355_gb300 import workloads as W
from tests._stats import sigma_over_dmax
from tests.paper_values import table1

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("row", table1(), ids=lambda r: "%s-%s" % (r["source"], r["middle"]))
def test_table1_precision(row):
    particle = W.ELECTRON if row["source"] == "electron" else W.PHOTON
    prob = W.paper_slab_problem(row["middle"], particle, n_histories=row["histories"])
    eng = G.Engine(prob)
    try:
        d, s, st = eng.run()
        d, s = d.cpu().numpy(), s.cpu().numpy()
    finally:
        eng.close()
    got = sigma_over_dmax(d, s)
    print("%s %s: sigma/Dmax %.3f %% (paper GPU %.2f %%), %.3f s of transport" %
          (row["source"], row["middle"], 100 * got, 100 * row["sigma_gpu"], st["transport_ms"] / 1e3))
    assert got == pytest.approx(st["sigma_over_dmax"], rel=1e-6)
    assert row["sigma_gpu"] / 1.25 < got < row["sigma_gpu"] * 1.25
    assert got < 0.015
    bal = st["deposited"] + st["escaped"] + st["discarded"]
    assert bal == pytest.approx(st["source_energy"], rel=1e-5)
