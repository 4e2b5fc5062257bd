"""The bounds-checked build (libgdpm_checked.so, GDPM_CHECKED=1).

Every voxel, tally, table, queue and record index is tested before use in
that build.  On valid inputs no check may fire, and the checks must not
change what is computed: the same per-history event records and ledger as
the normal build.  Each run is a child process, since a process loads one
of the two libraries.
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, sys
import numpy as np
import torch
sys.path.insert(0, %(root)r)
from paper_1107_3355_gb300 import gdpm as G, workloads as W
case, out = sys.argv[1], sys.argv[2]
if case == "slab":
    prob = W.slab_photon_problem(n_histories=200_000, n_batches=10)
elif case == "electron":
    prob = W.slab_electron_problem(n_histories=20_000, n_batches=10)
elif case == "ct":
    prob = W.ct_imrt_problem(n_histories=200_000, n_batches=10)
else:
    prob = W.beamlet_matrix_problem(n_beamlets=6, seed=7, n_batches=10, hist_range=(3000, 20000),
                                    shape=(32, 32, 32), voxel=(0.5, 0.5, 0.5))
eng = G.Engine(prob)
try:
    n = prob.n_histories
    rec = torch.zeros(n * 4, dtype=torch.int32, device="cuda")
    recd = torch.zeros(n * 2, dtype=torch.float64, device="cuda")
    G.gdpm_set_history_records(eng.ctx, rec, recd, n)
    if case == "matrix":
        dose, _, st = eng.run_beamlets()
    else:
        dose, _, st = eng.run()
    np.save(out + ".rec.npy", rec.cpu().numpy())
    np.save(out + ".dose.npy", dose.cpu().numpy())
    json.dump({"checked": G.checked_build(), "lib": G.library_path(),
               "deposited": st["deposited"], "escaped": st["escaped"],
               "n_primary": st["n_primary"]}, open(out + ".json", "w"))
finally:
    eng.close()
"""


def run_child(case, checked, tmp_path):
    out = str(tmp_path / ("%s_%d" % (case, checked)))
    env = dict(os.environ, GDPM_CHECKED="1" if checked else "0")
    script = tmp_path / "child.py"
    script.write_text(CHILD % {"root": ROOT})
    r = subprocess.run([sys.executable, str(script), case, out], env=env, capture_output=True,
                       text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    meta = json.load(open(out + ".json"))
    return meta, np.load(out + ".rec.npy"), np.load(out + ".dose.npy")


@pytest.mark.parametrize("case", ["slab", "electron", "ct", "matrix"])
def test_checked_build_is_silent_and_transparent(case, tmp_path):
    m1, rec1, dose1 = run_child(case, True, tmp_path)
    m0, rec0, dose0 = run_child(case, False, tmp_path)
    assert m1["checked"] and m1["lib"].endswith("libgdpm_checked.so")
    assert not m0["checked"] and m0["lib"].endswith("libgdpm.so")
    # no check fired (the call would have raised GDPM_E_BOUNDS), and the
    # per-history event records are the same as without checks
    same = (rec1.reshape(-1, 4) == rec0.reshape(-1, 4)).all(axis=1).mean()
    assert same > 0.999, same
    assert m1["n_primary"] == m0["n_primary"]
    assert m1["deposited"] == pytest.approx(m0["deposited"], rel=1e-3)
    assert np.isfinite(dose1).all()
