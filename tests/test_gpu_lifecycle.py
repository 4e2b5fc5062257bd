"""Handles and contexts: repeated create / run / destroy cycles return
every byte of device memory (workspaces, tables, phantoms, sampler
buffers, serving slots and pooled results)."""
import gc

import pytest

from paper_1107_3355_gb300 import gdpm as G
from paper_1107_3355_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def cycle(prob):
    eng = G.Engine(prob)
    try:
        eng.run()
        if prob.source.kind == "beamlets":
            eng.run_beamlets() if prob.sub_histories else None
        rid = G.gdpm_request_submit(eng.ctx, eng.phantom, eng.tables, prob.source, 20_000, 10)
        d = torch.empty(prob.phantom.n_voxels, dtype=torch.float64, device="cuda")
        while not G.gdpm_request_poll(eng.ctx, rid, d, d)[0]:
            pass
    finally:
        eng.close()


def test_no_device_memory_leaks():
    torch.cuda.synchronize()
    probs = [W.tiny_problem(n_histories=50_000, n_batches=10),
             W.beamlet_matrix_problem(n_beamlets=4, n_batches=2, hist_range=(2000, 5000),
                                      shape=(32, 32, 32), voxel=(0.5, 0.5, 0.5))]
    probs[1].source.sampler = "metropolis"
    for p in probs:            # the first cycle loads modules and sizes pools
        cycle(p)
    gc.collect()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        for p in probs:
            cycle(p)
    gc.collect()
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    # allow for allocator granularity, nothing more
    assert free0 - free1 <= (4 << 20), (free0, free1)
