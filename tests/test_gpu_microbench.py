"""The resource microbenchmarks (gdpm_microbench) that back the roofline.

The atomic kinds must leave exactly the number of adds they report in the
buffer (every add of 1 lands once); the FP32 FMA rate cannot exceed one FMA
per lane per clock (128 lanes per SM at the maximum SM clock).
"""
import pytest

from paper_1107_3355_gb300 import gdpm as G

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = G.gdpm_context_create(0, torch.cuda.current_stream().cuda_stream, 1)
    yield c
    G.gdpm_context_destroy(c)


@pytest.mark.parametrize("kind,dtype", [("red_f64", torch.float64), ("red_f32", torch.float32),
                                        ("atom_f32", torch.float32)])
def test_atomic_kinds_count_every_add(ctx, kind, dtype):
    n_slots = 2_000_003                              # not a power of two
    buf = torch.full((n_slots,), 7.0, dtype=dtype, device="cuda")
    rate, done, ms = G.gdpm_microbench(ctx, kind, buf, n_slots, 50_000_000)
    assert done >= 50_000_000 and ms > 0 and rate > 0
    # each slot holds far fewer than 2^24 adds, so FP32 counts are exact too
    assert buf.max().item() < 2 ** 24
    assert buf.to(torch.float64).sum().item() == done
    print(kind, "%.3g adds/s" % rate)


def test_alu_rates_are_physical(ctx):
    sink = torch.zeros(1, dtype=torch.float32, device="cuda")
    props = torch.cuda.get_device_properties(0)
    lane_peak = props.multi_processor_count * 128 * 2.07e9
    ffma, done, _ = G.gdpm_microbench(ctx, "ffma", sink, 1, int(2e10))
    assert done >= 2e10
    assert 0.3 * lane_peak < ffma < 1.05 * lane_peak, (ffma, lane_peak)
    mufu, _, _ = G.gdpm_microbench(ctx, "mufu_lg2", sink, 1, int(4e9))
    dfma, _, _ = G.gdpm_microbench(ctx, "dfma", sink, 1, int(1e9))
    assert 0 < mufu < ffma and 0 < dfma < ffma
    assert sink.item() == 0.0
    print("ffma %.3g  mufu %.3g  dfma %.3g  (lane peak %.3g)" % (ffma, mufu, dfma, lane_peak))


def test_bad_arguments(ctx):
    buf = torch.zeros(16, dtype=torch.float64, device="cuda")
    for kind, slots, n in ((9, 16, 100), (-1, 16, 100), (0, 0, 100), (0, 16, 0)):
        with pytest.raises(G.GdpmError) as e:
            G.gdpm_microbench(ctx, kind, buf, slots, n)
        assert e.value.code == G.GDPM_E_ARG
    with pytest.raises(G.GdpmError) as e:                 # host memory
        G.gdpm_microbench(ctx, 0, torch.zeros(16, dtype=torch.float64), 16, 100)
    assert e.value.code == G.GDPM_E_ARG
