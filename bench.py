#!/usr/bin/env python
"""Throughput benchmark of the GB300 gDPM engine.

Workload (default, ``ct256_imrt7``): the 256x256x128 patient-like CT phantom
at 0.25 cm (seeded ellipsoids: body, lungs, spine and ribs, an air cavity)
under a 7-beam coplanar IMRT plan, each beam a 20x20 fluence map of 1 cm
beamlets with seeded intensities, 6 MV-like spectrum (Kramers thick target,
24 equal intervals), SAD 100 cm, cutoffs 50 keV / 200 keV, 1e8 histories in
100 batches, FP32 transport with FP64 tallies.  One step = one full dose
calculation of that workload (all batches, statistics and sigma/Dmax); the
line also carries the time to sigma/Dmax = 1 % measured by running to it and,
under "serving", the request latency (p50/p99) and histories/s of a serving
mix on the same phantom at 130 % of its capacity, served continuously and one
request at a time (``--no-serve`` leaves it out).
``--workload slab128_6MV`` is the 128^3 water/lung/bone/water slab with a
10x10 cm field at SSD 100 cm.

Prints one JSON line.  ``--impl reference`` times the CPU oracle instead.
Under torchrun each rank runs the same workload with its own Philox key
(independent histories, no data exchange): weak scaling.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1107_3355_gb300 import workloads as W  # noqa: E402

WORKLOADS = {
    "slab128_6MV": lambda n, nb: W.slab_photon_problem(n_histories=n, n_batches=nb),
    "ct256_imrt7": lambda n, nb: W.ct_imrt_problem(n_histories=n, n_batches=nb),
    "slab128_e20MeV": lambda n, nb: W.slab_electron_problem(n_histories=n, n_batches=nb),
    "water32_1MeV_pencil": lambda n, nb: W.tiny_problem(n_histories=n, n_batches=nb),
    # the phantom cases of Sec. 3.1 (Tables 1 and 2), the paper's own geometry
    "paper_slab_e20_lung": lambda n, nb: W.paper_slab_problem("lung", W.ELECTRON, n, nb),
    "paper_slab_e20_bone": lambda n, nb: W.paper_slab_problem("bone", W.ELECTRON, n, nb),
    "paper_slab_6MV_lung": lambda n, nb: W.paper_slab_problem("lung", W.PHOTON, n, nb),
    "paper_slab_6MV_bone": lambda n, nb: W.paper_slab_problem("bone", W.PHOTON, n, nb),
    # the comparison case of Sec. 4: 64^3 water, 15 MeV beams, annihilation off
    "water64_e15": lambda n, nb: W.water64_problem(W.ELECTRON, n, nb),
    "water64_g15": lambda n, nb: W.water64_problem(W.PHOTON, n, nb),
}
# histories and batches of a step when not given: the paper's for its cases
DEFAULT_SIZE = {"paper_slab_e20_lung": (2.5e6, 10), "paper_slab_e20_bone": (2.5e6, 10),
                "paper_slab_6MV_lung": (2.5e8, 10), "paper_slab_6MV_bone": (2.5e8, 10),
                "water64_e15": (1e6, 10), "water64_g15": (4e6, 10)}
# The paper's GPU throughput on its Table 2 cases and its Sec. 4 comparison
# case (histories / T_GPU, Tesla C2050, transfers included): the published
# numbers these workloads compare to.
PAPER_RATE = {"paper_slab_e20_lung": 2.5e6 / 1.70, "paper_slab_e20_bone": 2.5e6 / 1.65,
              "paper_slab_6MV_lung": 2.5e8 / 16.1, "paper_slab_6MV_bone": 2.5e8 / 20.5,
              "water64_e15": 1e6 / 0.47, "water64_g15": 4e6 / 0.90}
PHANTOM_DESC = {"slab128_6MV": "128^3 slab @0.25cm", "slab128_e20MeV": "128^3 slab @0.25cm",
                "ct256_imrt7": "256x256x128 ellipsoid CT @0.25cm",
                "water32_1MeV_pencil": "32^3 water @0.5cm"}
for _k in DEFAULT_SIZE:
    PHANTOM_DESC[_k] = "61x61x150 slab @0.5x0.5x0.2cm (Sec. 3.1), %s middle" % _k.rsplit("_", 1)[1]
PHANTOM_DESC["water64_e15"] = PHANTOM_DESC["water64_g15"] = "64^3 water @0.5cm (Sec. 4)"

# Nominal algorithmic FP32 work per unit of the method's steps: a Woodcock
# flight about 30 operations, a Klein-Nishina interaction about 60, an
# electron condensed-history step about 100 (its voxel crossings, range
# inverse and angular deflection included).  The roofline fraction `frac` is
# taken with these; units come from the engine's own event counters.
NOMINAL_OPS = {"ph_flights": 30, "compton": 60, "el_steps": 100}

# Detailed count of the same steps as this engine executes them (FP32
# arithmetic, integer arithmetic of the Philox rounds and index math, and
# special-function calls, one each), reported beside `frac` as
# `frac_detailed`: it adds the random-number generation (Philox4x32-10 per
# four uniforms) and prices voxel crossings and hard events separately.
OPS_PER_DRAW = 72          # Philox4x32-10 (10 rounds x 6 ops) + 4 uniform conversions x 3
OPS = {
    "ph_flights": 32 + OPS_PER_DRAW + 10,     # Woodcock flight: lerps, log, move, voxel, test
    "compton": 96 + int(1.4 * OPS_PER_DRAW),  # KN sampling (~1.4 trials), rotation, recoil
    "el_steps": 143 + OPS_PER_DRAW + 12,      # CH step: limits, range inverse, MS angle, hinge
    "crossings": 23 + 8,                      # DDA voxel crossing with its deposit
    "moller": 120 + int(2.5 * OPS_PER_DRAW),  # candidate + Moller sampling + two rotations
    "brems": 25 + OPS_PER_DRAW,               # candidate + 1/k sampling
}
LANES_PER_SM = 128

HERE = os.path.dirname(os.path.abspath(__file__))

# DRAM bytes (read + write) per source history of the phase kernels, from
# one ncu capture per workload (dram__bytes_read.sum + dram__bytes_write.sum
# over every launch of the kernel in one calculation, divided by its
# histories; profiles/ holds the summaries).  A capture may be of a smaller
# history count than the bench step: the per-launch figure is then the
# per-history bytes times the step's histories over the step's launches of
# that kernel.  They hold while the kernel sources hash to `sha1`; otherwise
# traffic is null.
TRAFFIC_SOURCES = ("transport.cu", "common.cuh", "internal.h")
TRAFFIC = {
    # profiles/dram_k_phase_ct256_imrt7_2e6hist.md: 2e6 histories, 10 batches
    # side by side, 4 launches of each phase kernel
    "ct256_imrt7": {"tally": "fp64", "sha1": "31312f47325a5bfd8a40fe10bd545f4941ec33d6",
                    "bytes_per_history": {"electron phase": 338.9, "photon phase": 337.5}},
}


def sources_sha1():
    import hashlib
    h = hashlib.sha1()
    for f in TRAFFIC_SOURCES:
        with open(os.path.join(HERE, "paper_1107_3355_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def measured_traffic(args, kernel, launches_per_step):
    """DRAM bytes per launch of the named kernel, scaled from the workload's
    ncu capture, or None when there is none for this workload and tally
    mode, or the kernels changed since."""
    cap = TRAFFIC.get(args.workload)
    if not cap or args.tally != cap["tally"] or kernel not in cap["bytes_per_history"]:
        return None
    if sources_sha1() != cap["sha1"] or launches_per_step <= 0:
        return None
    return cap["bytes_per_history"][kernel] * float(args.histories) / launches_per_step


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gdpm", choices=["gdpm", "reference"])
    ap.add_argument("--workload", default="ct256_imrt7", choices=sorted(WORKLOADS))
    ap.add_argument("--histories", type=float, default=None,
                    help="histories per step (default 1e8; the paper's count for its cases)")
    ap.add_argument("--batches", type=int, default=None,
                    help="batches (default 100; 10 for the paper's cases)")
    ap.add_argument("--tally", default="fp64", choices=["fp64", "fp32pair"],
                    help="dose tally: FP64 atomics, or FP32 hi/lo compensated pairs")
    ap.add_argument("--electron-walk", type=int, default=None, choices=[0, 1],
                    help="electron phase form (GDPM_PARAM_ELECTRON_WALK): 1 resumable steps "
                         "(the library's default), 0 a whole step per loop iteration")
    ap.add_argument("--autotune-ms", type=float, default=0.0,
                    help="run gdpm_autotune on the step's calculation for this wall-clock "
                         "budget before the warm-up, and time the configuration it sets")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--no-serve", action="store_true",
                    help="leave out the serving comparison the default line carries")
    ap.add_argument("--serve-line-requests", type=int, default=120,
                    help="requests of the serving comparison on the default line (130 %% load)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-run-to-1pct", action="store_true",
                    help="skip the measured run to 1 %% (e.g. for a launch list of the timed steps)")
    ap.add_argument("--mode", default="throughput", choices=["throughput", "serve", "beamlets",
                                                             "resources"])
    ap.add_argument("--matrix-beamlets", type=int, default=400)
    ap.add_argument("--matrix-batches", type=int, default=2)
    ap.add_argument("--graph", type=int, default=0, choices=[0, 1],
                    help="beamlet mode: run the phases as one CUDA graph with a conditional "
                         "WHILE node (GDPM_PARAM_GRAPH; per-kernel times are then not taken)")
    ap.add_argument("--serve-requests", type=int, default=60)
    ap.add_argument("--serve-load", type=float, default=0.7)
    ap.add_argument("--serve-arc-histories", type=float, default=5e8)
    ap.add_argument("--serve-slots", type=int, default=4)
    ap.add_argument("--serve-big-slots", type=int, default=1)
    ap.add_argument("--serve-phase-cap", type=float, default=0.0)
    ap.add_argument("--serve-share", type=int, default=7)
    ap.add_argument("--serve-seed", type=int, default=3)
    args = ap.parse_args()
    h, nb = DEFAULT_SIZE.get(args.workload, (1e8, 100))
    if args.histories is None:
        args.histories = h
    if args.batches is None:
        args.batches = nb
    return args


# ---------------------------------------------------------------- clocks
class Clocks:
    """nvidia-smi samples of the SM clock and throttle reasons every 100 ms.
    Start it before the warm-up (nvidia-smi takes a while to come up), mark
    the timed region with begin()/end(); stop() keeps the samples whose
    timestamps fall inside that region."""
    FIELDS = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.path = tempfile.mktemp(prefix="gdpm_clk_", suffix=".csv")
        self.proc = None
        self.t0 = self.t1 = None

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "100"], stdout=self.f,
                stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def begin(self):
        self.t0 = time.time()

    def end(self):
        self.t1 = time.time()

    @staticmethod
    def _stamp(text):
        import datetime
        try:
            return datetime.datetime.strptime(text, "%Y/%m/%d %H:%M:%S.%f").timestamp()
        except ValueError:
            return None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        if self.t1 is None:
            self.end()
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        window = "timed region"
        if self.t0 is not None:
            inside = [r for r in rows if (self._stamp(r[0]) or 0.0) >= self.t0 - 0.05 and
                      (self._stamp(r[0]) or 0.0) <= self.t1 + 0.05]
            if inside:
                rows = inside
            else:
                window = "no sample inside the timed region: all samples of the run"
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None

        sm = [num(r[1]) for r in rows if num(r[1])]
        mx = [num(r[2]) for r in rows if num(r[2])]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows), "window": window}


# ---------------------------------------------------------------- CPU oracle
def oracle_rate(prob_fn, seconds, first_n=2000):
    """Time the CPU oracle (single thread) on a bounded sample of the workload."""
    from oracle import oracle as O
    O.build()
    n = first_n
    while True:
        t0 = time.perf_counter()
        O.run(prob_fn(n))
        dt = time.perf_counter() - t0
        if dt >= seconds or n >= 10_000_000:
            return n, dt
        n = int(max(n * 2, n * seconds / max(dt, 1e-3) * 1.1))


def _oracle_worker(workload, n, rid, steps, barrier, out):
    """One single-thread oracle process: `steps` runs of n histories on its
    own random stream (request id rid), each started at a shared barrier."""
    from oracle import oracle as O
    O.run(WORKLOADS[workload](200, 10).with_(request_id=rid))       # load the library
    prob = WORKLOADS[workload](n, 10).with_(request_id=rid)
    for _ in range(steps):
        barrier.wait(timeout=600)
        t0 = time.perf_counter()
        O.run(prob)
        out.put((n, time.perf_counter() - t0))


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_rate_parallel(workload, n_per_proc, procs, steps=1):
    """Time the CPU oracle as `procs` independent single-thread processes on
    disjoint history streams, started together (the paper's multi-processor
    runs summed independent jobs the same way).  Spawned, so a process that
    already holds a CUDA context can call it.  Returns histories/s of all
    processes together, one value per step."""
    import multiprocessing as mp
    from oracle import oracle as O
    O.build()
    ctx = mp.get_context("spawn")
    barrier = ctx.Barrier(procs)
    out = ctx.Queue()
    ps = [ctx.Process(target=_oracle_worker, args=(workload, n_per_proc, 1 + w, steps, barrier, out))
          for w in range(procs)]
    for p in ps:
        p.start()
    rates = []
    try:
        for _ in range(steps):
            res = [out.get(timeout=1200) for _ in range(procs)]
            rates.append(sum(n for n, _ in res) / max(dt for _, dt in res))
    finally:
        for p in ps:
            p.join(timeout=60)
        for p in ps:
            if p.is_alive():
                p.terminate()
    return rates


def serve_bench(args):
    """Request stream on the patient-like phantom (Poisson arrivals, seeded):
    60 % single beamlets (1e5 histories), 30 % full fluence-map beams (1e7),
    10 % VMAT arcs (180 control points, MLC apertures).  Served with
    continuous batching (gdpm_request_submit/poll, several slots) and one at a
    time with plain gdpm_simulate calls; same requests, same histories."""
    print(json.dumps(serve_measure(args, args.serve_requests, args.serve_load)))


def serve_measure(args, n_requests, load):
    """The serving comparison of serve_bench for n_requests at offered load
    `load` (relative to the mix's capacity); returns its JSON object."""
    import numpy as np
    import torch
    from paper_1107_3355_gb300 import gdpm as G

    rng = np.random.default_rng(args.serve_seed)
    ph = W.ct_phantom()
    base = W.Problem(ph, W.single_beamlet(ph, 0.0, 0.0, 0.0, 1.0), 100, 10, eabs_photon=0.05,
                     eabs_electron=0.2, e_min=0.005, e_max=6.5)
    iso = tuple(e / 2 for e in ph.extent)
    reqs = []
    for k in range(n_requests):
        r = rng.uniform()
        ang = float(rng.uniform(0, 360))
        if r < 0.6:
            u, v = rng.uniform(-8, 7, 2)
            reqs.append(("beamlet", W.single_beamlet(ph, ang, float(u), float(v), 1.0), 100_000))
        elif r < 0.9:
            fr = W.beam_frame(ang, iso)
            rows = W.fluence_map_rows(fr, rng.uniform(0, 1, (20, 20)), 1.0)
            reqs.append(("beam", W.beamlet_source(rows, W.kramers_spectrum()), 10_000_000))
        else:
            reqs.append(("arc", W.vmat_arc(ph, seed=int(rng.integers(1 << 30))),
                         int(args.serve_arc_histories)))
    eng = G.Engine(base)
    ctx = eng.ctx
    V = ph.n_voxels
    dose = torch.empty(V, dtype=torch.float64, device="cuda")
    sig = torch.empty(V, dtype=torch.float64, device="cuda")
    # capacity of the mix for the arrival process: one request of each kind
    # served alone (after a warm-up), weighted by how often the stream holds it
    service = {}
    for kind in ("beamlet", "beam", "arc"):
        sample = next(((src, n) for k, src, n in reqs if k == kind), None)
        if sample is None:
            continue
        G.gdpm_source_set(ctx, sample[0])
        G.gdpm_simulate(ctx, eng.phantom, eng.tables, min(sample[1], 2_000_000), 10, dose, sig)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        G.gdpm_simulate(ctx, eng.phantom, eng.tables, sample[1], 10, dose, sig)
        torch.cuda.synchronize()
        service[kind] = time.perf_counter() - t0
    busy = sum(service[k] for k, _, _ in reqs)
    total_hist = sum(n for _, _, n in reqs)
    rate = total_hist / busy                       # histories/s of the mix served alone
    mean_hist = total_hist / len(reqs)
    lam = load * rate / mean_hist
    arrivals = np.cumsum(rng.exponential(1.0 / lam, len(reqs)))

    # (a) one at a time, plain gdpm_simulate calls in arrival order
    lat_a = []
    start = time.perf_counter()
    for k, (kind, src, n) in enumerate(reqs):
        now = time.perf_counter() - start
        if now < arrivals[k]:
            time.sleep(arrivals[k] - now)
        G.gdpm_source_set(ctx, src)
        G.gdpm_simulate(ctx, eng.phantom, eng.tables, n, 10, dose, sig)
        lat_a.append(time.perf_counter() - start - arrivals[k])
    span_a = time.perf_counter() - start

    # (b) continuous batching through the request loop
    G.gdpm_set_param(ctx, G.GDPM_PARAM_SERVE_SLOTS, args.serve_slots)
    G.gdpm_set_param(ctx, G.GDPM_PARAM_SERVE_BIG_SLOTS, args.serve_big_slots)
    G.gdpm_set_param(ctx, G.GDPM_PARAM_SERVE_PHASE_CAP, args.serve_phase_cap)
    G.gdpm_set_param(ctx, G.GDPM_PARAM_SERVE_SHARE, args.serve_share)
    import threading
    ids = [None] * len(reqs)
    done_at = [None] * len(reqs)
    start = time.perf_counter()

    def submitter():
        for k, (kind, src, n) in enumerate(reqs):
            now = time.perf_counter() - start
            if now < arrivals[k]:
                time.sleep(arrivals[k] - now)
            ids[k] = G.gdpm_request_submit(ctx, eng.phantom, eng.tables, src, n, 10)

    th = threading.Thread(target=submitter)
    th.start()
    outstanding = set(range(len(reqs)))
    while outstanding:
        for k in list(outstanding):
            if ids[k] is None:
                continue
            fin, _ = G.gdpm_request_poll(ctx, ids[k], dose, sig)
            if fin:
                done_at[k] = time.perf_counter() - start
                outstanding.discard(k)
        time.sleep(0.0005)
    th.join()
    span_b = time.perf_counter() - start
    lat_b = [done_at[k] - arrivals[k] for k in range(len(reqs))]
    eng.close()

    def pct(x, q):
        return float(np.percentile(np.asarray(x) * 1e3, q))

    def by_kind(lat):
        out = {}
        for kind in ("beamlet", "beam", "arc"):
            xs = [l for (k, _, _), l in zip(reqs, lat) if k == kind]
            if xs:
                out[kind] = {"n": len(xs), "p50_ms": pct(xs, 50), "p99_ms": pct(xs, 99)}
        return out

    line = {"metric": "p50/p99 request latency", "unit": "ms", "mode": "serve",
            "value": pct(lat_b, 99), "higher_is_better": False, "n_gpus": 1,
            "data": "synthetic",
            "config": {"workload": "ct256_serving_mix", "requests": len(reqs),
                       "mix": "60%% beamlet 1e5, 30%% beam 1e7, 10%% VMAT arc %.0e" % args.serve_arc_histories,
                       "load": load, "slots": args.serve_slots,
                       "big_slots": args.serve_big_slots, "phase_cap": args.serve_phase_cap,
                       "share_eighths": args.serve_share, "batches": 10,
                       "load_basis": "offered histories/s over the mix's capacity, each kind "
                                     "timed once alone: %s s" % {k: round(v, 4) for k, v in service.items()}},
            "continuous": {"p50_ms": pct(lat_b, 50), "p99_ms": pct(lat_b, 99),
                           "histories_per_s": total_hist / span_b, "makespan_s": span_b,
                           "by_kind": by_kind(lat_b)},
            "one_at_a_time": {"p50_ms": pct(lat_a, 50), "p99_ms": pct(lat_a, 99),
                              "histories_per_s": total_hist / span_a, "makespan_s": span_a,
                              "by_kind": by_kind(lat_a)},
            "calibrated_histories_per_s": rate, "total_histories": int(total_hist)}
    return line


def beamlet_matrix_bench(args):
    """Beamlet dose matrix on the 128^3 slab: 400 beamlets (sides U{0.5, 1,
    1.5, 2} cm, centres within +-8 cm, log-uniform 1e5..5e6 histories each,
    seed 7), one tally per beamlet.  Timed as one gdpm_simulate_beamlets call
    (all beamlets in one sequence of phases) and as 400 gdpm_simulate calls,
    one beamlet at a time; same histories either way."""
    import numpy as np
    import torch
    from paper_1107_3355_gb300 import gdpm as G

    nb = args.matrix_batches
    prob = W.beamlet_matrix_problem(n_beamlets=args.matrix_beamlets, n_batches=nb)
    K, V, total = len(prob.sub_histories), prob.phantom.n_voxels, prob.n_histories
    eng = G.Engine(prob, params={G.GDPM_PARAM_PROFILE: 0 if args.graph else 1,
                                 G.GDPM_PARAM_GRAPH: args.graph})
    dose = torch.empty((K, V), dtype=torch.float64, device="cuda")
    sigma = torch.empty((K, V), dtype=torch.float64, device="cuda") if nb >= 2 else None
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    clocks = Clocks(0)
    clocks.start()
    for _ in range(args.warmup):
        G.gdpm_simulate_beamlets(eng.ctx, eng.phantom, eng.tables, prob.sub_histories, nb, dose, sigma)
    torch.cuda.synchronize()
    clocks.begin()
    stream = torch.cuda.current_stream()
    ms = []
    for k in range(args.steps):
        flush.fill_(float(k))
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st = G.gdpm_simulate_beamlets(eng.ctx, eng.phantom, eng.tables, prob.sub_histories, nb, dose, sigma)
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    clocks.end()
    clk = clocks.stop()
    batched = total / (float(np.median(ms)) / 1e3)
    # one beamlet at a time (dose of each beamlet alone, 2 batches: the
    # smallest a single calculation allows)
    one = torch.empty(V, dtype=torch.float64, device="cuda")
    single = W.beamlet_source(prob.source.beamlets[:1], prob.source.spectrum)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(K):
        single.beamlets = prob.source.beamlets[k:k + 1]
        G.gdpm_source_set(eng.ctx, single)
        G.gdpm_simulate(eng.ctx, eng.phantom, eng.tables, int(prob.sub_histories[k]), 2, one, None)
    torch.cuda.synchronize()
    serial = total / (time.perf_counter() - t0)
    eng.close()
    line = {"metric": "histories/s", "mode": "beamlet_matrix", "value": batched,
            "unit": "histories/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": float(np.median(ms)), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "slab128_beamlet_matrix", "beamlets": K, "histories": total,
                       "batches": nb, "outputs": "dose and sigma per beamlet" if nb >= 2 else "dose per beamlet",
                       "tally": "%d FP64 grids per beamlet (%.1f GB)" % (nb, nb * K * V * 8 / 1e9),
                       "l2": "flushed between steps (256 MB write)",
                       "phase_loop": "CUDA graph (conditional WHILE node)" if args.graph else "host"},
            "one_beamlet_at_a_time": {"value": serial, "unit": "histories/s",
                                      "calls": K, "batches_per_call": 2},
            "kernel_ms_per_step": list(st["kernel_ms"]),
            "gpu_launches": int(st["launches"]), "clocks": clk}
    print(json.dumps(line))


def rank_env():
    """(world size, rank, local rank) as torchrun sets them (1, 0, 0 alone)."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def max_over_ranks(value, world, device=None):
    """The largest value over all ranks (the timed region of the slowest rank)."""
    if world == 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world, steps, n_hist, t_max_ms):
    """Histories per second of the whole job: every rank runs n_hist histories
    per step (replicas with disjoint random streams), timed by the slowest."""
    return world * steps * n_hist / (t_max_ms / 1e3)


def resources_bench(args):
    """Rates of the resources behind the transport kernels (gdpm_microbench):
    scattered atomic adds into arrays from 32K cells (contended) to 64M cells
    (larger than L2), and FP32 FMA, FP64 FMA and MUFU issue.  Best of three
    launches each; one JSON line."""
    import torch
    from paper_1107_3355_gb300 import gdpm as G
    ctx = G.gdpm_context_create(0, torch.cuda.current_stream().cuda_stream, 1)
    out = {}
    try:
        for kind in ("red_f64", "red_f32", "atom_f32"):
            for n in (32768, 262144, 2097152, 8388608, 67108864):
                dt = torch.float64 if kind == "red_f64" else torch.float32
                buf = torch.zeros(n, dtype=dt, device="cuda")
                out["%s_%dcells_per_s" % (kind, n)] = max(
                    G.gdpm_microbench(ctx, kind, buf, n, int(2e9))[0] for _ in range(3))
                del buf
        sink = torch.zeros(1, dtype=torch.float32, device="cuda")
        for kind, n in (("ffma", 2e11), ("dfma", 2e9), ("mufu_lg2", 4e10)):
            out[kind + "_per_s"] = max(G.gdpm_microbench(ctx, kind, sink, 1, int(n))[0] for _ in range(3))
    finally:
        G.gdpm_context_destroy(ctx)
    props = torch.cuda.get_device_properties(0)
    print(json.dumps({"mode": "resources", "sms": props.multi_processor_count,
                      "lane_peak_at_2070MHz_per_s": props.multi_processor_count * LANES_PER_SM * 2.07e9,
                      "rates": out}))


def main():
    args = parse()
    if args.mode == "resources":
        resources_bench(args)
        return
    if args.mode == "serve":
        serve_bench(args)
        return
    if args.mode == "beamlets":
        beamlet_matrix_bench(args)
        return
    world, rank, local = rank_env()
    n_hist = int(args.histories)
    make = WORKLOADS[args.workload]
    config = {"workload": args.workload, "histories_per_step": n_hist, "batches": args.batches,
              "phantom": PHANTOM_DESC[args.workload],
              "l2": "flushed between steps (256 MB write)", "tally": args.tally,
              "parallelism": "replicas" if world > 1 else "single GPU"}

    if args.impl == "reference":
        if rank != 0:
            return
        # one core calibrates the sample; then every host core runs the
        # oracle as its own process, about 3 s per step
        n1, dt1 = oracle_rate(lambda k: make(k, 10), max(args.cpu_seconds / 3, 1.0))
        procs = host_cores()
        per = max(2000, int(3.0 * n1 / dt1))
        vals = oracle_rate_parallel(args.workload, per, procs, args.steps)
        v = statistics.median(vals)
        config = dict(config, parallelism="%d single-thread CPU processes" % procs, tally="fp64 (oracle)")
        sample = per * procs
        line = {"impl": "reference", "metric": "histories/s", "value": v, "unit": "histories/s",
                "n_gpus": 0, "steps": args.steps, "warmup": 0, "ms_per_step": 1e3 * sample / v,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic", "config": config,
                "cpu_baseline": {"value": v, "unit": "histories/s", "cores": procs, "kind": "oracle",
                                 "sample": "%d single-thread processes x %d histories of the "
                                           "workload per step, 10 batches, disjoint streams"
                                           % (procs, per),
                                 "single_core_value": n1 / dt1},
                "e2e": {"value": v, "unit": "histories/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return

    import torch
    from paper_1107_3355_gb300 import gdpm as G

    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    prob = make(n_hist, args.batches).with_(request_id=rank)
    params = {G.GDPM_PARAM_PROFILE: 1, G.GDPM_PARAM_TALLY_MODE: 1 if args.tally == "fp32pair" else 0}
    if args.electron_walk is not None:
        params[G.GDPM_PARAM_ELECTRON_WALK] = args.electron_walk
        config["electron_walk"] = args.electron_walk
    eng = G.Engine(prob, device=local, params=params)
    if args.autotune_ms > 0:
        tuned = G.gdpm_autotune(eng.ctx, eng.phantom, eng.tables, n_hist, args.batches,
                                budget_ms=args.autotune_ms)
        G.gdpm_set_param(eng.ctx, G.GDPM_PARAM_PROFILE, 1)
        config["autotuned"] = {k: tuned[k] for k in ("batch_mode", "source_chunk", "speculative",
                                                     "electron_walk", "block_threads",
                                                     "queue_capacity", "graph")}
    V = prob.phantom.n_voxels
    dose = torch.empty(V, dtype=torch.float64, device=dev)
    sigma = torch.empty(V, dtype=torch.float64, device=dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    clocks = Clocks(local)
    clocks.start()
    for _ in range(args.warmup):
        eng.run(dose=dose, sigma=sigma)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize(dev)

    barrier()
    clocks.begin()
    stream = torch.cuda.current_stream(dev)
    total_ms = 0.0
    agg = {}
    for k in range(args.steps):
        flush.fill_(float(k))
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        _, _, st = eng.run(dose=dose, sigma=sigma)
        e1.record(stream)
        e1.synchronize()
        total_ms += e0.elapsed_time(e1)
        for key, v in st.items():
            if isinstance(v, list):
                agg[key] = [a + b for a, b in zip(agg.get(key, [0] * len(v)), v)]
            elif isinstance(v, (int, float)):
                agg[key] = agg.get(key, 0) + v
        last = st
    barrier()
    clocks.end()
    clk = clocks.stop()
    t_max = max_over_ranks(total_ms, world, dev)
    value = whole_job_rate(world, args.steps, n_hist, t_max)

    # end to end through the C ABI with host buffers: tables, phantom upload
    # (pinned host), source, simulate into host outputs
    import numpy as np
    mat_h = torch.from_numpy(np.ascontiguousarray(prob.phantom.mat)).pin_memory()
    rho_h = torch.from_numpy(np.ascontiguousarray(prob.phantom.rho)).pin_memory()
    dose_h = torch.empty(V, dtype=torch.float64).pin_memory()
    sig_h = torch.empty(V, dtype=torch.float64).pin_memory()
    ctx = eng.ctx
    e2e_s = 0.0
    for k in range(args.e2e_steps):
        flush.fill_(float(k))
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        tb = G.gdpm_tables_build(ctx, prob.phantom.materials, prob.e_min, prob.e_max, prob.n_energy,
                                 prob.eabs_photon, prob.eabs_electron, prob.ms_loss_fraction,
                                 G.table_flags(prob))
        ph = G.gdpm_phantom_create(ctx, prob.phantom.shape, prob.phantom.voxel, mat_h, rho_h)
        G.gdpm_source_set(ctx, G.problem_source(prob))
        G.gdpm_simulate(ctx, ph, tb, n_hist, args.batches, dose_h, sig_h)
        G.gdpm_phantom_destroy(ph)
        G.gdpm_tables_destroy(tb)
        e2e_s += time.perf_counter() - t0
    e2e_s = max_over_ranks(e2e_s, world, dev)          # the slowest rank's end-to-end time

    # time to 1 % measured by running to it: a pilot of up to 5e7 histories,
    # then runs of the histories sigma/Dmax ~ N^(-1/2) predicts (wall clock,
    # device outputs, after the timed region)
    run_to_1pct = None
    if not args.no_run_to_1pct:
        pilot = min(n_hist, 50_000_000)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        st1, total1 = G.gdpm_simulate_to_precision(eng.ctx, eng.phantom, eng.tables, 0.01, pilot,
                                                   2 ** 32 - 1, args.batches, dose, sigma)
        torch.cuda.synchronize(dev)
        run_to_1pct = {"s": time.perf_counter() - t0, "pilot_histories": pilot,
                       "histories_last_run": st1["n_primary"], "histories_all_runs": total1,
                       "sigma_over_dmax": st1["sigma_over_dmax"]}
    e2e_value = world * args.e2e_steps * n_hist / e2e_s if args.e2e_steps > 0 else None

    # roofline of the dominant kernel kind, from its live event time
    kinds = ["photon phase", "electron phase", "batch fold"]
    kms = agg.get("kernel_ms", [0, 0, 0, 0])
    dom = max(range(3), key=lambda i: kms[i])
    if dom == 0:
        ops = agg["ph_flights"] * NOMINAL_OPS["ph_flights"] + agg["compton"] * NOMINAL_OPS["compton"]
        ops_detailed = agg["ph_flights"] * OPS["ph_flights"] + agg["compton"] * OPS["compton"]
    else:
        ops = agg["el_steps"] * NOMINAL_OPS["el_steps"]
        ops_detailed = (agg["el_steps"] * OPS["el_steps"] + agg["crossings"] * OPS["crossings"] +
                        agg["moller"] * OPS["moller"] + agg["brems"] * OPS["brems"])
    launches_dom = max(1, agg.get("kernel_launches", [1, 1, 1, 1])[dom])
    achieved = ops / (kms[dom] / 1e3) / 1e12
    achieved_detailed = ops_detailed / (kms[dom] / 1e3) / 1e12
    props = torch.cuda.get_device_properties(dev)
    sm_mhz = clk.get("sm_mhz") or 2070.0
    peak = props.multi_processor_count * LANES_PER_SM * sm_mhz * 1e6 / 1e12

    # the resources behind the roofline, measured on this GPU after the timed
    # region: FP32 FMA and MUFU issue, and scattered FP64 atomics into a
    # buffer the size of one dose grid (the tally's target)
    probe = torch.zeros(V, dtype=torch.float64, device=dev)
    ffma, _, _ = G.gdpm_microbench(ctx, "ffma", probe, 1, int(1e11))
    mufu, _, _ = G.gdpm_microbench(ctx, "mufu_lg2", probe, 1, int(2e10))
    red64, _, _ = G.gdpm_microbench(ctx, "red_f64", probe, V, int(2e9))
    del probe
    # tally atomics of the electron phase: a track tallies once per voxel it
    # leaves and once where it stops (at most crossings + terminations)
    tally_n = agg["crossings"] + agg["el_terminated"]
    tally_rate = tally_n / (kms[1] / 1e3) if kms[1] > 0 else 0.0
    resources = {"ffma_Tops": ffma / 1e12, "mufu_lg2_Tops": mufu / 1e12,
                 "red_f64_Gops": red64 / 1e9,
                 "tally_atomics_Gops": tally_rate / 1e9,
                 "tally_frac_of_red_f64": tally_rate / red64 if red64 > 0 else None,
                 "note": "measured by gdpm_microbench after the timed region; tally atomics "
                         "counted as voxel crossings + electron terminations (an upper bound)"}

    sig = last["sigma_over_dmax"]
    n_to_1pct = n_hist * (sig / 0.01) ** 2 if sig > 0 else float("nan")
    t_to_1pct = n_to_1pct / (value / world) if value > 0 else float("nan")

    line = {"metric": "histories/s", "value": value, "unit": "histories/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_max / args.steps,
            "higher_is_better": True, "scaling": "weak",
            "vs_baseline": (value / PAPER_RATE[args.workload]
                            if args.workload in PAPER_RATE and n_hist == int(DEFAULT_SIZE[args.workload][0])
                            and args.batches == DEFAULT_SIZE[args.workload][1] else None),
            "dtype": "f32",
            "data": "synthetic", "config": config,
            "time_to_1pct_s": t_to_1pct,
            "time_to_1pct_run": run_to_1pct,
            "sigma_over_dmax": sig, "histories_for_1pct": n_to_1pct,
            "e2e": {"value": e2e_value, "unit": "histories/s",
                    "h2d_bytes_per_step": int(V * 5), "d2h_bytes_per_step": int(V * 16)},
            "gpu_launches": int(agg.get("launches", 0)),
            "roofline": {"bound": "alu", "kernel": kinds[dom], "achieved": achieved,
                         "peak": peak, "unit": "Tops/s", "frac": achieved / peak,
                         "traffic": measured_traffic(args, kinds[dom], launches_dom / args.steps),
                         "traffic_unit": "DRAM bytes per launch (ncu, scaled per history)",
                         "launches_per_step": launches_dom / args.steps,
                         "ops_per_unit": {k: NOMINAL_OPS[k] for k in
                                          (("ph_flights", "compton") if dom == 0 else ("el_steps",))},
                         "achieved_detailed": achieved_detailed,
                         "frac_detailed": achieved_detailed / peak,
                         "ops_per_unit_detailed": ({k: OPS[k] for k in ("ph_flights", "compton")}
                                                   if dom == 0 else
                                                   {k: OPS[k] for k in ("el_steps", "crossings",
                                                                        "moller", "brems")}),
                         "note": "ALU lane-operations/s vs SMs x 128 lanes x sampled SM clock; "
                                 "achieved = events x ops_per_unit / the kernel's summed event "
                                 "time (kernel_ms_per_step x steps)"},
            "resources": resources,
            "kernel_ms_per_step": [k / args.steps for k in kms],
            "events_per_history": {k: agg[k] / (args.steps * n_hist) for k in
                                   ("ph_flights", "compton", "el_steps", "crossings", "moller",
                                    "brems")},
            "clocks": clk}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # single core first (it also sizes the sample), then every host core
        # as an independent oracle process for about 2 s each
        n, dt = oracle_rate(lambda k: make(k, 10), args.cpu_seconds)
        procs = host_cores()
        per = max(2000, int(2.0 * n / dt))
        v = oracle_rate_parallel(args.workload, per, procs, 1)[0]
        line["cpu_baseline"] = {"value": v, "unit": "histories/s", "cores": procs,
                                "kind": "oracle",
                                "sample": "%d single-thread processes x %d histories of %s, "
                                          "10 batches, disjoint streams" % (procs, per, args.workload),
                                "single_core_value": n / dt,
                                "single_core_sample": "%d histories, one thread" % n}
    eng.close()
    if rank == 0 and world == 1 and not args.no_serve and args.workload == "ct256_imrt7":
        # the metric's request latency: the serving mix on the same phantom at
        # saturation (130 % of the mix's capacity), served continuously and
        # one request at a time
        del dose, sigma, flush
        torch.cuda.empty_cache()
        sv = serve_measure(args, args.serve_line_requests, 1.3)
        line["serving"] = {"p50_ms": sv["continuous"]["p50_ms"], "p99_ms": sv["continuous"]["p99_ms"],
                           "histories_per_s": sv["continuous"]["histories_per_s"],
                           "one_at_a_time": {k: sv["one_at_a_time"][k] for k in
                                             ("p50_ms", "p99_ms", "histories_per_s")},
                           "by_kind": sv["continuous"]["by_kind"],
                           "config": dict(sv["config"], load_basis=None),
                           "capacity_histories_per_s": sv["calibrated_histories_per_s"]}
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
