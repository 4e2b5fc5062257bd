"""Python binding of the C ABI in ``include/gdpm.h`` (argument marshalling only).

Every function here calls straight into ``libgdpm.so``; all computation runs
in the library's CUDA kernels.  There is no CPU fallback: if the library
cannot be built or loaded, or no CUDA device is present, calls raise.
PyTorch is used only for device memory and the current CUDA stream.
"""
from __future__ import annotations

import ctypes as C
import os
import threading
from typing import Optional

import numpy as np

from . import build as _build
from . import workloads as W

GDPM_OK = 0
GDPM_E_ARG, GDPM_E_NOMEM, GDPM_E_QUEUE_OVERFLOW, GDPM_E_TIMEOUT = -1, -2, -3, -4
GDPM_E_CUDA, GDPM_E_STATE, GDPM_E_BUSY, GDPM_E_BOUNDS = -5, -6, -7, -8
GDPM_PHOTON, GDPM_ELECTRON = 0, 1
GDPM_GEO_PENCIL, GDPM_GEO_POINT_FIELD, GDPM_GEO_BEAMLETS = 0, 1, 2
GDPM_FLAG_COMPTON_ONLY, GDPM_FLAG_NO_HARD, GDPM_FLAG_SAUTER = 2, 4, 8
GDPM_PARAM_QUEUE_CAPACITY = 1
GDPM_PARAM_BLOCK_THREADS = 2
GDPM_PARAM_BLOCKS_PER_SM = 3
GDPM_PARAM_TALLY_MODE = 4
GDPM_PARAM_SOURCE_CHUNK = 5
GDPM_PARAM_MAX_PHASES = 6
GDPM_PARAM_REQUEST_ID = 7
GDPM_PARAM_SPECULATIVE = 8
GDPM_PARAM_PROFILE = 10
GDPM_PARAM_OVERLAP_FOLD = 11
GDPM_PARAM_SERVE_SLOTS = 12
GDPM_PARAM_SERVE_RESERVE_MB = 13
GDPM_PARAM_METRIC_MIN_DENSITY = 14
GDPM_PARAM_BATCH_MODE = 15
GDPM_PARAM_CONCURRENT_MAX_HIST = 16
GDPM_PARAM_CONCURRENT_MAX_MB = 17
GDPM_PARAM_GRAPH = 18
GDPM_PARAM_MAX_ITERS = 19
GDPM_PARAM_ELECTRON_WALK = 20
GDPM_PARAM_SERVE_BIG_SLOTS = 21
GDPM_PARAM_SERVE_SMALL_HIST = 22
GDPM_PARAM_SERVE_PHASE_CAP = 23
GDPM_PARAM_SERVE_SHARE = 24
MICROBENCH = {"red_f64": 0, "red_f32": 1, "atom_f32": 2, "ffma": 3, "dfma": 4, "mufu_lg2": 5}
MAX_EL, MAX_MAT, MAX_BINS = 16, 8, 256

EXPORTED = ["gdpm_context_create", "gdpm_context_destroy", "gdpm_set_param",
            "gdpm_phantom_create", "gdpm_phantom_destroy", "gdpm_tables_build",
            "gdpm_tables_destroy", "gdpm_source_set", "gdpm_simulate",
            "gdpm_set_history_records", "gdpm_request_submit", "gdpm_request_poll",
            "gdpm_strerror", "gdpm_debug_philox", "gdpm_debug_sample", "gdpm_tables_export",
            "gdpm_debug_sources", "gdpm_debug_beamlets", "gdpm_simulate_noalloc",
            "gdpm_simulate_beamlets", "gdpm_autotune", "gdpm_simulate_part", "gdpm_finalize",
            "gdpm_microbench", "gdpm_simulate_to_precision"]


class gdpm_material_desc(C.Structure):
    _fields_ = [("n_elements", C.c_int), ("Z", C.c_int * MAX_EL), ("A", C.c_double * MAX_EL),
                ("mass_fraction", C.c_double * MAX_EL), ("mean_excitation_MeV", C.c_double)]


class gdpm_source_desc(C.Structure):
    _fields_ = [("particle", C.c_int), ("geometry", C.c_int),
                ("origin", C.c_double * 3), ("direction", C.c_double * 3),
                ("center", C.c_double * 3), ("axis_u", C.c_double * 3),
                ("axis_v", C.c_double * 3), ("half_u", C.c_double), ("half_v", C.c_double),
                ("n_bins", C.c_int), ("bin_edges", C.POINTER(C.c_double)),
                ("bin_weights", C.POINTER(C.c_double)), ("n_beamlets", C.c_int),
                ("beamlets", C.POINTER(C.c_double)), ("annihilation", C.c_int),
                ("beamlet_sampler", C.c_int), ("metropolis_chains", C.c_int)]

GDPM_SAMPLE_CDF, GDPM_SAMPLE_ALIAS, GDPM_SAMPLE_METROPOLIS = 0, 1, 2
SAMPLERS = {"cdf": GDPM_SAMPLE_CDF, "alias": GDPM_SAMPLE_ALIAS,
            "metropolis": GDPM_SAMPLE_METROPOLIS}


_STAT_D1 = ["source_energy", "deposited", "escaped", "discarded"]
_STAT_I = ["n_primary", "ph_created", "ph_terminated", "ph_flights", "ph_real", "compton",
           "photoelectric", "pair", "el_created", "el_terminated", "el_steps", "moller", "brems",
           "annihilations", "local_deposits"]


class gdpm_stats(C.Structure):
    _fields_ = ([(n, C.c_double) for n in _STAT_D1] + [(n, C.c_int64) for n in _STAT_I] +
                [("pushes", C.c_int64 * 2), ("pops", C.c_int64 * 2), ("phases", C.c_int64),
                 ("launches", C.c_int64), ("dmax", C.c_double), ("sigma_over_dmax", C.c_double),
                 ("transport_ms", C.c_double), ("crossings", C.c_int64),
                 ("kernel_ms", C.c_double * 4), ("kernel_launches", C.c_int64 * 4)])

    def as_dict(self):
        d = {n: getattr(self, n) for n in _STAT_D1 + _STAT_I}
        d.update(pushes=list(self.pushes), pops=list(self.pops), phases=self.phases,
                 launches=self.launches, dmax=self.dmax, sigma_over_dmax=self.sigma_over_dmax,
                 transport_ms=self.transport_ms, crossings=self.crossings,
                 kernel_ms=list(self.kernel_ms), kernel_launches=list(self.kernel_launches))
        return d


class gdpm_request_desc(C.Structure):
    _fields_ = [("phantom", C.c_void_p), ("tables", C.c_void_p), ("source", gdpm_source_desc),
                ("n_histories", C.c_uint64), ("n_batches", C.c_int), ("stream_id", C.c_uint32)]


_lib = None
_lock = threading.Lock()


class GdpmError(RuntimeError):
    def __init__(self, code, where):
        super().__init__("%s failed: %s (%d)" % (where, gdpm_strerror(code), code))
        self.code = code


def checked_build() -> bool:
    """True when GDPM_CHECKED=1 in the environment: this process loads the
    bounds-checked library (libgdpm_checked.so) instead of libgdpm.so."""
    return os.environ.get("GDPM_CHECKED", "0") == "1"


def library_path() -> str:
    return _build.LIB_CHECKED if checked_build() else _build.LIB


def lib():
    """Load libgdpm.so, or libgdpm_checked.so under GDPM_CHECKED=1 (building
    it with nvcc first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build(checked=checked_build())
            L = C.CDLL(path)
            vp, i, u64, d = C.c_void_p, C.c_int, C.c_uint64, C.c_double
            sig = {
                "gdpm_context_create": [C.POINTER(vp), i, vp, u64],
                "gdpm_context_destroy": [vp],
                "gdpm_set_param": [vp, i, d],
                "gdpm_phantom_create": [vp, i, i, i, C.c_float, C.c_float, C.c_float, vp, vp,
                                        C.POINTER(vp)],
                "gdpm_phantom_destroy": [vp],
                "gdpm_tables_build": [vp, C.POINTER(gdpm_material_desc), i, d, d, i, d, d, d, i,
                                      C.POINTER(vp)],
                "gdpm_tables_destroy": [vp],
                "gdpm_source_set": [vp, C.POINTER(gdpm_source_desc)],
                "gdpm_simulate": [vp, vp, vp, u64, i, vp, vp, C.POINTER(gdpm_stats)],
                "gdpm_set_history_records": [vp, vp, vp, u64],
                "gdpm_request_submit": [vp, C.POINTER(gdpm_request_desc), C.POINTER(u64)],
                "gdpm_request_poll": [vp, u64, C.POINTER(i), vp, vp, C.POINTER(gdpm_stats)],
                "gdpm_strerror": [i],
                "gdpm_debug_philox": [vp, vp, C.c_uint32, C.c_uint32, vp, u64],
                "gdpm_debug_sample": [vp, i, d, d, u64, u64, vp, vp],
                "gdpm_tables_export": [vp, i, vp, C.POINTER(C.c_int64)],
                "gdpm_debug_sources": [vp, vp, vp, u64, i, u64, u64, vp],
                "gdpm_debug_beamlets": [vp, u64, u64, vp],
                "gdpm_simulate_noalloc": [vp, vp, vp, u64, i, vp, vp, C.POINTER(gdpm_stats)],
                "gdpm_simulate_beamlets": [vp, vp, vp, vp, i, vp, vp, C.POINTER(gdpm_stats)],
                "gdpm_autotune": [vp, vp, vp, u64, i, d, C.POINTER(gdpm_tune_result)],
                "gdpm_simulate_part": [vp, vp, vp, u64, i, i, i, vp, vp, C.POINTER(gdpm_stats)],
                "gdpm_finalize": [vp, vp, i, vp, vp, vp, vp, C.POINTER(gdpm_stats)],
                "gdpm_microbench": [vp, i, vp, u64, u64, C.POINTER(d), C.POINTER(d)],
                "gdpm_simulate_to_precision": [vp, vp, vp, d, u64, u64, i, vp, vp, C.POINTER(gdpm_stats),
                                               C.POINTER(u64)],
            }
            for name, args in sig.items():
                f = getattr(L, name)
                f.argtypes = args
                f.restype = C.c_int
            L.gdpm_strerror.restype = C.c_char_p
            _lib = L
        return _lib


def _check(rc, where):
    if rc != GDPM_OK:
        raise GdpmError(rc, where)


def gdpm_strerror(code: int) -> str:
    return lib().gdpm_strerror(code).decode()


def _ptr(t) -> Optional[int]:
    """Data pointer of a torch tensor or numpy array (None passes NULL)."""
    if t is None:
        return None
    if hasattr(t, "data_ptr"):
        return t.data_ptr()
    return t.ctypes.data


# ------------------------------------------------------------------ C ABI calls

def gdpm_context_create(device: int = 0, stream=None, seed: int = 12345):
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("gdpm needs a CUDA device; none is available")
    if stream is None:
        stream = torch.cuda.current_stream(device)
    s = stream.cuda_stream if hasattr(stream, "cuda_stream") else stream
    h = C.c_void_p()
    _check(lib().gdpm_context_create(C.byref(h), device, s, seed), "gdpm_context_create")
    return h


def gdpm_context_destroy(ctx):
    _check(lib().gdpm_context_destroy(ctx), "gdpm_context_destroy")


def gdpm_set_param(ctx, param: int, value: float):
    _check(lib().gdpm_set_param(ctx, param, float(value)), "gdpm_set_param")


def gdpm_phantom_create(ctx, shape, voxel, material, density):
    h = C.c_void_p()
    nx, ny, nz = shape
    _check(lib().gdpm_phantom_create(ctx, nx, ny, nz, voxel[0], voxel[1], voxel[2],
                                     _ptr(material), _ptr(density), C.byref(h)),
           "gdpm_phantom_create")
    return h


def gdpm_phantom_destroy(ph):
    _check(lib().gdpm_phantom_destroy(ph), "gdpm_phantom_destroy")


def material_descs(materials):
    arr = (gdpm_material_desc * len(materials))()
    for k, m in enumerate(materials):
        arr[k].n_elements = len(m.elements)
        for j, (z, a, w) in enumerate(m.elements):
            arr[k].Z[j] = z
            arr[k].A[j] = a
            arr[k].mass_fraction[j] = w
        arr[k].mean_excitation_MeV = m.mean_excitation_MeV
    return arr


def gdpm_tables_build(ctx, materials, e_min, e_max, n_energy, eabs_photon, eabs_electron,
                      ms_loss=0.2, flags=0):
    arr = material_descs(materials)
    h = C.c_void_p()
    _check(lib().gdpm_tables_build(ctx, arr, len(materials), e_min, e_max, n_energy,
                                   eabs_photon, eabs_electron, ms_loss, flags, C.byref(h)),
           "gdpm_tables_build")
    return h


def gdpm_tables_destroy(t):
    _check(lib().gdpm_tables_destroy(t), "gdpm_tables_destroy")


class _SourceKeep:
    """A gdpm_source_desc plus the arrays its pointers refer to."""

    def __init__(self, src: "W.Source"):
        d = gdpm_source_desc()
        d.particle = src.particle
        d.geometry = {"pencil": 0, "point_field": 1, "beamlets": 2}[src.kind]
        for name in ("origin", "direction", "center", "axis_u", "axis_v"):
            getattr(d, name)[:] = [float(v) for v in getattr(src, name)]
        d.half_u, d.half_v = src.half_u, src.half_v
        self.edges = np.ascontiguousarray(src.spectrum.edges, np.float64)
        self.weights = np.ascontiguousarray(src.spectrum.weights, np.float64)
        d.n_bins = len(self.weights)
        d.bin_edges = self.edges.ctypes.data_as(C.POINTER(C.c_double))
        d.bin_weights = self.weights.ctypes.data_as(C.POINTER(C.c_double))
        self.beamlets = None
        if src.beamlets is not None:
            self.beamlets = np.ascontiguousarray(src.beamlets, np.float64)
            d.n_beamlets = self.beamlets.shape[0]
            d.beamlets = self.beamlets.ctypes.data_as(C.POINTER(C.c_double))
        d.annihilation = 1 if src.annihilation else 0
        d.beamlet_sampler = SAMPLERS[src.sampler]
        d.metropolis_chains = src.chains
        self.desc = d


def gdpm_source_set(ctx, src: "W.Source"):
    keep = _SourceKeep(src)
    _check(lib().gdpm_source_set(ctx, C.byref(keep.desc)), "gdpm_source_set")


def gdpm_simulate(ctx, phantom, tables, n_histories, n_batches, dose_out=None, sigma_out=None):
    st = gdpm_stats()
    _check(lib().gdpm_simulate(ctx, phantom, tables, n_histories, n_batches, _ptr(dose_out),
                               _ptr(sigma_out), C.byref(st)), "gdpm_simulate")
    return st.as_dict()


def gdpm_simulate_to_precision(ctx, phantom, tables, target, n_pilot, n_max, n_batches,
                               dose_out=None, sigma_out=None):
    """Run until sigma/Dmax <= target (Sec. 3.1 metric); returns (stats of
    the last run, histories of all runs)."""
    st = gdpm_stats()
    total = C.c_uint64()
    _check(lib().gdpm_simulate_to_precision(ctx, phantom, tables, target, int(n_pilot), int(n_max),
                                            n_batches, _ptr(dose_out), _ptr(sigma_out), C.byref(st),
                                            C.byref(total)), "gdpm_simulate_to_precision")
    return st.as_dict(), total.value


def gdpm_simulate_beamlets(ctx, phantom, tables, n_histories, n_batches, dose_out,
                           sigma_out=None):
    """Beamlet dose matrix: row k of the current fluence map is its own
    calculation of n_histories[k] histories; dose_out/sigma_out hold
    K x n_voxels doubles (host or device)."""
    n = np.ascontiguousarray(np.asarray(n_histories, dtype=np.uint64))
    st = gdpm_stats()
    _check(lib().gdpm_simulate_beamlets(ctx, phantom, tables, n.ctypes.data_as(C.c_void_p),
                                        n_batches, _ptr(dose_out), _ptr(sigma_out), C.byref(st)),
           "gdpm_simulate_beamlets")
    return st.as_dict()


class gdpm_tune_result(C.Structure):
    _fields_ = [("batch_mode", C.c_int), ("source_chunk", C.c_uint32), ("speculative", C.c_int),
                ("candidates_tried", C.c_int), ("histories_per_s", C.c_double),
                ("electron_walk", C.c_int), ("block_threads", C.c_int),
                ("queue_capacity", C.c_uint32), ("graph", C.c_int)]


def gdpm_autotune(ctx, phantom, tables, n_histories, n_batches, budget_ms=2000.0):
    """Try launch configurations on this calculation, keep and set the fastest;
    returns it as a dict."""
    r = gdpm_tune_result()
    _check(lib().gdpm_autotune(ctx, phantom, tables, n_histories, n_batches, budget_ms,
                               C.byref(r)), "gdpm_autotune")
    return {k: getattr(r, k) for k, _ in r._fields_}


def gdpm_simulate_part(ctx, phantom, tables, n_histories, n_batches, first_batch, n_part,
                       sum1, sum2):
    """Run batches [first_batch, first_batch+n_part) and add their per-batch
    x_b, x_b^2 into sum1, sum2 (checkpointable run state)."""
    st = gdpm_stats()
    _check(lib().gdpm_simulate_part(ctx, phantom, tables, n_histories, n_batches, first_batch,
                                    n_part, _ptr(sum1), _ptr(sum2), C.byref(st)),
           "gdpm_simulate_part")
    return st.as_dict()


def gdpm_finalize(ctx, phantom, n_batches, sum1, sum2, dose_out=None, sigma_out=None):
    """Dose and sigma from the sums of all n_batches batches."""
    st = gdpm_stats()
    _check(lib().gdpm_finalize(ctx, phantom, n_batches, _ptr(sum1), _ptr(sum2), _ptr(dose_out),
                               _ptr(sigma_out), C.byref(st)), "gdpm_finalize")
    return st.as_dict()


def gdpm_set_history_records(ctx, rec, recd, n):
    _check(lib().gdpm_set_history_records(ctx, _ptr(rec), _ptr(recd), n),
           "gdpm_set_history_records")


def gdpm_request_submit(ctx, phantom, tables, src: "W.Source", n_histories, n_batches,
                        stream_id=0):
    keep = _SourceKeep(src)
    r = gdpm_request_desc()
    r.phantom = phantom.value if hasattr(phantom, "value") else phantom
    r.tables = tables.value if hasattr(tables, "value") else tables
    r.source = keep.desc
    r.n_histories = n_histories
    r.n_batches = n_batches
    r.stream_id = stream_id
    rid = C.c_uint64()
    _check(lib().gdpm_request_submit(ctx, C.byref(r), C.byref(rid)), "gdpm_request_submit")
    return rid.value


def gdpm_request_poll(ctx, req_id, dose_out=None, sigma_out=None):
    done = C.c_int()
    st = gdpm_stats()
    _check(lib().gdpm_request_poll(ctx, req_id, C.byref(done), _ptr(dose_out), _ptr(sigma_out),
                                   C.byref(st)), "gdpm_request_poll")
    return bool(done.value), (st.as_dict() if done.value else None)


def gdpm_debug_philox(ctx, ctr, k0, k1, out, n):
    _check(lib().gdpm_debug_philox(ctx, _ptr(ctr), k0, k1, _ptr(out), n), "gdpm_debug_philox")


def gdpm_microbench(ctx, kind, buf, n_slots, n_ops):
    """Rate of one resource (MICROBENCH name or code) in operations per
    second; buf is a device tensor of n_slots cells.  Returns
    (ops/s, ops done, ms)."""
    kind = MICROBENCH.get(kind, kind)
    ops, ms = C.c_double(), C.c_double()
    _check(lib().gdpm_microbench(ctx, kind, _ptr(buf), n_slots, n_ops, C.byref(ops), C.byref(ms)),
           "gdpm_microbench")
    return ops.value / (ms.value * 1e-3), ops.value, ms.value


def gdpm_debug_sample(ctx, kind, a, b, n, seed, out1, out2=None):
    _check(lib().gdpm_debug_sample(ctx, kind, a, b, n, seed, _ptr(out1), _ptr(out2)),
           "gdpm_debug_sample")


def gdpm_tables_export(tables, which, out=None):
    cnt = C.c_int64()
    _check(lib().gdpm_tables_export(tables, which, _ptr(out), C.byref(cnt)), "gdpm_tables_export")
    return cnt.value


def gdpm_debug_sources(ctx, phantom, tables, n_histories, n_batches, first, n, out):
    _check(lib().gdpm_debug_sources(ctx, phantom, tables, n_histories, n_batches, first, n,
                                    _ptr(out)), "gdpm_debug_sources")


def gdpm_debug_beamlets(ctx, first, n, out):
    """Beamlet rows the current source's sampler picks for histories
    [first, first+n), into the device int32 array ``out``."""
    _check(lib().gdpm_debug_beamlets(ctx, first, n, _ptr(out)), "gdpm_debug_beamlets")


def gdpm_simulate_noalloc(ctx, phantom, tables, n_histories, n_batches, dose_out=None,
                          sigma_out=None):
    """gdpm_simulate for small problems without any allocation: every work
    buffer lives in the library's fixed static device array (see gdpm.h for
    the limits).  For callers that may not allocate device memory, such as
    code running under CUDA graph capture.  dose_out/sigma_out: device arrays."""
    st = gdpm_stats()
    _check(lib().gdpm_simulate_noalloc(ctx, phantom, tables, n_histories, n_batches,
                                       _ptr(dose_out), _ptr(sigma_out), C.byref(st)),
           "gdpm_simulate_noalloc")
    return st.as_dict()


# ------------------------------------------------------------------ marshalling helper

def table_flags(prob) -> int:
    """The physics switches of a Problem that belong to the tables."""
    return prob.flags & (GDPM_FLAG_COMPTON_ONLY | GDPM_FLAG_NO_HARD | GDPM_FLAG_SAUTER)


def problem_source(prob):
    """A Problem's source, with annihilation off when the Problem says so."""
    src = prob.source
    if prob.flags & W.FLAG_NO_ANNIHILATION and src.annihilation:
        import dataclasses
        src = dataclasses.replace(src, annihilation=False)
    return src


class Engine:
    """One context bound to a problem's phantom, tables and source.

    ``run()`` returns (dose, sigma, stats) with dose/sigma as torch tensors
    on the device (MeV/g per history, flat x-fastest voxel order).
    """

    def __init__(self, prob: "W.Problem", device: int = 0, seed: Optional[int] = None,
                 params: Optional[dict] = None):
        import torch
        self.prob = prob
        self.device = device
        self.ctx = gdpm_context_create(device, None, prob.seed if seed is None else seed)
        for k, v in (params or {}).items():
            gdpm_set_param(self.ctx, k, v)
        if prob.request_id:
            gdpm_set_param(self.ctx, GDPM_PARAM_REQUEST_ID, prob.request_id)
        ph = prob.phantom
        self.mat = torch.from_numpy(np.ascontiguousarray(ph.mat)).to(f"cuda:{device}")
        self.rho = torch.from_numpy(np.ascontiguousarray(ph.rho)).to(f"cuda:{device}")
        torch.cuda.synchronize(device)
        self.phantom = gdpm_phantom_create(self.ctx, ph.shape, ph.voxel, self.mat, self.rho)
        self.tables = gdpm_tables_build(self.ctx, ph.materials, prob.e_min, prob.e_max,
                                        prob.n_energy, prob.eabs_photon, prob.eabs_electron,
                                        prob.ms_loss_fraction, table_flags(prob))
        gdpm_source_set(self.ctx, problem_source(prob))

    def set_param(self, param, value):
        gdpm_set_param(self.ctx, param, value)

    def run(self, n_histories=None, n_batches=None, dose=None, sigma=None):
        import torch
        n = self.prob.n_histories if n_histories is None else n_histories
        nb = self.prob.n_batches if n_batches is None else n_batches
        V = self.prob.phantom.n_voxels
        if dose is None:
            dose = torch.empty(V, dtype=torch.float64, device=f"cuda:{self.device}")
        if sigma is None:
            sigma = torch.empty(V, dtype=torch.float64, device=f"cuda:{self.device}")
        st = gdpm_simulate(self.ctx, self.phantom, self.tables, n, nb, dose, sigma)
        return dose, sigma, st

    def run_beamlets(self, n_batches=None, with_sigma=True):
        """The problem's beamlet dose matrix (its sub_histories per fluence
        row): (dose, sigma or None, stats) with K x n_voxels device tensors."""
        import torch
        nb = self.prob.n_batches if n_batches is None else n_batches
        K, V = len(self.prob.sub_histories), self.prob.phantom.n_voxels
        dose = torch.empty((K, V), dtype=torch.float64, device=f"cuda:{self.device}")
        sigma = torch.empty((K, V), dtype=torch.float64, device=f"cuda:{self.device}") if with_sigma else None
        st = gdpm_simulate_beamlets(self.ctx, self.phantom, self.tables, self.prob.sub_histories, nb,
                                    dose, sigma)
        return dose, sigma, st

    def close(self):
        if getattr(self, "ctx", None) is not None:
            gdpm_tables_destroy(self.tables)
            gdpm_phantom_destroy(self.phantom)
            gdpm_context_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
