"""ctypes wrapper around the CPU oracle (``gdpm_oracle.c``) -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline and reference legs of
``bench.py`` use this module.  It converts a ``workloads.Problem`` into the
oracle's own C struct and calls the plain single-threaded FP64 oracle.
It imports nothing from the CUDA path.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gdpm_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

MAX_MAT, MAX_EL, MAX_BINS = 8, 16, 256
# per-history record columns
HR_PH_REAL, HR_EL_STEPS, HR_HARD, HR_BANKED, HR_NI = 0, 1, 2, 3, 4
HD_ESCAPED, HD_EL_MASSPATH, HD_ND = 0, 1, 2
# orc_eval function ids
(OF_SIGMA_KN, OF_MU_C, OF_MU_PE, OF_MU_PAIR, OF_SCOL, OF_LOSS_MOLLER, OF_SIG_MOLLER,
 OF_SREST, OF_SIG_BREMS, OF_RANGE, OF_BCONST, OF_NE, OF_G1_OF_A, OF_SOLVE_A) = range(14)
# orc_table_lookup ids
OT_MU_C, OT_MU_PE, OT_MU_PAIR, OT_SIG_M, OT_SIG_B, OT_RANGE, OT_RANGE_INV, OT_MUMAX = range(8)
# orc_sample ids
OS_KN, OS_MOLLER, OS_BREMS, OS_SR, OS_ISO, OS_SAUTER = range(6)


class OrcMaterial(C.Structure):
    _fields_ = [("n_el", C.c_int), ("Z", C.c_int * MAX_EL), ("A", C.c_double * MAX_EL),
                ("w", C.c_double * MAX_EL), ("I", C.c_double)]


class OrcProblem(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("dx", C.c_double), ("dy", C.c_double), ("dz", C.c_double),
                ("mat", C.POINTER(C.c_uint8)), ("rho", C.POINTER(C.c_float)),
                ("n_mat", C.c_int), ("mats", OrcMaterial * MAX_MAT),
                ("e_min", C.c_double), ("e_max", C.c_double), ("n_energy", C.c_int),
                ("eabs_ph", C.c_double), ("eabs_el", C.c_double), ("ms_loss", C.c_double),
                ("particle", C.c_int), ("geometry", C.c_int),
                ("origin", C.c_double * 3), ("direction", C.c_double * 3),
                ("center", C.c_double * 3), ("axis_u", C.c_double * 3),
                ("axis_v", C.c_double * 3), ("half_u", C.c_double), ("half_v", C.c_double),
                ("n_bins", C.c_int), ("edges", C.c_double * (MAX_BINS + 1)),
                ("weights", C.c_double * MAX_BINS),
                ("n_beamlets", C.c_int), ("beamlets", C.POINTER(C.c_double)),
                ("n_hist", C.c_ulonglong), ("n_batches", C.c_int), ("seed", C.c_ulonglong),
                ("request_id", C.c_uint), ("flags", C.c_int),
                ("beamlet_sampler", C.c_int), ("metro_chains", C.c_int),
                ("first_hist", C.c_ulonglong)]

SAMPLERS = {"cdf": 0, "alias": 1, "metropolis": 2}


_RESULT_FIELDS = ["source_energy", "deposited", "escaped", "discarded", "n_primary",
                  "ph_created", "ph_terminated", "ph_flights", "ph_real", "compton",
                  "photoelectric", "pair", "el_created", "el_terminated", "el_steps",
                  "moller", "brems", "annihilations", "local_deposits", "dmax",
                  "sigma_over_dmax"]


class OrcResult(C.Structure):
    _fields_ = ([(n, C.c_double) for n in _RESULT_FIELDS[:4]] +
                [(n, C.c_longlong) for n in _RESULT_FIELDS[4:19]] +
                [(n, C.c_double) for n in _RESULT_FIELDS[19:]])

    def as_dict(self):
        return {n: getattr(self, n) for n in _RESULT_FIELDS}


def build(force: bool = False) -> str:
    """Compile the oracle as a shared library (plain gcc, no -ffast-math)."""
    with _lock:
        if force or not os.path.exists(_LIB_PATH) or \
                os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
            tmp = _LIB_PATH + ".tmp%d" % os.getpid()
            subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp,
                                   _SRC, "-lm"])
            os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        L.orc_run.argtypes = [C.POINTER(OrcProblem), C.c_void_p, C.c_void_p,
                              C.POINTER(OrcResult), C.c_void_p, C.c_void_p]
        L.orc_run.restype = C.c_int
        L.orc_philox.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
        L.orc_child_id.argtypes = [C.c_uint64, C.c_uint32]
        L.orc_child_id.restype = C.c_uint64
        L.orc_eval.argtypes = [C.POINTER(OrcProblem), C.c_int, C.c_int, C.c_double]
        L.orc_eval.restype = C.c_double
        L.orc_tables_export.argtypes = [C.POINTER(OrcProblem)] + [C.c_void_p] * 12
        L.orc_table_lookup.argtypes = [C.POINTER(OrcProblem), C.c_int, C.c_int, C.c_void_p,
                                       C.c_void_p, C.c_int]
        L.orc_sample.argtypes = [C.c_int, C.c_double, C.c_double, C.c_longlong,
                                 C.c_ulonglong, C.c_void_p, C.c_void_p]
        L.orc_first_interaction.argtypes = [C.POINTER(OrcProblem), C.c_longlong, C.c_void_p,
                                            C.c_void_p]
        L.orc_allot.argtypes = [C.POINTER(OrcProblem), C.c_ulonglong, C.c_void_p]
        L.orc_rotate.argtypes = [C.c_void_p, C.c_double, C.c_double, C.c_void_p]
        L.orc_event.argtypes = [C.c_int, C.c_double, C.c_void_p, C.c_double, C.c_ulonglong,
                                C.c_longlong, C.c_void_p]
        L.orc_event.restype = C.c_int
        L.orc_sources.argtypes = [C.POINTER(OrcProblem), C.c_ulonglong, C.c_ulonglong, C.c_void_p]
        L.orc_beamlet_tables.argtypes = [C.POINTER(OrcProblem), C.c_void_p, C.c_void_p,
                                         C.c_void_p]
        L.orc_beamlet_tables.restype = C.c_int
        L.orc_beamlet_picks.argtypes = [C.POINTER(OrcProblem), C.c_ulonglong, C.c_ulonglong,
                                        C.c_void_p]
        L.orc_history_records.argtypes = [C.POINTER(OrcProblem), C.c_ulonglong, C.c_ulonglong,
                                          C.c_void_p, C.c_void_p]
        _lib = L
    return _lib


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


class _Prepared:
    """Holds the C struct and keeps the numpy buffers it points to alive."""

    def __init__(self, prob):
        ph, src = prob.phantom, prob.source
        self.mat = np.ascontiguousarray(ph.mat, np.uint8)
        self.rho = np.ascontiguousarray(ph.rho, np.float32)
        p = OrcProblem()
        p.nx, p.ny, p.nz = ph.shape
        p.dx, p.dy, p.dz = ph.voxel
        p.mat = self.mat.ctypes.data_as(C.POINTER(C.c_uint8))
        p.rho = self.rho.ctypes.data_as(C.POINTER(C.c_float))
        if len(ph.materials) > MAX_MAT:
            raise ValueError("too many materials")
        p.n_mat = len(ph.materials)
        for i, m in enumerate(ph.materials):
            om = p.mats[i]
            om.n_el = len(m.elements)
            for j, (z, a, w) in enumerate(m.elements):
                om.Z[j] = z; om.A[j] = a; om.w[j] = w
            om.I = m.mean_excitation_MeV
        p.e_min, p.e_max, p.n_energy = prob.e_min, prob.e_max, prob.n_energy
        p.eabs_ph, p.eabs_el, p.ms_loss = prob.eabs_photon, prob.eabs_electron, prob.ms_loss_fraction
        p.particle = src.particle
        p.geometry = {"pencil": 0, "point_field": 1, "beamlets": 2}[src.kind]
        for name in ("origin", "direction", "center", "axis_u", "axis_v"):
            getattr(p, name)[:] = list(getattr(src, name))
        p.half_u, p.half_v = src.half_u, src.half_v
        sp = src.spectrum
        p.n_bins = sp.n_bins
        for j, e in enumerate(sp.edges):
            p.edges[j] = float(e)
        for j, w in enumerate(sp.weights):
            p.weights[j] = float(w)
        self.beamlets = None
        if src.beamlets is not None:
            self.beamlets = np.ascontiguousarray(src.beamlets, np.float64)
            p.n_beamlets = self.beamlets.shape[0]
            p.beamlets = self.beamlets.ctypes.data_as(C.POINTER(C.c_double))
        p.beamlet_sampler = SAMPLERS[src.sampler]
        p.metro_chains = src.chains
        p.n_hist, p.n_batches = prob.n_histories, prob.n_batches
        p.first_hist = prob.first_history
        p.seed, p.request_id = prob.seed, prob.request_id
        flags = prob.flags
        if not src.annihilation:
            flags |= 1
        p.flags = flags
        self.c = p


def run(prob, per_history: bool = False):
    """Run the full dose calculation.  Returns (dose, sigma, ledger dict[, hrec, hrecd])
    with dose/sigma as flat float64 arrays in MeV/g per history."""
    prep = _Prepared(prob)
    V = prob.phantom.n_voxels
    dose = np.zeros(V, np.float64)
    sigma = np.zeros(V, np.float64)
    res = OrcResult()
    hrec = hrecd = None
    if per_history:
        hrec = np.zeros((prob.n_histories, HR_NI), np.int32)
        hrecd = np.zeros((prob.n_histories, HD_ND), np.float64)
    rc = lib().orc_run(C.byref(prep.c), _ptr(dose), _ptr(sigma), C.byref(res), _ptr(hrec),
                       _ptr(hrecd))
    if rc != 0:
        raise ValueError("oracle rejected the problem (rc=%d)" % rc)
    if per_history:
        return dose, sigma, res.as_dict(), hrec, hrecd
    return dose, sigma, res.as_dict()


def evaluate(prob, material: int, fn: int, x) -> np.ndarray:
    prep = _Prepared(prob)
    xs = np.atleast_1d(np.asarray(x, np.float64))
    return np.array([lib().orc_eval(C.byref(prep.c), material, fn, float(v)) for v in xs])


def tables(prob) -> dict:
    prep = _Prepared(prob)
    n, M = prob.n_energy, len(prob.phantom.materials)
    out = {k: np.zeros((M, n)) for k in ("mu_c", "mu_pe", "mu_pair", "scol", "srest",
                                          "sig_m", "sig_b", "range")}
    E = np.zeros(n); mumax = np.zeros(n); x0 = np.zeros(M); sigmax = np.zeros(M)
    lib().orc_tables_export(C.byref(prep.c), _ptr(E), _ptr(out["mu_c"]), _ptr(out["mu_pe"]),
                            _ptr(out["mu_pair"]), _ptr(out["scol"]), _ptr(out["srest"]),
                            _ptr(out["sig_m"]), _ptr(out["sig_b"]), _ptr(out["range"]),
                            _ptr(mumax), _ptr(x0), _ptr(sigmax))
    out.update(E=E, mumax=mumax, x0=x0, sigmax=sigmax)
    return out


def lookup(prob, material: int, which: int, x) -> np.ndarray:
    prep = _Prepared(prob)
    xs = np.ascontiguousarray(np.atleast_1d(x), np.float64)
    ys = np.zeros_like(xs)
    lib().orc_table_lookup(C.byref(prep.c), material, which, _ptr(xs), _ptr(ys), len(xs))
    return ys


def sample(which: int, a: float, b: float, n: int, seed: int = 1):
    o1 = np.zeros(n); o2 = np.zeros(n)
    lib().orc_sample(which, a, b, n, seed, _ptr(o1), _ptr(o2))
    return o1, o2


def philox(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, np.uint32)
    k = np.ascontiguousarray(key, np.uint32)
    o = np.zeros(4, np.uint32)
    lib().orc_philox(_ptr(c), _ptr(k), _ptr(o))
    return o


def child_id(parent: int, k: int) -> int:
    return int(lib().orc_child_id(parent, k))


def first_interaction(prob, n: int):
    prep = _Prepared(prob)
    z = np.zeros(n); t = np.zeros(n, np.int32)
    lib().orc_first_interaction(C.byref(prep.c), n, _ptr(z), _ptr(t))
    return z, t


def allot(prob, nb: int) -> np.ndarray:
    prep = _Prepared(prob)
    out = np.zeros(prob.source.spectrum.n_bins, np.uint64)
    lib().orc_allot(C.byref(prep.c), nb, _ptr(out))
    return out


def rotate(u, cost: float, phi: float) -> np.ndarray:
    a = np.ascontiguousarray(u, np.float64)
    o = np.zeros(3)
    lib().orc_rotate(_ptr(a), cost, phi, _ptr(o))
    return o


def event(kind: int, E: float, u, cut: float, n: int, seed: int = 1) -> np.ndarray:
    """n single events as the transport applies them: kind 0 Compton of a
    photon of energy E, kind 1 hard Moller of an electron of kinetic energy E
    (cut W_cc), kind 2 annihilation of a positron at rest, kind 3 pair
    production by a photon of energy E, kind 4 photoelectric absorption
    (Sauter angles when cut != 0), kind 5 hard bremsstrahlung (cut W_cb).
    Rows: particle after the event (E, u), banked secondary (E, u); for
    kind 2 the two photons, for kind 3 the electron and the positron."""
    out = np.zeros((n, 8))
    uu = np.ascontiguousarray(u, np.float64)
    if lib().orc_event(kind, E, _ptr(uu), cut, seed, n, _ptr(out)) != 0:
        raise ValueError("bad event kind")
    return out


def sources(prob, first: int, n: int) -> np.ndarray:
    """Primaries [first, first+n) of batch 0 after entry: rows x y z u v w E entered."""
    prep = _Prepared(prob)
    out = np.zeros((n, 8))
    lib().orc_sources(C.byref(prep.c), first, n, _ptr(out))
    return out


def beamlet_tables(prob):
    """(index, prob, alias): the positive-weight beamlet list (rows of the
    fluence map) and its Walker alias table, positions in that list."""
    prep = _Prepared(prob)
    nb = prep.beamlets.shape[0]
    index = np.zeros(nb, np.int32)
    cut = np.zeros(nb)
    alias = np.zeros(nb, np.int32)
    nf = lib().orc_beamlet_tables(C.byref(prep.c), _ptr(index), _ptr(cut), _ptr(alias))
    return index[:nf], cut[:nf], alias[:nf]


def beamlet_picks(prob, first: int, n: int) -> np.ndarray:
    """Beamlet rows chosen for histories [first, first+n) by the source's sampler."""
    prep = _Prepared(prob)
    out = np.zeros(n, np.int32)
    lib().orc_beamlet_picks(C.byref(prep.c), first, n, _ptr(out))
    return out


def history_records(prob, first: int, n: int):
    """Per-history records of histories [first, first+n) of the full problem."""
    prep = _Prepared(prob)
    rec = np.zeros((n, HR_NI), np.int32)
    recd = np.zeros((n, HD_ND), np.float64)
    lib().orc_history_records(C.byref(prep.c), first, n, _ptr(rec), _ptr(recd))
    return rec, recd
