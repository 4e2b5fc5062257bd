"""Seeded synthetic inputs for the gDPM dose engine.

This module builds the *inputs* of a dose calculation: voxel phantoms
(material index + mass density per voxel), material compositions, source
descriptions (particle type, energy spectrum, field geometry) and run
parameters.  It holds none of the method's arithmetic: no cross sections,
no sampling, no transport.  Both the CUDA path and the CPU oracle consume
the same :class:`Problem` objects, each converting it to its own C structs.

Stand-ins (the paper's own inputs are not available):

* The paper's slab phantoms (Sec. 3.1: 30.5x30.5x30 cm, 0.5x0.5x0.2 cm voxels,
  water/bone/lung layers) are replaced by a 128^3 slab at 0.25 cm with
  water 0-3 cm, lung (0.26 g/cm3) 3-10 cm, bone (1.85 g/cm3) 10-12 cm, water
  beyond.
* The "realistic 6 MV energy spectrum" (Sec. 3.1) is replaced by a Kramers
  thick-target shape phi(k) ~ (E0 - k)/k on [k_lo, E0] with k_lo chosen for a
  1.8 MeV mean, histogrammed into equal-width intervals (Sec. 2.3.2 divides
  the spectrum into equal intervals).
* The DICOM patient CTs and plans (Sec. 3.2) are replaced by seeded ellipsoid
  phantoms and seeded fluence maps.

Layout conventions: voxel (ix, iy, iz) has flat index ix + nx*(iy + ny*iz)
(x fastest); the phantom occupies [0, nx*dx] x [0, ny*dy] x [0, nz*dz] cm;
energies are in MeV, lengths in cm, densities in g/cm3.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence, Tuple

import numpy as np

# ---------------------------------------------------------------------------
# Materials (compositions by mass fraction; standard atomic weights).
# ---------------------------------------------------------------------------

_ATOMIC_WEIGHT = {1: 1.008, 6: 12.011, 7: 14.007, 8: 15.999, 11: 22.990,
                  12: 24.305, 15: 30.974, 16: 32.06, 17: 35.45, 18: 39.948, 19: 39.098,
                  20: 40.078}


@dataclasses.dataclass(frozen=True)
class Material:
    name: str
    density_ref: float                    # nominal density, g/cm3 (informational)
    mean_excitation_MeV: float            # I value for the Bethe formula
    elements: Tuple[Tuple[int, float, float], ...]   # (Z, A g/mol, mass fraction)


def _mat(name, rho, I_eV, zw):
    tot = sum(w for _, w in zw)
    els = tuple((z, _ATOMIC_WEIGHT[z], w / tot) for z, w in zw)
    return Material(name, rho, I_eV * 1e-6, els)


WATER = _mat("water", 1.0, 75.0, [(1, 0.111894), (8, 0.888106)])
# Lung read as low-density water (same composition, 0.26 g/cm3).
LUNG = _mat("lung", 0.26, 75.0, [(1, 0.111894), (8, 0.888106)])
# ICRU Report 44 lung tissue (composition by mass), inflated to 0.26 g/cm3
LUNG_ICRU = _mat("lung_icru", 0.26, 75.3, [(1, 0.103), (6, 0.105), (7, 0.031), (8, 0.749),
                                           (11, 0.002), (15, 0.002), (16, 0.003), (17, 0.003),
                                           (19, 0.002)])
# Cortical bone, ICRU-44-like composition.
BONE = _mat("bone", 1.85, 106.4, [(1, 0.034), (6, 0.155), (7, 0.042), (8, 0.435),
                                  (11, 0.001), (12, 0.002), (15, 0.103), (16, 0.003),
                                  (20, 0.225)])
AIR = _mat("air", 0.0012, 85.7, [(7, 0.7553), (8, 0.2318), (18, 0.0128), (6, 0.0001)])


# ---------------------------------------------------------------------------
# Phantoms
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class Phantom:
    shape: Tuple[int, int, int]           # (nx, ny, nz)
    voxel: Tuple[float, float, float]     # (dx, dy, dz) cm
    mat: np.ndarray                       # uint8, nx*ny*nz, x fastest
    rho: np.ndarray                       # float32 g/cm3, same layout
    materials: List[Material]

    @property
    def n_voxels(self) -> int:
        return int(self.shape[0] * self.shape[1] * self.shape[2])

    @property
    def extent(self) -> Tuple[float, float, float]:
        return tuple(n * d for n, d in zip(self.shape, self.voxel))

    def grid3(self, a: np.ndarray) -> np.ndarray:
        """View a flat voxel array as [iz, iy, ix]."""
        nx, ny, nz = self.shape
        return np.asarray(a).reshape(nz, ny, nx)


def homogeneous_phantom(shape=(32, 32, 32), voxel=(0.5, 0.5, 0.5), material=WATER,
                        density: Optional[float] = None) -> Phantom:
    n = shape[0] * shape[1] * shape[2]
    rho = material.density_ref if density is None else density
    return Phantom(tuple(shape), tuple(float(v) for v in voxel),
                   np.zeros(n, np.uint8), np.full(n, rho, np.float32), [material])


def slab_phantom(shape=(128, 128, 128), voxel=(0.25, 0.25, 0.25),
                 layers=((3.0, WATER, 1.0), (10.0, LUNG, 0.26), (12.0, BONE, 1.85),
                         (1e30, WATER, 1.0))) -> Phantom:
    """Layered phantom along z.  ``layers`` = (z_upper_cm, material, density);
    a voxel takes the layer that contains its centre."""
    nx, ny, nz = shape
    mats: List[Material] = []
    for _, m, _ in layers:
        if m not in mats:
            mats.append(m)
    zc = (np.arange(nz) + 0.5) * voxel[2]
    mat_z = np.zeros(nz, np.uint8)
    rho_z = np.zeros(nz, np.float32)
    lo = -1e30
    for up, m, d in layers:
        sel = (zc >= lo) & (zc < up)
        mat_z[sel] = mats.index(m)
        rho_z[sel] = d
        lo = up
    mat = np.broadcast_to(mat_z[:, None, None], (nz, ny, nx)).reshape(-1).copy()
    rho = np.broadcast_to(rho_z[:, None, None], (nz, ny, nx)).reshape(-1).copy()
    return Phantom(tuple(shape), tuple(float(v) for v in voxel), mat, rho, mats)


def ct_phantom(shape=(256, 256, 128), voxel=(0.25, 0.25, 0.25), seed=11) -> Phantom:
    """Patient-like phantom from seeded ellipsoids: a water-density body
    (0.95-1.05), two lungs (0.20-0.30), a spine and ribs of bone (1.4-1.85) and
    one air cavity (0.001).  Air outside the body."""
    rng = np.random.default_rng(seed)
    nx, ny, nz = shape
    dx, dy, dz = voxel
    X, Y, Z = np.meshgrid((np.arange(nx) + 0.5) * dx, (np.arange(ny) + 0.5) * dy,
                          (np.arange(nz) + 0.5) * dz, indexing="xy")
    # meshgrid 'xy' gives [iy, ix, iz]; move to [iz, iy, ix]
    X, Y, Z = (np.transpose(a, (2, 0, 1)) for a in (X, Y, Z))
    cx, cy, cz = nx * dx / 2, ny * dy / 2, nz * dz / 2
    mats = [AIR, WATER, LUNG, BONE]
    mat = np.zeros((nz, ny, nx), np.uint8)
    rho = np.full((nz, ny, nx), AIR.density_ref, np.float32)

    def ell(c, r):
        return ((X - c[0]) / r[0]) ** 2 + ((Y - c[1]) / r[1]) ** 2 + ((Z - c[2]) / r[2]) ** 2 <= 1.0

    body = ell((cx, cy, cz), (0.45 * nx * dx, 0.32 * ny * dy, 0.6 * nz * dz))
    mat[body] = 1
    rho[body] = rng.uniform(0.95, 1.05)
    for k in range(3):                      # a few soft-tissue density variations
        c = (cx + rng.uniform(-8, 8), cy + rng.uniform(-5, 5), cz + rng.uniform(-6, 6))
        s = ell(c, (rng.uniform(2, 5), rng.uniform(2, 4), rng.uniform(2, 5))) & body
        rho[s] = rng.uniform(0.95, 1.05)
    for side in (-1, 1):                    # lungs
        s = ell((cx + side * 0.22 * nx * dx, cy - 0.02 * ny * dy, cz),
                (0.15 * nx * dx, 0.2 * ny * dy, 0.45 * nz * dz)) & body
        mat[s] = 2
        rho[s] = rng.uniform(0.20, 0.30)
    spine = ell((cx, cy + 0.2 * ny * dy, cz), (1.5, 1.5, 0.55 * nz * dz)) & body
    mat[spine] = 3
    rho[spine] = rng.uniform(1.4, 1.85)
    for k in range(10):                     # ribs: thin elongated ellipsoids
        z0 = cz + (k - 4.5) * 0.09 * nz * dz
        for side in (-1, 1):
            s = ell((cx + side * 0.33 * nx * dx, cy, z0), (1.0, 0.25 * ny * dy, 0.5)) & body
            mat[s] = 3
            rho[s] = rng.uniform(1.4, 1.85)
    cav = ell((cx + rng.uniform(-3, 3), cy - 0.15 * ny * dy, cz + rng.uniform(-3, 3)),
              (2.0, 1.5, 2.5)) & body
    mat[cav] = 0
    rho[cav] = 0.001
    return Phantom(tuple(shape), tuple(float(v) for v in voxel),
                   mat.reshape(-1).copy(), rho.reshape(-1).copy(), mats)


# ---------------------------------------------------------------------------
# Energy spectra
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class Spectrum:
    edges: np.ndarray      # n_bins + 1, MeV, increasing
    weights: np.ndarray    # n_bins, relative (need not be normalised)

    @property
    def n_bins(self) -> int:
        return len(self.weights)


def kramers_spectrum(e_max=6.0, mean=1.8, n_bins=24) -> Spectrum:
    """Thick-target (Kramers) bremsstrahlung shape phi(k) ~ (E0-k)/k on
    [k_lo, E0], k_lo solved for the requested mean, integrated over
    ``n_bins`` equal-width intervals of (0, E0]."""
    E0 = e_max

    def mean_of(klo):
        num = E0 * (E0 - klo) - 0.5 * (E0 ** 2 - klo ** 2)
        den = E0 * math.log(E0 / klo) - (E0 - klo)
        return num / den

    lo, hi = 1e-4, E0 * (1 - 1e-9)
    for _ in range(200):                   # bisection: mean_of is increasing in k_lo
        mid = 0.5 * (lo + hi)
        if mean_of(mid) < mean:
            lo = mid
        else:
            hi = mid
    klo = 0.5 * (lo + hi)
    edges = np.linspace(0.0, E0, n_bins + 1)
    w = np.zeros(n_bins)
    for j in range(n_bins):
        a, b = max(edges[j], klo), edges[j + 1]
        if b > a:
            w[j] = E0 * math.log(b / a) - (b - a)
    return Spectrum(edges, w / w.sum())


def mono_spectrum(energy: float) -> Spectrum:
    return Spectrum(np.array([energy, energy]), np.array([1.0]))


# ---------------------------------------------------------------------------
# Sources
# ---------------------------------------------------------------------------

PHOTON, ELECTRON = 0, 1


@dataclasses.dataclass
class Source:
    """Primary particle source.

    kind 'pencil': every primary starts at ``origin`` moving along ``direction``.
    kind 'point_field': a point source at ``origin``; each primary aims at a
    point uniform in the rectangle centre ``center`` spanned by unit axes
    ``axis_u``/``axis_v`` with half widths ``half_u``/``half_v``.
    kind 'beamlets': a fluence map; beamlet rows in ``beamlets`` are
    [src(3), centre(3), axis_u(3), axis_v(3), u0, u1, v0, v1, weight].
    """
    particle: int
    spectrum: Spectrum
    kind: str = "pencil"
    origin: Tuple[float, float, float] = (0.0, 0.0, 0.0)
    direction: Tuple[float, float, float] = (0.0, 0.0, 1.0)
    center: Tuple[float, float, float] = (0.0, 0.0, 0.0)
    axis_u: Tuple[float, float, float] = (1.0, 0.0, 0.0)
    axis_v: Tuple[float, float, float] = (0.0, 1.0, 0.0)
    half_u: float = 0.0
    half_v: float = 0.0
    beamlets: Optional[np.ndarray] = None
    annihilation: bool = True
    sampler: str = "cdf"           # beamlet sampler: "cdf", "alias" or "metropolis"
    chains: int = 4096             # Metropolis chains (Algorithm A1)


def pencil_source(phantom: Phantom, energy: float, particle=PHOTON) -> Source:
    """Pencil beam along +z entering at the centre of the z=0 face."""
    X, Y, _ = phantom.extent
    return Source(particle, mono_spectrum(energy), "pencil", (X / 2, Y / 2, 0.0), (0.0, 0.0, 1.0))


def field_source(phantom: Phantom, spectrum: Spectrum, particle=PHOTON, ssd=100.0,
                 field=(10.0, 10.0)) -> Source:
    """Point source on the central axis at distance ``ssd`` above the z=0
    face; field ``field`` (cm) defined on the z=0 plane."""
    X, Y, _ = phantom.extent
    return Source(particle, spectrum, "point_field", (X / 2, Y / 2, -ssd), (0.0, 0.0, 1.0),
                  (X / 2, Y / 2, 0.0), (1.0, 0.0, 0.0), (0.0, 1.0, 0.0),
                  field[0] / 2, field[1] / 2)


# ---------------------------------------------------------------------------
# Beam geometry: gantry frames, fluence-map beamlets, MLC apertures
# ---------------------------------------------------------------------------

@dataclasses.dataclass(frozen=True)
class BeamFrame:
    """A beam at gantry angle ``gantry_deg`` rotating about the z axis through
    the isocentre: point source at distance ``sad`` from the isocentre, beam
    axis through the isocentre, iso-plane axes ``axis_u`` (in the rotation
    plane) and ``axis_v`` (= z).  At 0 degrees the source sits on the -y side."""
    source: Tuple[float, float, float]
    iso: Tuple[float, float, float]
    axis_u: Tuple[float, float, float]
    axis_v: Tuple[float, float, float]


def beam_frame(gantry_deg: float, iso, sad: float = 100.0) -> BeamFrame:
    t = math.radians(gantry_deg)
    src = (iso[0] + sad * math.sin(t), iso[1] - sad * math.cos(t), iso[2])
    return BeamFrame(src, tuple(iso), (math.cos(t), math.sin(t), 0.0), (0.0, 0.0, 1.0))


def beamlet_row(fr: BeamFrame, u0, u1, v0, v1, weight) -> List[float]:
    """One beamlet: rectangle [u0,u1] x [v0,v1] (cm) on the iso plane."""
    return [*fr.source, *fr.iso, *fr.axis_u, *fr.axis_v, u0, u1, v0, v1, weight]


def fluence_map_rows(fr: BeamFrame, intensity: np.ndarray, size: float = 1.0) -> List[List[float]]:
    """Beamlets of a fluence map (rows = v, cols = u) centred on the isocentre;
    the weight f_I of a beamlet is its intensity times its area (Sec. 2.3.1);
    beamlets with zero intensity are left out."""
    nv, nu = intensity.shape
    rows = []
    for j in range(nv):
        for i in range(nu):
            f = float(intensity[j, i])
            if f > 0:
                u0 = (i - nu / 2) * size
                v0 = (j - nv / 2) * size
                rows.append(beamlet_row(fr, u0, u0 + size, v0, v0 + size, f * size * size))
    return rows


def aperture_rows(fr: BeamFrame, leaves: np.ndarray, leaf_width: float, v_start: float,
                  weight: float = 1.0) -> List[List[float]]:
    """An MLC aperture: leaf pair k spans v in [v_start + k w, v_start + (k+1) w]
    and is open between leaves[k] = (u_left, u_right); uniform fluence."""
    rows = []
    for k, (a, b) in enumerate(leaves):
        if b > a:
            v0 = v_start + k * leaf_width
            rows.append(beamlet_row(fr, float(a), float(b), v0, v0 + leaf_width,
                                    weight * (b - a) * leaf_width))
    return rows


def beamlet_source(rows, spectrum: "Spectrum", particle=PHOTON) -> "Source":
    return Source(particle, spectrum, "beamlets", beamlets=np.asarray(rows, np.float64))


def imrt_plan(phantom: "Phantom", n_beams: int = 7, map_size: int = 20, beamlet: float = 1.0,
              seed: int = 11, sad: float = 100.0) -> "Source":
    """Coplanar IMRT plan: n_beams equally spaced gantry angles, each a
    map_size^2 fluence map of beamlet-cm beamlets with intensities U[0,1]."""
    rng = np.random.default_rng(seed)
    iso = tuple(e / 2 for e in phantom.extent)
    rows = []
    for b in range(n_beams):
        fr = beam_frame(360.0 * b / n_beams, iso, sad)
        rows += fluence_map_rows(fr, rng.uniform(0, 1, (map_size, map_size)), beamlet)
    return beamlet_source(rows, kramers_spectrum())


def vmat_arc(phantom: "Phantom", n_points: int = 180, step_deg: float = 2.0, field: float = 10.0,
             leaf_width: float = 0.5, seed: int = 3, sad: float = 100.0) -> "Source":
    """VMAT arc: n_points control points step_deg apart; at each, the MLC
    leaf pairs that cover the field are open between seeded leaf positions
    inside the field."""
    rng = np.random.default_rng(seed)
    iso = tuple(e / 2 for e in phantom.extent)
    n_pairs = int(round(field / leaf_width))
    rows = []
    for c in range(n_points):
        fr = beam_frame(c * step_deg, iso, sad)
        left = rng.uniform(-field / 2, 0.0, n_pairs)
        right = rng.uniform(0.0, field / 2, n_pairs)
        rows += aperture_rows(fr, np.stack([left, right], 1), leaf_width, -field / 2)
    return beamlet_source(rows, kramers_spectrum())


def single_beamlet(phantom: "Phantom", gantry_deg: float, u: float, v: float, size: float,
                   sad: float = 100.0) -> "Source":
    iso = tuple(e / 2 for e in phantom.extent)
    fr = beam_frame(gantry_deg, iso, sad)
    return beamlet_source([beamlet_row(fr, u, u + size, v, v + size, 1.0)], kramers_spectrum())


def ct_imrt_problem(n_histories=250_000_000, n_batches=100, shape=(256, 256, 128),
                    voxel=(0.25, 0.25, 0.25), seed=12345) -> "Problem":
    """Patient-like ellipsoid phantom with a 7-beam 20x20 fluence-map IMRT
    plan, 6 MV-like spectrum (stands in for the paper's DICOM IMRT/VMAT plans)."""
    ph = ct_phantom(shape, voxel)
    return Problem(ph, imrt_plan(ph), n_histories, n_batches, eabs_photon=0.05,
                   eabs_electron=0.2, e_min=0.005, e_max=6.5, seed=seed)


# ---------------------------------------------------------------------------
# Problem = everything one dose calculation needs
# ---------------------------------------------------------------------------

FLAG_NO_ANNIHILATION = 1     # positrons end without annihilation photons (paper Sec. 4)
FLAG_COMPTON_ONLY = 2        # photoelectric and pair cross sections set to zero
FLAG_NO_HARD = 4             # no hard Moller / bremsstrahlung events for electrons
FLAG_SAUTER = 8              # photoelectrons leave at Sauter's K-shell angle (physics variant)


@dataclasses.dataclass
class Problem:
    phantom: Phantom
    source: Source
    n_histories: int
    n_batches: int = 100
    eabs_photon: float = 0.05      # MeV; also the hard-bremsstrahlung threshold W_cb
    eabs_electron: float = 0.2     # MeV; also the hard-Moller threshold W_cc
    e_min: float = 0.005           # table grid, MeV
    e_max: float = 21.0
    n_energy: int = 512
    ms_loss_fraction: float = 0.2  # CSDA energy-loss fraction that limits an electron step
    seed: int = 12345
    request_id: int = 0
    flags: int = 0
    first_history: int = 0         # id of the first history (Philox counter word 0)
    # beamlet dose matrix: one sub-problem per fluence-map row, with these
    # histories each (n_histories is then their sum)
    sub_histories: Optional[Tuple[int, ...]] = None

    def with_(self, **kw) -> "Problem":
        return dataclasses.replace(self, **kw)

    def sub_problem(self, k: int) -> "Problem":
        """Beamlet k of a dose-matrix problem as a problem of its own: that
        row alone as the source, its histories, and its range of history ids."""
        n = [int(v) for v in self.sub_histories]
        rows = np.asarray(self.source.beamlets[k:k + 1], np.float64).copy()
        rows[0, 16] = 1.0
        src = dataclasses.replace(self.source, beamlets=rows, sampler="cdf")
        return dataclasses.replace(self, source=src, n_histories=n[k],
                                   first_history=self.first_history + sum(n[:k]),
                                   sub_histories=None)


def tiny_problem(n_histories=100_000, seed=12345, n_batches=100) -> Problem:
    """1.0 MeV photon pencil beam on a 32^3 water cube of 0.5 cm voxels;
    photon cutoff 10 keV, electron cutoff 200 keV."""
    ph = homogeneous_phantom((32, 32, 32), (0.5, 0.5, 0.5), WATER, 1.0)
    return Problem(ph, pencil_source(ph, 1.0), n_histories, n_batches,
                   eabs_photon=0.01, eabs_electron=0.2, e_min=0.005, e_max=1.5, seed=seed)


def slab_photon_problem(n_histories=100_000_000, seed=12345, n_batches=100,
                        shape=(128, 128, 128), voxel=(0.25, 0.25, 0.25)) -> Problem:
    """128^3 water/lung/bone/water slab, 6 MV-like spectrum, 10x10 cm field
    at SSD 100 cm; cutoffs 50 keV (photons) / 200 keV (electrons)."""
    ph = slab_phantom(shape, voxel)
    return Problem(ph, field_source(ph, kramers_spectrum()), n_histories, n_batches,
                   eabs_photon=0.05, eabs_electron=0.2, e_min=0.005, e_max=6.5, seed=seed)


def paper_slab_problem(middle="lung", particle=PHOTON, n_histories=None, n_batches=10,
                       seed=12345) -> Problem:
    """The phantom cases of Sec. 3.1 (Table 1): a 30.5 x 30.5 x 30.0 cm slab of
    0.5 x 0.5 x 0.2 cm voxels (61 x 61 x 150), 5 cm water, 5 cm lung or bone,
    20 cm water along z; a point source at SSD 90 cm whose 10 x 10 cm field at
    SAD 100 cm is 9 x 9 cm on the surface; 20 MeV electrons or the 6 MV-like
    spectrum; absorption energies 200 keV (electrons) and 50 keV (photons);
    10 batches.  Histories default to the paper's: 2.5e6 electrons, 2.5e8
    photons.  Lung and bone take this module's densities (0.26, 1.85 g/cm3);
    the paper does not state them."""
    mid = {"lung": (LUNG, 0.26), "bone": (BONE, 1.85)}[middle]
    ph = slab_phantom((61, 61, 150), (0.5, 0.5, 0.2),
                      layers=((5.0, WATER, 1.0), (10.0, mid[0], mid[1]), (1e30, WATER, 1.0)))
    if n_histories is None:
        n_histories = 2_500_000 if particle == ELECTRON else 250_000_000
    if particle == ELECTRON:
        src, e_max = field_source(ph, mono_spectrum(20.0), ELECTRON, ssd=90.0, field=(9.0, 9.0)), 21.0
    else:
        src, e_max = field_source(ph, kramers_spectrum(), PHOTON, ssd=90.0, field=(9.0, 9.0)), 6.5
    return Problem(ph, src, n_histories, n_batches, eabs_photon=0.05, eabs_electron=0.2,
                   e_min=0.005, e_max=e_max, seed=seed)


def water64_problem(particle=PHOTON, n_histories=None, n_batches=10, seed=12345) -> Problem:
    """The comparison case of Sec. 4: a homogeneous water phantom of 64^3
    voxels of 0.5 cm, a 15 MeV monoenergetic, mono-directional beam entering
    normally, annihilation photons switched off; 1e6 electrons or 4e6
    photons by default.  The paper states neither the beam's width nor the
    cutoffs: the beam is read as a pencil at the centre of the entry face and
    the absorption energies as those of Sec. 3.1 (200 keV electrons, 50 keV
    photons)."""
    ph = homogeneous_phantom((64, 64, 64), (0.5, 0.5, 0.5), WATER, 1.0)
    if n_histories is None:
        n_histories = 1_000_000 if particle == ELECTRON else 4_000_000
    return Problem(ph, pencil_source(ph, 15.0, particle), n_histories, n_batches, eabs_photon=0.05,
                   eabs_electron=0.2, e_min=0.005, e_max=16.0, seed=seed,
                   flags=FLAG_NO_ANNIHILATION)


def beamlet_matrix_problem(n_beamlets=400, seed=7, n_batches=1, hist_range=(1e5, 5e6),
                           shape=(128, 128, 128), voxel=(0.25, 0.25, 0.25)) -> Problem:
    """Beamlet dose matrix on the 128^3 slab: n_beamlets square beamlets of
    side U{0.5, 1, 1.5, 2} cm centred U within +-8 cm of the axis on the z = 0
    face, point source at SSD 100 cm on the axis, 6 MV-like spectrum; each
    beamlet gets log-uniform(hist_range) histories and its own tally."""
    ph = slab_phantom(shape, voxel)
    X, Y, _ = ph.extent
    fr = BeamFrame((X / 2, Y / 2, -100.0), (X / 2, Y / 2, 0.0), (1.0, 0.0, 0.0), (0.0, 1.0, 0.0))
    rng = np.random.default_rng(seed)
    rows, hist = [], []
    for _ in range(n_beamlets):
        a = float(rng.choice([0.5, 1.0, 1.5, 2.0]))
        cu, cv = rng.uniform(-8.0, 8.0, 2)
        rows.append(beamlet_row(fr, cu - a / 2, cu + a / 2, cv - a / 2, cv + a / 2, 1.0))
        hist.append(int(round(math.exp(rng.uniform(math.log(hist_range[0]), math.log(hist_range[1]))))))
    return Problem(ph, beamlet_source(rows, kramers_spectrum()), sum(hist), n_batches,
                   eabs_photon=0.05, eabs_electron=0.2, e_min=0.005, e_max=6.5,
                   sub_histories=tuple(hist))


def slab_electron_problem(n_histories=10_000_000, seed=12345, n_batches=100,
                          shape=(128, 128, 128), voxel=(0.25, 0.25, 0.25)) -> Problem:
    """Same slab, 20 MeV monoenergetic electrons, 10x10 cm field at SSD 100."""
    ph = slab_phantom(shape, voxel)
    return Problem(ph, field_source(ph, mono_spectrum(20.0), ELECTRON), n_histories,
                   n_batches, eabs_photon=0.05, eabs_electron=0.2, e_min=0.005,
                   e_max=21.0, seed=seed)
