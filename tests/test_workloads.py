"""The seeded input generators (no method arithmetic): shapes, layouts and
the geometry each one promises, so that every test and benchmark runs on
the inputs it names."""
import math

import numpy as np
import pytest

from paper_1107_3355_gb300 import workloads as W


def test_paper_slab_geometry_matches_sec_3_1():
    """61 x 61 x 150 voxels of 0.5 x 0.5 x 0.2 cm; 5 cm water, 5 cm lung or
    bone, 20 cm water; point source at SSD 90 cm whose field is 10 x 10 cm
    at SAD 100 cm (the isocentre plane, 10 cm deep)."""
    for middle, mat, rho in (("lung", W.LUNG, 0.26), ("bone", W.BONE, 1.85)):
        p = W.paper_slab_problem(middle, W.PHOTON)
        ph = p.phantom
        assert ph.shape == (61, 61, 150) and ph.voxel == (0.5, 0.5, 0.2)
        assert ph.extent == pytest.approx((30.5, 30.5, 30.0))
        m = ph.mat.reshape(150, 61, 61)
        r = ph.rho.reshape(150, 61, 61)
        for z, want, dens in ((2.5, W.WATER, 1.0), (7.5, mat, rho), (20.0, W.WATER, 1.0)):
            iz = int(z / 0.2)
            assert ph.materials[m[iz, 30, 30]] == want and r[iz, 30, 30] == pytest.approx(dens)
            assert np.all(m[iz] == m[iz, 0, 0])                      # layers are uniform in x, y
        s = p.source
        assert s.kind == "point_field" and s.origin[2] == pytest.approx(-90.0)
        assert 2 * s.half_u * 100.0 / 90.0 == pytest.approx(10.0)   # 10 cm at SAD 100
        assert (p.n_histories, p.n_batches) == (250_000_000, 10)
        assert (p.eabs_electron, p.eabs_photon) == (0.2, 0.05)
    assert W.paper_slab_problem("bone", W.ELECTRON).n_histories == 2_500_000


def test_flat_index_layout_is_x_fastest():
    ph = W.slab_phantom((4, 3, 60), (0.25, 0.25, 0.25))   # 15 cm deep
    m = ph.mat.reshape(60, 3, 4)                      # [iz][iy][ix]
    assert np.all(m == m[:, :1, :1])                  # layers vary with z only
    for z, want in ((1.0, W.WATER), (5.0, W.LUNG), (11.0, W.BONE), (14.0, W.WATER)):
        assert ph.materials[m[int(z / 0.25), 0, 0]] == want, z


def test_kramers_spectrum_has_its_mean():
    sp = W.kramers_spectrum()
    assert sp.n_bins == 24 and sp.edges[0] == 0.0 and sp.edges[-1] == pytest.approx(6.0)
    w = sp.weights / sp.weights.sum()
    mid = 0.5 * (sp.edges[1:] + sp.edges[:-1])
    assert float((w * mid).sum()) == pytest.approx(1.8, abs=0.1)     # binned mean of a 1.8 MeV shape
    assert np.all(sp.weights >= 0)


def test_ct_phantom_is_seeded_and_patient_like():
    a = W.ct_phantom((64, 64, 32), (1.0, 1.0, 1.0))
    b = W.ct_phantom((64, 64, 32), (1.0, 1.0, 1.0))
    assert np.array_equal(a.mat, b.mat) and np.array_equal(a.rho, b.rho)
    names = [m.name for m in a.materials]
    present = {names[k] for k in np.unique(a.mat)}
    assert present == {"air", "water", "lung", "bone"}
    m = a.mat.reshape(32, 64, 64)
    assert a.materials[m[0, 0, 0]].name == "air"                      # outside the body
    assert a.materials[m[16, 32, 32]].name in ("water", "lung")       # inside
    assert a.rho.min() > 0 and a.rho.max() <= 1.85


def test_plans_have_their_beams_and_control_points():
    ph = W.ct_phantom((64, 64, 32), (1.0, 1.0, 1.0))
    imrt = W.imrt_plan(ph)
    rows = np.asarray(imrt.beamlets)
    assert rows.shape == (7 * 400, 17)
    assert np.all((rows[:, 16] >= 0) & (rows[:, 16] <= 1))
    iso = np.array(ph.extent) / 2
    src = rows[::400, :3]                                               # one per beam
    ang = np.degrees(np.arctan2(src[:, 0] - iso[0], -(src[:, 1] - iso[1]))) % 360
    np.testing.assert_allclose(np.sort(ang), 360.0 * np.arange(7) / 7, atol=1e-6)
    np.testing.assert_allclose(np.linalg.norm(src - iso, axis=1), 100.0)
    arc = np.asarray(W.vmat_arc(ph).beamlets)
    srcs = {tuple(np.round(r[:3], 6)) for r in arc}
    assert len(srcs) == 180


def test_sec_4_water_case():
    for particle, n in ((W.ELECTRON, 1_000_000), (W.PHOTON, 4_000_000)):
        p = W.water64_problem(particle)
        assert p.phantom.shape == (64, 64, 64) and p.phantom.voxel == (0.5, 0.5, 0.5)
        assert p.n_histories == n and p.flags & W.FLAG_NO_ANNIHILATION
        assert p.source.kind == "pencil" and p.source.origin[:2] == (16.0, 16.0)
        assert p.source.spectrum.edges[0] == p.source.spectrum.edges[-1] == 15.0


def test_vmat_apertures_have_uniform_fluence():
    """Each control point's MLC aperture is a set of leaf-pair openings whose
    weights equal their open areas, so the fluence is uniform over the
    aperture (Sec. 2.3 aperture sources); the pairs tile the field along v
    without overlap and open inside it along u."""
    ph = W.ct_phantom((64, 64, 32), (1.0, 1.0, 1.0))
    rows = np.asarray(W.vmat_arc(ph, n_points=12).beamlets)
    u0, u1, v0, v1, wgt = rows[:, 12], rows[:, 13], rows[:, 14], rows[:, 15], rows[:, 16]
    np.testing.assert_allclose(wgt, (u1 - u0) * (v1 - v0), rtol=1e-12)
    assert np.all(u1 > u0) and np.all(u0 >= -5.0) and np.all(u1 <= 5.0)
    np.testing.assert_allclose(v1 - v0, 0.5)
    for src in np.unique(np.round(rows[:, :3], 9), axis=0):
        cp = rows[np.all(np.abs(rows[:, :3] - src) < 1e-6, axis=1)]
        vs = np.sort(cp[:, 14])
        assert np.all(np.diff(vs) >= 0.5 - 1e-12)
        assert vs[0] >= -5.0 - 1e-12 and vs[-1] + 0.5 <= 5.0 + 1e-12
