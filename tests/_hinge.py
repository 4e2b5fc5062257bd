"""The random-hinge depth moment: a 2 MeV electron pencil deep in water with
hard events off, and the closed form of the energy-weighted depth of its dose
(Sec. 2.1 condensed history: CSDA steps, random hinge, screened-Rutherford
deflection matched to the step's first transport moment G1).

With no hard events every step is fixed by its start energy: mass length
x_j, energy loss dT_j, and a deflection whose mean cosine is m_j = 1 - G1_j,
G1_j = x_j (E_s / p beta c)^2 / (2 X0) at the mid-step energy.  Deflections
with a uniform azimuth scale the expected direction by m_j (Lewis' moment
argument), so before step j the expected direction along the beam is
c_j = prod_{i<j} m_i.  For a hinge at zeta ~ U(0,1) and the loss spread
evenly along the step, the expected depth averaged over the step is
Z_j + x_j c_j (1/3 + m_j/6), and the step moves the expected depth by
x_j c_j (1 + m_j)/2.  The energy-weighted depth of the dose is then
sum_j dT_j (...) plus E_abs at the track end, over T0.  A hinge at either end
of the step, or G1 off by a factor of two, moves it by about 0.06-0.1 cm; a
per-step mean cosine 2 % low, by 0.0064 cm.
"""
import numpy as np
from scipy import optimize

from oracle import oracle as O
from paper_1107_3355_gb300 import workloads as W

MC2 = 0.51099895
E_S = 21.2                       # Rossi-Greisen scattering energy, MeV
T0, NZ, DZ, Z0 = 2.0, 200, 0.02, 1.5
AREA = 100.0 * 100.0             # one voxel across: no lateral boundary within reach


def problem(n_histories, request_id=0):
    ph = W.homogeneous_phantom((1, 1, NZ), (100.0, 100.0, DZ), W.WATER, 1.0)
    src = W.Source(W.ELECTRON, W.mono_spectrum(T0), "pencil", (50.0, 50.0, Z0), (0.0, 0.0, 1.0))
    return W.Problem(ph, src, n_histories, 2, eabs_photon=0.05, eabs_electron=0.2, e_min=0.005,
                     e_max=T0 * 1.05, flags=W.FLAG_NO_HARD, request_id=request_id)


def step_sequence(p):
    """The deterministic CSDA steps from T0 to E_abs: (mass length, energy
    loss, mean deflection cosine m) per step."""
    k, eabs = p.ms_loss_fraction, p.eabs_electron
    rng_of = lambda t: float(O.evaluate(p, 0, O.OF_RANGE, t)[0])      # CSDA range, g/cm^2
    x0 = 1.0 / float(O.evaluate(p, 0, O.OF_BCONST, 1.0)[0])           # radiation length
    steps, E = [], T0
    while True:
        r0 = rng_of(E)
        x_cut, x_ms = r0 - rng_of(eabs), r0 - rng_of((1.0 - k) * E)
        if x_cut <= x_ms:
            x, te = x_cut, eabs
        else:
            x = x_ms
            te = optimize.brentq(lambda t: rng_of(t) - (r0 - x), eabs, E, xtol=1e-13)
        tm = 0.5 * (E + te)
        pbc = tm * (tm + 2 * MC2) / (tm + MC2)
        g1 = x * (E_S / pbc) ** 2 / (2.0 * x0)
        steps.append((x, E - te, 0.0 if g1 >= 1.0 else 1.0 - g1))
        if te <= eabs:
            break
        E = te
    return steps


def closed_form(p):
    """Expected energy-weighted depth (cm) from the deterministic step sequence."""
    eabs = p.eabs_electron
    steps = step_sequence(p)
    Z, c, num = Z0, 1.0, 0.0
    for x, dT, m in steps:                      # density 1: mass length = cm
        num += dT * (Z + x * c * (1.0 / 3.0 + m / 6.0))
        Z += x * c * (1.0 + m) / 2.0
        c *= m
    return (num + eabs * Z) / T0


def _g1_of_a(a):
    return 2.0 * a * ((1.0 + a) * np.log1p(1.0 / a) - 1.0)


def _mu2_mean(g1):
    """E[mu^2] of the screened-Rutherford law p(mu) ~ (1 - mu + 2A)^-2 whose
    E[1 - mu] is g1 (quadrature of the density; isotropic for g1 >= 1)."""
    from scipy import integrate
    if g1 >= 1.0:
        return 1.0 / 3.0
    a = optimize.brentq(lambda x: _g1_of_a(x) - g1, 1e-30, 1e12, xtol=1e-300, rtol=1e-15)
    f = lambda mu: (1.0 - mu + 2.0 * a) ** -2
    pts = [1.0 - 1e-3, 1.0 - 1e-6]
    nrm = integrate.quad(f, -1.0, 1.0, epsabs=0, epsrel=1e-12, points=pts)[0]
    return integrate.quad(lambda mu: mu * mu * f(mu), -1.0, 1.0, epsabs=0, epsrel=1e-12,
                          points=pts)[0] / nrm


def second_moment(p):
    """Expected energy-weighted (z - Z0)^2 (cm^2).  Along z only: a straight
    piece of length s moves z by s w, a deflection scales E[w] and E[z w] by
    m_j and maps E[w^2] to q E[w^2] + (1 - q)(1 - E[w^2])/2 with q = E[mu^2]
    (uniform azimuth).  The hinge position zeta ~ U(0,1) enters as a
    polynomial of degree 3, averaged exactly by 8-point Gauss-Legendre."""
    zeta, wq = np.polynomial.legendre.leggauss(8)
    zeta, wq = 0.5 * (zeta + 1.0), 0.5 * wq
    z, w, z2, zw, w2 = 0.0, 1.0, 0.0, 0.0, 1.0
    num = 0.0
    for x, dT, m in step_sequence(p):
        q = _mu2_mean(1.0 - m)
        acc = np.zeros(6)
        for zt, wt in zip(zeta, wq):
            a, b = zt * x, (1.0 - zt) * x
            avg1 = z2 + a * zw + a * a * w2 / 3.0
            z_1, z2_1, zw_1 = z + a * w, z2 + 2 * a * zw + a * a * w2, zw + a * w2
            w_d, zw_d, w2_d = m * w, m * zw_1, q * w2 + (1.0 - q) * (1.0 - w2) / 2.0
            avg2 = z2_1 + b * zw_d + b * b * w2_d / 3.0
            acc += wt * np.array([(a * avg1 + b * avg2) / x, z_1 + b * w_d,
                                  z2_1 + 2 * b * zw_d + b * b * w2_d, zw_d + b * w2_d, w2_d, w_d])
        num += dT * acc[0]
        z, z2, zw, w2, w = acc[1], acc[2], acc[3], acc[4], acc[5]
    return (num + p.eabs_electron * z2) / T0


def depth_moment(dose):
    """(energy-weighted depth in cm, energy per history in MeV) of a dose grid
    in MeV/g per history; voxel centres stand in for positions inside a voxel."""
    e = np.asarray(dose, np.float64) * (AREA * DZ)
    zc = (np.arange(NZ) + 0.5) * DZ
    return float((e * zc).sum() / e.sum()), float(e.sum())


def depth_second_moment(dose):
    """Energy-weighted (z - Z0)^2 of a dose grid (cm^2), with the DZ^2/12 of
    positions spread over a voxel added to the voxel-centre sum."""
    e = np.asarray(dose, np.float64) * (AREA * DZ)
    zc = (np.arange(NZ) + 0.5) * DZ - Z0
    return float((e * zc * zc).sum() / e.sum()) + DZ * DZ / 12.0


# The same electron in z-layers of water at different densities.  Every step
# quantity is per unit mass (mass length, G1 with X0 in g/cm^2) and the voxel
# walk spends the step's mass length voxel by voxel, so along z the mass depth
# moves by w dm whatever the densities: with the same random draws the
# mass-depth history equals the homogeneous one, up to the rounding of
# positions and the binning of the grid.
LAYER_RHO = (1.0, 0.5, 1.5, 0.3)
LAYER_NZ, LAYER_M0 = 300, 2.0         # start at mass depth 2 g/cm^2


def layered_problem(n_histories, request_id=0):
    rho = np.resize(np.array(LAYER_RHO), LAYER_NZ).astype(np.float32)
    faces = np.concatenate([[0.0], np.cumsum(rho.astype(np.float64) * DZ)])
    iz = int(np.searchsorted(faces, LAYER_M0) - 1)
    z0 = iz * DZ + (LAYER_M0 - faces[iz]) / float(rho[iz])
    ph = W.Phantom((1, 1, LAYER_NZ), (100.0, 100.0, DZ), np.zeros(LAYER_NZ, np.uint8), rho,
                   [W.WATER])
    src = W.Source(W.ELECTRON, W.mono_spectrum(T0), "pencil", (50.0, 50.0, z0), (0.0, 0.0, 1.0))
    return W.Problem(ph, src, n_histories, 2, eabs_photon=0.05, eabs_electron=0.2, e_min=0.005,
                     e_max=T0 * 1.05, flags=W.FLAG_NO_HARD, request_id=request_id)


def mass_depth_moment(dose, rho):
    """(energy-weighted mass depth in g/cm^2, energy per history in MeV)."""
    rho = np.asarray(rho, np.float64)
    faces = np.concatenate([[0.0], np.cumsum(rho * DZ)])
    e = np.asarray(dose, np.float64) * rho * (AREA * DZ)
    mc = 0.5 * (faces[:-1] + faces[1:])
    return float((e * mc).sum() / e.sum()), float(e.sum())


def mass_depth_second_moment(dose, rho, m0):
    """Energy-weighted (m - m0)^2 in mass depth (g^2/cm^4), with each voxel's
    (rho DZ)^2/12 of positions spread over it."""
    rho = np.asarray(rho, np.float64)
    faces = np.concatenate([[0.0], np.cumsum(rho * DZ)])
    e = np.asarray(dose, np.float64) * rho * (AREA * DZ)
    mc = 0.5 * (faces[:-1] + faces[1:]) - m0
    return float((e * (mc * mc + (rho * DZ) ** 2 / 12.0)).sum() / e.sum())
