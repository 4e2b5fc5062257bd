// Interpolation tables (Sec. 2.2.2), built on the device in FP64 and stored
// as FP32.  Physics readings (the paper defers all formulas to DPM):
//   Compton: free-electron Klein-Nishina, mu = n_e sigma_KN.
//   Photoelectric: mu/rho = C_PE sum_i n_i Z_i^4 / E^3, C_PE fixed so that
//     water's mu_pe equals its Compton mu at 30 keV.
//   Pair: sum_i n_i alpha re^2 Z(Z+1) [28/9 ln(183 Z^-1/3) - 2/27] ((k-2)/k)^3.
//   Electrons: Bethe collision stopping power (no density effect) minus the
//     hard Moller loss above W_cc, plus soft Kramers radiation B*min(T,W_cb)
//     with dSigma_b/dk = B/k; B = 4 alpha re^2 sum_i n_i Z(Z+1) ln(183 Z^-1/3)
//     also gives X0 = 1/B.  Hard Moller cross section on W in [W_cc, T/2],
//     hard bremsstrahlung B ln(T/W_cb).
//   CSDA range R(T) = int_{E_abs}^{T} dT'/S_r(T'); multiple-scattering step
//     x_ms(T) = R(T) - R(keep*T); screened-Rutherford parameter A solving
//     2A[(1+A) ln(1+1/A) - 1] = G1.
#include <cmath>
#include <cstdio>
#include <cstring>

#include "internal.h"

namespace gdpm {
namespace {

constexpr double kRe = 2.8179403262e-13;
constexpr double kAlpha = 1.0 / 137.035999084;
constexpr double kNA = 6.02214076e23;
constexpr double kPi = 3.14159265358979323846;
constexpr double kCpe = 3.9365358876e-32;

struct Build {
    const MatDev* mats;
    int n_mat, n, n_r, n_a;
    double lemin, dle;
    double eabs_ph, eabs_el, ms_keep;
    int flags;
    double a_l1lo, a_dl;
    // FP64 scratch, [m*n + i]
    double *mu_c, *mu_pe, *mu_pair, *sig_m, *sig_b, *intv, *R;
    double* scal;          // per material: 0 x0, 1 sigmax, 2 r_eabs, 3 rinv_lo, 4 rinv_hi
    // FP32 outputs
    float* ph_tot;
    float2* ph_cum;
    float4* el;
    float* rinv;
    float* atab;
};

// ---------------------------------------------------------------- material sums
__device__ double mat_ne(const MatDev& m) {
    double s = 0.0;
    for (int i = 0; i < m.n; ++i) s += m.w[i] * double(m.Z[i]) / m.A[i];
    return kNA * s;
}
__device__ double mat_sum(const MatDev& m, int kind) {
    // kind 0: sum n_i Z^4; 1: pair bracket; 2: bremsstrahlung bracket
    double s = 0.0;
    for (int i = 0; i < m.n; ++i) {
        const double z = m.Z[i], ni = kNA * m.w[i] / m.A[i];
        const double lscr = log(183.0 / cbrt(z));
        if (kind == 0) s += ni * (z * z) * (z * z);
        else if (kind == 1) s += ni * z * (z + 1.0) * (28.0 / 9.0 * lscr - 2.0 / 27.0);
        else s += ni * z * (z + 1.0) * lscr;
    }
    return s;
}

// ---------------------------------------------------------------- photon physics
__device__ double sigma_kn(double E) {
    const double k = E / kMC2, a = 1.0 + 2.0 * k, l = log(a);
    const double t1 = (1.0 + k) / (k * k) * (2.0 * (1.0 + k) / a - l / k);
    const double t2 = 0.5 * l / k;
    const double t3 = (1.0 + 3.0 * k) / (a * a);
    return 2.0 * kPi * kRe * kRe * (t1 + t2 - t3);
}

// ---------------------------------------------------------------- electron physics
struct Eph {
    double ne, bconst, I;
};

__device__ double bethe(const Eph& q, double T) {
    const double tau = T / kMC2, g = tau + 1.0;
    const double beta2 = tau * (tau + 2.0) / (g * g);
    const double x = q.I / kMC2;
    const double F = 1.0 - beta2 + (0.125 * tau * tau - (2.0 * tau + 1.0) * 0.69314718055994531) / (g * g);
    return 2.0 * kPi * kRe * kRe * kMC2 * q.ne / beta2 * (log(tau * tau * (tau + 2.0) / (2.0 * x * x)) + F);
}

// Hard Moller cross section and energy loss, closed forms of the integrals
// of the Moller density over eps = W/T in [W_cc/T, 1/2].
__device__ void moller_hard(const Eph& q, double T, double wcc, double& sig, double& loss) {
    if (T <= 2.0 * wcc) { sig = 0.0; loss = 0.0; return; }
    const double tau = T / kMC2, g = tau + 1.0;
    const double beta2 = tau * (tau + 2.0) / (g * g);
    const double c1 = (tau / g) * (tau / g), c2 = (2.0 * tau + 1.0) / (g * g);
    const double K = q.ne * 2.0 * kPi * kRe * kRe * kMC2 / beta2;
    const double e = wcc / T, oe = 1.0 - e;
    // int (1/e^2 + 1/(1-e)^2 + c1 - c2/(e(1-e))) de
    sig = K / T * ((1.0 / e - 2.0) + (2.0 - 1.0 / oe) + c1 * (0.5 - e) - c2 * log(oe / e));
    // int e * (...) de
    const double ln2 = 0.69314718055994531;
    loss = K * (-log(2.0 * e) + (2.0 - ln2 - 1.0 / oe - log(oe)) + c1 * (0.125 - 0.5 * e * e) -
                c2 * (ln2 + log(oe)));
}

__device__ double s_restricted(const Eph& q, double T, double wcc, double wcb) {
    double sig, loss;
    moller_hard(q, T, wcc, sig, loss);
    return bethe(q, T) - loss + q.bconst * fmin(T, wcb);
}

// int_a^b dT/S_r(T) with T = e^s, composite Simpson in s (32 panels),
// split at the kinks of S_r (T = 2 W_cc and T = W_cb).  Called by a whole
// warp: lane k takes Simpson node k of each piece (lane 0 also node 32) and
// the weighted values are summed across the warp; every lane gets the sum.
__device__ double range_piece(const Eph& q, double a, double b, double wcc, double wcb) {
    if (b <= a) return 0.0;
    double cuts[4] = {a, 0.0, 0.0, b};
    int nc = 1;
    const double k1 = fmin(2.0 * wcc, wcb), k2 = fmax(2.0 * wcc, wcb);
    if (k1 > a && k1 < b) cuts[nc++] = k1;
    if (k2 > a && k2 < b && k2 != k1) cuts[nc++] = k2;
    cuts[nc] = b;
    const int lane = int(threadIdx.x & 31u);
    constexpr int np = 32;
    double total = 0.0;
    for (int c = 0; c < nc; ++c) {
        const double sa = log(cuts[c]), sb = log(cuts[c + 1]);
        const double h = (sb - sa) / np;
        auto node = [&](int k) {
            const double T = exp(sa + k * h);
            const double wgt = (k == 0 || k == np) ? 1.0 : ((k & 1) ? 4.0 : 2.0);
            return wgt * T / s_restricted(q, T, wcc, wcb);
        };
        double acc = node(lane);
        if (lane == 0) acc += node(np);
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xFFFFFFFFu, acc, o);
        total += acc * h / 3.0;
    }
    return total;
}

__device__ Eph eph_of(const MatDev& m) {
    Eph q;
    q.ne = mat_ne(m);
    q.bconst = 4.0 * kAlpha * kRe * kRe * mat_sum(m, 2);
    q.I = m.I;
    return q;
}

__device__ double r_interp(const double* R, double lemin, double dle, int n, double T) {
    const double u = (log(T) - lemin) / dle;
    int i = int(floor(u));
    i = i < 0 ? 0 : (i > n - 2 ? n - 2 : i);
    double f = u - i;
    f = f < 0.0 ? 0.0 : (f > 1.0 ? 1.0 : f);
    return R[i] + f * (R[i + 1] - R[i]);
}

// ---------------------------------------------------------------- kernels
// One warp per table point (material m, energy i): lane 0 stores the point
// values, the warp shares the range integral over [E_{i-1}, E_i].
__global__ void k_point(Build B) {
    const int idx = int((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (idx >= B.n_mat * B.n) return;
    const int m = idx / B.n, i = idx % B.n;
    const MatDev& mt = B.mats[m];
    const double E = exp(B.lemin + i * B.dle);
    const bool conly = (B.flags & GDPM_FLAG_COMPTON_ONLY) != 0;
    const double k = E / kMC2;
    const double th = k > 2.0 ? (k - 2.0) / k : 0.0;
    const Eph q = eph_of(mt);
    const double iv = i > 0 ? range_piece(q, exp(B.lemin + (i - 1) * B.dle), E, B.eabs_el, B.eabs_ph) : 0.0;
    if ((threadIdx.x & 31u) != 0u) return;
    B.mu_c[idx] = mat_ne(mt) * sigma_kn(E);
    B.mu_pe[idx] = conly ? 0.0 : kCpe * mat_sum(mt, 0) / (E * E * E);
    B.mu_pair[idx] = conly ? 0.0 : kAlpha * kRe * kRe * mat_sum(mt, 1) * th * th * th;
    double sig, loss;
    moller_hard(q, E, B.eabs_el, sig, loss);
    B.sig_m[idx] = sig;
    B.sig_b[idx] = E > B.eabs_ph ? q.bconst * log(E / B.eabs_ph) : 0.0;
    B.intv[idx] = iv;
}

// Per material (one warp each): accumulate the range, shift it to
// R(E_abs) = 0, majorant of the hard cross sections, X0.  The running sum
// goes 32 points at a time: an inclusive shuffle scan of the chunk plus the
// total so far.
__global__ void k_scan(Build B) {
    const int m = int(blockIdx.x);
    const int lane = int(threadIdx.x & 31u);
    if (m >= B.n_mat) return;
    const int n = B.n;
    double* R = B.R + size_t(m) * n;
    const double* I = B.intv + size_t(m) * n;
    double carry = 0.0;
    for (int i0 = 0; i0 < n; i0 += 32) {
        const int i = i0 + lane;
        double v = (i > 0 && i < n) ? I[i] : 0.0;
        for (int o = 1; o < 32; o <<= 1) {
            const double u = __shfl_up_sync(0xFFFFFFFFu, v, o);
            if (lane >= o) v += u;
        }
        if (i < n) R[i] = carry + v;
        carry += __shfl_sync(0xFFFFFFFFu, v, 31);
    }
    __syncwarp();
    const Eph q = eph_of(B.mats[m]);
    // c = int_{E_0}^{E_abs} dT/S_r
    const double le = log(B.eabs_el);
    int k = int(floor((le - B.lemin) / B.dle));
    k = k < 0 ? 0 : (k > n - 1 ? n - 1 : k);
    const double Ek = exp(B.lemin + k * B.dle);
    const double c = R[k] + (B.eabs_el >= Ek ? range_piece(q, Ek, B.eabs_el, B.eabs_el, B.eabs_ph)
                                             : -range_piece(q, B.eabs_el, Ek, B.eabs_el, B.eabs_ph));
    double smax = 0.0;
    for (int i = lane; i < n; i += 32) {
        R[i] -= c;
        const double s = B.sig_m[size_t(m) * n + i] + B.sig_b[size_t(m) * n + i];
        smax = s > smax ? s : smax;
    }
    for (int o = 16; o > 0; o >>= 1) smax = fmax(smax, __shfl_xor_sync(0xFFFFFFFFu, smax, o));
    __syncwarp();
    if (lane != 0) return;
    double* sc = B.scal + 8 * m;
    sc[0] = 1.0 / q.bconst;
    sc[1] = smax;
    sc[2] = r_interp(R, B.lemin, B.dle, n, B.eabs_el);
    sc[3] = sc[2];
    sc[4] = R[n - 1];
}

__global__ void k_derived(Build B) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= B.n_mat * B.n) return;
    const int m = idx / B.n, i = idx % B.n;
    const double* R = B.R + size_t(m) * B.n;
    const double E = exp(B.lemin + i * B.dle);
    const double xms = R[i] - r_interp(R, B.lemin, B.dle, B.n, B.ms_keep * E);
    B.ph_tot[idx] = float(B.mu_c[idx] + B.mu_pe[idx] + B.mu_pair[idx]);
    B.ph_cum[idx] = make_float2(float(B.mu_c[idx]), float(B.mu_c[idx] + B.mu_pe[idx]));
    B.el[idx] = make_float4(float(R[i]), float(xms), float(B.sig_m[idx]), float(B.sig_b[idx]));
}

// Range inverse on a uniform grid in r: exact inverse of the FP64 range
// interpolant (binary search, then inverse linear interpolation in ln E).
__global__ void k_rinv(Build B) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= B.n_mat * B.n_r) return;
    const int m = idx / B.n_r, j = idx % B.n_r;
    const double* R = B.R + size_t(m) * B.n;
    const double lo = B.scal[8 * m + 3], hi = B.scal[8 * m + 4];
    const double r = lo + (hi - lo) * j / double(B.n_r - 1);
    int a = 0, b = B.n - 1;
    double T;
    if (r <= R[0]) T = exp(B.lemin);
    else if (r >= R[b]) T = exp(B.lemin + b * B.dle);
    else {
        while (b - a > 1) {
            const int c = (a + b) >> 1;
            if (R[c] <= r) a = c; else b = c;
        }
        const double f = (r - R[a]) / (R[a + 1] - R[a]);
        T = exp(B.lemin + (a + f) * B.dle);
    }
    B.rinv[idx] = float(T);
}

// ln A as a function of ln G1 for the screened-Rutherford distribution.
__global__ void k_atab(Build B) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= B.n_a) return;
    const double g1 = exp(B.a_l1lo + k * B.a_dl);
    // bisection on [-80, 40]: 72 halvings leave 120 / 2^72 = 2.5e-20, below
    // the FP64 spacing of any root the table needs
    double lo = -80.0, hi = 40.0;
    for (int it = 0; it < 72; ++it) {
        const double mid = 0.5 * (lo + hi), A = exp(mid);
        const double h = 2.0 * A * ((1.0 + A) * log1p(1.0 / A) - 1.0);
        if (h < g1) lo = mid; else hi = mid;
    }
    B.atab[k] = float(0.5 * (lo + hi));
}

}  // namespace

int build_tables_device(gdpm_ctx* ctx, gdpm_tables* t, const gdpm_material_desc* mats) {
    const int M = t->n_mat, n = t->n_e;
    t->n_r = 2 * n;
    t->n_a = 1024;
    std::vector<MatDev> hm(M);
    for (int m = 0; m < M; ++m) {
        const gdpm_material_desc& d = mats[m];
        double wsum = 0;
        for (int i = 0; i < d.n_elements; ++i) wsum += d.mass_fraction[i];
        hm[m].n = d.n_elements;
        for (int i = 0; i < d.n_elements; ++i) {
            hm[m].Z[i] = d.Z[i];
            hm[m].A[i] = d.A[i];
            hm[m].w[i] = d.mass_fraction[i] / wsum;
        }
        hm[m].I = d.mean_excitation_MeV;
    }
    Buffer dm, scratch, scal;
    const size_t mn = size_t(M) * n;
    int rc;
    if ((rc = ensure(dm, sizeof(MatDev) * M)) || (rc = ensure(scratch, sizeof(double) * mn * 7)) ||
        (rc = ensure(scal, sizeof(double) * 8 * M)) ||
        (rc = ensure(t->ph_tot, sizeof(float) * mn)) || (rc = ensure(t->ph_cum, sizeof(float2) * mn)) ||
        (rc = ensure(t->el, sizeof(float4) * mn)) ||
        (rc = ensure(t->rinv, sizeof(float) * M * t->n_r)) ||
        (rc = ensure(t->atab, sizeof(float) * t->n_a))) {
        release(dm); release(scratch); release(scal);
        return rc;
    }
    Build B{};
    B.mats = static_cast<const MatDev*>(dm.p);
    B.n_mat = M; B.n = n; B.n_r = t->n_r; B.n_a = t->n_a;
    B.lemin = std::log(t->e_min);
    B.dle = (std::log(t->e_max) - std::log(t->e_min)) / (n - 1);
    B.eabs_ph = t->eabs_ph; B.eabs_el = t->eabs_el; B.ms_keep = 1.0 - t->ms_loss;
    B.flags = t->flags;
    const double g1lo = 1e-10, g1hi = 0.999;
    B.a_l1lo = std::log(g1lo);
    B.a_dl = (std::log(g1hi) - std::log(g1lo)) / (t->n_a - 1);
    double* s = static_cast<double*>(scratch.p);
    B.mu_c = s; B.mu_pe = s + mn; B.mu_pair = s + 2 * mn; B.sig_m = s + 3 * mn;
    B.sig_b = s + 4 * mn; B.intv = s + 5 * mn; B.R = s + 6 * mn;
    B.scal = static_cast<double*>(scal.p);
    B.ph_tot = static_cast<float*>(t->ph_tot.p);
    B.ph_cum = static_cast<float2*>(t->ph_cum.p);
    B.el = static_cast<float4*>(t->el.p);
    B.rinv = static_cast<float*>(t->rinv.p);
    B.atab = static_cast<float*>(t->atab.p);
    cudaStream_t st = ctx->stream;
    GDPM_CUDA_TRY(cudaMemcpyAsync(dm.p, hm.data(), sizeof(MatDev) * M, cudaMemcpyHostToDevice, st));
    const int th = 128;
    k_point<<<int((mn * 32 + th - 1) / th), th, 0, st>>>(B);
    k_scan<<<M, 32, 0, st>>>(B);
    k_derived<<<int((mn + th - 1) / th), th, 0, st>>>(B);
    k_rinv<<<int((size_t(M) * t->n_r + th - 1) / th), th, 0, st>>>(B);
    // the screened-Rutherford table depends on no material or grid: the
    // context computes it once and copies it into later table sets
    const size_t atab_bytes = sizeof(float) * size_t(t->n_a);
    if (ctx->atab_cache.p && ctx->atab_cache.bytes >= atab_bytes) {
        GDPM_CUDA_TRY(cudaMemcpyAsync(t->atab.p, ctx->atab_cache.p, atab_bytes, cudaMemcpyDeviceToDevice, st));
    } else {
        k_atab<<<(t->n_a + 31) / 32, 32, 0, st>>>(B);
        if (ensure(ctx->atab_cache, atab_bytes) == GDPM_OK)
            GDPM_CUDA_TRY(cudaMemcpyAsync(ctx->atab_cache.p, t->atab.p, atab_bytes, cudaMemcpyDeviceToDevice, st));
    }
    GDPM_CUDA_TRY(cudaGetLastError());
    std::vector<double> hs(8 * M);
    GDPM_CUDA_TRY(cudaMemcpyAsync(hs.data(), scal.p, sizeof(double) * 8 * M, cudaMemcpyDeviceToHost, st));
    GDPM_CUDA_TRY(cudaStreamSynchronize(st));
    release(dm); release(scratch); release(scal);

    DevTables& T = t->dev;
    T.n_mat = M; T.n_e = n; T.n_r = t->n_r; T.n_a = t->n_a;
    T.l2min = float(std::log2(t->e_min));
    T.inv_dl2 = float((n - 1) / (std::log2(t->e_max) - std::log2(t->e_min)));
    T.ph_tot = B.ph_tot; T.ph_cum = B.ph_cum; T.el = B.el; T.rinv = B.rinv; T.atab = B.atab;
    T.a_l1lo = float(B.a_l1lo);
    T.a_idl = float(1.0 / B.a_dl);
    T.a_g1hi = float(g1hi);
    for (int m = 0; m < M; ++m) {
        const double* sc = &hs[8 * m];
        T.x0[m] = float(sc[0]);
        T.inv_x0[m] = float(1.0 / sc[0]);
        T.sigmax[m] = float(sc[1]);
        T.inv_sigmax[m] = sc[1] > 0 ? float(1.0 / sc[1]) : 0.f;
        T.r_eabs[m] = float(sc[2]);
        T.rinv_lo[m] = float(sc[3]);
        T.rinv_idr[m] = float((t->n_r - 1) / (sc[4] - sc[3]));
    }
    T.eabs_ph = float(t->eabs_ph);
    T.eabs_el = float(t->eabs_el);
    T.ms_keep = float(1.0 - t->ms_loss);
    T.flags = t->flags;
    return GDPM_OK;
}

}  // namespace gdpm
