// Transport kernels of the gDPM method on sm_103a.
//
// Photon and electron transport run in separate phases (Sec. 2.2.1: only
// one particle type is in flight at a time; secondaries go to per-type
// stacks).  Each phase is one persistent launch: every warp keeps its 32
// lanes busy by refilling a lane from the phase's input (a queue of banked
// particles, plus freshly generated primaries) whenever the lane's particle
// terminates, so warps stay full until the input is drained instead of
// idling on their longest history.  A lane advances its particle by one
// step per iteration:
//   photon:   Woodcock flights against the majorant until a real collision
//             (Sec. 2.1), then one Compton / photoelectric / pair event;
//   electron: one condensed-history step (CSDA loss over the step, random
//             hinge multiple scattering, voxel walk depositing along the
//             path) and, at a hard-event candidate, Moller or
//             bremsstrahlung (Sec. 2.1).
// A step runs with whatever lanes it diverges into and uses no warp-wide
// operation.  It leaves its event counts and the secondaries it created in
// registers; at the top of the next iteration, where all 32 lanes are
// present, the warp banks those secondaries into the queues and adds the
// counts with full-warp ballots and reductions.
// Tables live in shared memory (Sec. 2.2.2 reads them by linear
// interpolation); random numbers come from Philox4x32-10 keyed per history
// and particle, so results do not depend on scheduling.
#include <algorithm>
#include <cfloat>

#include "internal.h"

namespace gdpm {
namespace {

constexpr float kInf = FLT_MAX;
constexpr float kEs = 21.2f;            // Rossi-Greisen scattering energy, MeV
constexpr uint32_t kFull = 0xffffffffu;

// CTA shape each phase kernel is compiled for: threads per CTA and the
// resident CTAs per SM that fix its register budget.  The photon kernel fits
// 64 registers at 4 x 256 threads; so does the whole-step electron kernel,
// with a few spilled words, and the extra warps hide more latency than the
// spills cost (6 MV slab electron phase -4.6 %).  The resumable electron
// kernel keeps its step state across the loop top: at 2 x 448 threads (72
// registers, 24 bytes spilled, 28 warps per SM) it beats 3 x 256 (80
// registers, no spill, 24 warps) by 2.7 % on the CT plan; at 4 x 256 (64
// registers) it spills that state, +12 %.
#ifndef GDPM_MIN_CTAS_PHOTON
#define GDPM_MIN_CTAS_PHOTON 4
#endif
#ifndef GDPM_MIN_CTAS_ELECTRON_WHOLE
#define GDPM_MIN_CTAS_ELECTRON_WHOLE 4
#endif
#ifndef GDPM_THREADS_ELECTRON
#define GDPM_THREADS_ELECTRON 448
#endif
#ifndef GDPM_MIN_CTAS_ELECTRON
#define GDPM_MIN_CTAS_ELECTRON 2
#endif
template <int PT>
struct PhaseShape {
    static constexpr int threads = PT == 2 ? GDPM_THREADS_ELECTRON : 256;
    static constexpr int ctas = PT == 0 ? GDPM_MIN_CTAS_PHOTON
                                : PT == 1 ? GDPM_MIN_CTAS_ELECTRON_WHOLE
                                          : GDPM_MIN_CTAS_ELECTRON;
};

// Threads per CTA of phase kernel PT: its own shape, or the context's
// GDPM_PARAM_BLOCK_THREADS when set (at most 256, within every kernel's bound).
int phase_threads(const gdpm_ctx* ctx, int pt) {
    if (ctx->block_threads > 0) return ctx->block_threads;
    return pt == 0 ? PhaseShape<0>::threads : pt == 1 ? PhaseShape<1>::threads : PhaseShape<2>::threads;
}

// ---------------------------------------------------------------- ledger/tally
struct Acc {
    double src, esc, disc;
};

// Per-lane event counters: one byte per kind of event, four kinds to a
// word, plus the flight (photon) or voxel-crossing (electron) count.  Each
// kind happens at most once per lane and iteration, so folding the bytes
// into the block's counters every kFlushEvery (< 256) iterations keeps them
// from overflowing.
struct Ev {
    uint32_t a, b, c, n;
};
constexpr uint32_t EV_REAL = 1u, EV_COMPTON = 1u << 8, EV_PHOTO = 1u << 16, EV_PAIR = 1u << 24;  // a
constexpr uint32_t EV_TERM = 1u, EV_LOCAL = 1u << 8, EV_STEP = 1u << 16, EV_MOLLER = 1u << 24;   // b
constexpr uint32_t EV_BREMS = 1u, EV_ANNIHIL = 1u << 8;                                          // c
constexpr uint32_t kFlushEvery = 128u;

// Secondaries created by one step: n of them (0..2) at the particle's
// current position; the second is a positron (pair) or, for photons, the
// back-to-back partner (annihilation).
struct Sec {
    int n;
    bool photon, pos2;
    float E1, E2, dx, dy, dz;
};

// Deposit e MeV in voxel vox of the tally of the batch in `flags`.
__device__ __forceinline__ void tally(const SimParams& P, uint32_t flags, uint32_t vox0, float e) {
    size_t vox = size_t(vox0) + size_t((flags & kBatchMask) >> kBatchShift) * P.batch_stride;
#if GDPM_CHECKED
    if (vox < P.tally_lo || vox >= P.tally_hi) {
        bounds_fail(P.status, ST_B_TALLY);
        vox = P.tally_lo;
    }
#endif
    if (P.tally_mode == 0) {
        atomicAdd(&P.edep[vox], double(e));
    } else {
        // FP32 pair: hi accumulates, lo collects the exact rounding error of
        // each addition (TwoSum on the value the atomic returned).
        const float old = atomicAdd(&P.edep_hi[vox], e);
        const float s = old + e;
        const float bb = s - old;
        const float err = (old - (s - bb)) + (e - bb);
        if (err != 0.f) atomicAdd(&P.edep_lo[vox], err);
    }
}

__device__ __forceinline__ uint32_t vox_of(const SimParams& P, int ix, int iy, int iz) {
    return uint32_t(ix) + uint32_t(P.nx) * (uint32_t(iy) + uint32_t(P.ny) * uint32_t(iz));
}

__device__ __forceinline__ void hist_count(const SimParams& P, uint32_t hist, int k) {
    if (P.hrec) atomicAdd(&P.hrec[size_t(GDPM_IDX(P.status, hist, P.n_records, ST_B_RECORD)) * 4 + k], 1);
}
__device__ __forceinline__ void hist_add(const SimParams& P, uint32_t hist, int k, double v) {
    if (P.hrec) atomicAdd(&P.hrecd[size_t(GDPM_IDX(P.status, hist, P.n_records, ST_B_RECORD)) * 2 + k], v);
}
#if GDPM_CHECKED
__device__ __forceinline__ uint32_t n_voxels(const SimParams& P) {
    return uint32_t(P.nx) * uint32_t(P.ny) * uint32_t(P.nz);
}
#endif

// ---------------------------------------------------------------- samplers
// Klein-Nishina in eps = E'/E by the two-branch mixture method: with weight
// ln(1/eps0) sample from 1/eps, with weight (1-eps0^2)/2 from eps, accept
// with 1 - eps sin^2(theta)/(1+eps^2).  Draws: (branch, eps, accept, phi).
__device__ __forceinline__ void sample_kn(Part& p, const SimParams& P, float E, float& eps,
                                          float& cost, float& rphi) {
    const float k = E * (1.f / kMC2f);
    const float e0 = 1.f / fmaf(2.f, k, 1.f);
    const float a1 = -__logf(e0), a2 = 0.5f * (1.f - e0 * e0);
    float t = 0.f;
    eps = 1.f;
    rphi = 0.5f;
    for (int it = 0; it < 4096; ++it) {
        const float4 c = draw(p, P.key0, P.key1);
        if (c.x * (a1 + a2) < a1) eps = __expf(-a1 * c.y);
        else eps = sqrtf(fmaf(1.f - e0 * e0, c.y, e0 * e0));
        t = (1.f - eps) / (k * eps);
        const float g = 1.f - eps * t * (2.f - t) / fmaf(eps, eps, 1.f);
        rphi = c.w;
        if (c.z <= g) break;
    }
    cost = 1.f - t;
}

// Moller: eps = W/T on [W_cc/T, 1/2] from the 1/eps^2 proposal, accepted with
// eps^2 f(eps) / (2 + c1/4).  Draws: (eps, accept, phi, -).
__device__ __forceinline__ void sample_moller(Part& p, const SimParams& P, float T, float wcc,
                                              float& eps, float& rphi) {
    const float tau = T * (1.f / kMC2f);
    const float g = tau / (tau + 1.f);
    const float c1 = g * g, c2 = (2.f * tau + 1.f) / ((tau + 1.f) * (tau + 1.f));
    const float ec = wcc / T;
    const float bound = 2.f + 0.25f * c1;
    eps = ec;
    rphi = 0.5f;
    for (int it = 0; it < 4096; ++it) {
        const float4 w = draw(p, P.key0, P.key1);
        eps = ec / (1.f - w.x * (1.f - 2.f * ec));
        const float x = eps / (1.f - eps);
        const float gg = 1.f + x * x + c1 * eps * eps - c2 * x;
        rphi = w.z;
        if (w.y * bound <= gg) break;
    }
}

// Sauter's K-shell photoelectron distribution (physics variant) in
// mu = cos(theta), for kinetic energy T: p(mu) ~ (1-mu^2)/(1-beta mu)^4
// [1 + b (1 - beta mu)], b = gamma(gamma-1)(gamma-2)/2.  Proposal
// q(mu) ~ 1/(1 - beta mu)^2 by inversion, 1/(1 - beta mu) = 1/(1+beta) +
// xi 2beta/(1-beta^2); accepted with (1-mu^2)(1-beta^2)/(1-beta mu)^2 times
// g/g_max.  Draws per trial: (proposal, accept, phi, -).
__device__ __forceinline__ void sample_sauter(Part& p, const SimParams& P, float T, float& mu,
                                              float& rphi) {
    const float g = 1.f + T * (1.f / kMC2f);
    const float beta = sqrtf(fmaxf(0.f, 1.f - 1.f / (g * g)));
    const float b = 0.5f * g * (g - 1.f) * (g - 2.f);
    const float gmax = b >= 0.f ? 1.f + b * (1.f + beta) : 1.f + b * (1.f - beta);
    const float ib = 1.f / (1.f + beta), sc = 2.f * beta / (1.f - beta * beta);
    mu = 0.f;
    rphi = 0.f;
    for (int it = 0; it < 4096; ++it) {
        const float4 c = draw(p, P.key0, P.key1);
        const float x = ib + c.x * sc;
        const float m = fminf(fmaxf((1.f - 1.f / x) / beta, -1.f), 1.f);
        const float d = 1.f - beta * m;
        const float w = (1.f - m * m) * (1.f - beta * beta) / (d * d) * (1.f + b * d) / gmax;
        mu = m;
        rphi = c.z;
        if (c.y < w) break;
    }
}

// Screening parameter A for first moment G1 (table in ln G1; asymptote
// 1/A = 3d(1 + 3d/2), d = 1 - G1, near isotropy).
__device__ __forceinline__ float screening_A(const DevTables& T, const float* atab, float G1) {
    if (G1 > T.a_g1hi) {
        const float d = 1.f - G1;
        return 1.f / (3.f * d * (1.f + 1.5f * d));
    }
    float kk = (__logf(G1) - T.a_l1lo) * T.a_idl;
    kk = fmaxf(kk, 0.f);
    const int k = min(int(kk), T.n_a - 2);
    const float f = fminf(kk - float(k), 1.f);
    return __expf(lerpf(atab[k], atab[k + 1], f));
}

// ---------------------------------------------------------------- geometry
__device__ __forceinline__ bool inside(const SimParams& P, float x, float y, float z) {
    return x >= 0.f && x <= P.Lx && y >= 0.f && y <= P.Ly && z >= 0.f && z <= P.Lz;
}

__device__ __forceinline__ void voxel_of(const SimParams& P, Part& p) {
    p.ix = min(int(p.x * P.inv_dx), P.nx - 1);
    p.iy = min(int(p.y * P.inv_dy), P.ny - 1);
    p.iz = min(int(p.z * P.inv_dz), P.nz - 1);
}

// Move a primary from outside onto the phantom surface (ray-box slabs); the
// entry coordinate is set exactly on the face.  False if the ray misses.
__device__ bool enter_box(const SimParams& P, Part& p) {
    if (inside(P, p.x, p.y, p.z)) return true;
    const float o[3] = {p.x, p.y, p.z}, d[3] = {p.u, p.v, p.w}, L[3] = {P.Lx, P.Ly, P.Lz};
    float tmin = -kInf, tmax = kInf;
    int amin = -1;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (d[a] == 0.f) {
            if (o[a] < 0.f || o[a] > L[a]) return false;
            continue;
        }
        const float t1 = (0.f - o[a]) / d[a], t2 = (L[a] - o[a]) / d[a];
        const float lo = fminf(t1, t2), hi = fmaxf(t1, t2);
        if (lo > tmin) { tmin = lo; amin = a; }
        if (hi < tmax) tmax = hi;
    }
    if (amin < 0 || tmax <= tmin || tmax <= 0.f) return false;
    float q[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) q[a] = fminf(fmaxf(fmaf(tmin, d[a], o[a]), 0.f), L[a]);
    q[amin] = d[amin] > 0.f ? 0.f : L[amin];
    p.x = q[0]; p.y = q[1]; p.z = q[2];
    return true;
}

// Beamlet of history h as its position in the list of positive-weight
// beamlets (Sec. 2.3.1).  Metropolis picks were made by k_metropolis before
// the phase; the alias method reads the Philox block at (h, 0, 0, 0); the
// cumulative search uses the primary's own uniform rw.
__device__ __forceinline__ int pick_beamlet(const DevSource& S, const PhaseArgs& A, uint32_t idx,
                                            uint32_t h, float rw, uint32_t k0, uint32_t k1,
                                            const float* cdf) {
    if (S.sampler == GDPM_SAMPLE_METROPOLIS) return int(A.bl_pick[idx]);
    if (S.sampler == GDPM_SAMPLE_ALIAS) {
        const uint4 w = philox_block(h, 0u, 0u, 0u, k0, k1);
        const int J = int(__umulhi(w.x, uint32_t(S.n_beamlets)));
        return uint64_t(w.y) < S.al_cut[J] ? J : S.al_alias[J];   // u = (w.y + 1/2) 2^-32 < cut
    }
    // the I with P(I) <= r < P(I+1) (rounded-up FP32 table: the same decisions
    // as comparing double(r) with the FP64 cumulative weights)
    int l = 0, hi = S.n_beamlets - 1;
    while (l < hi) {
        const int mid = (l + hi) >> 1;
        if (rw < cdf[mid]) hi = mid; else l = mid + 1;
    }
    return l;
}

// Primary number `idx` of this phase (Sec. 2.3): energy from the batch's
// spectrum interval allotment (uniform inside the interval), position and
// direction from the source geometry.  Draw 0 of the primary's stream:
// (u-position, v-position, energy, beamlet).
// prefix_tab / cdf_tab: copies of A.bin_prefix and S.bl_cdf (e.g. in shared
// memory), or null to read the originals.
__device__ bool make_primary(const SimParams& P, const PhaseArgs& A, uint32_t idx, Part& p,
                             Acc& acc, const uint32_t* prefix_tab = nullptr,
                             const float* cdf_tab = nullptr) {
    const DevSource& S = P.S;
    const uint32_t h = A.src_first + idx;
    // a dose-matrix run: sub-problem k holds histories [sub_first[k],
    // sub_first[k+1]); its batches are slots k*nb .. k*nb+nb-1
    uint32_t k = 0u, h0 = 0u, nb_small = A.nb_small, nb_rem = A.nb_rem;
    if (A.n_sub) {
        uint32_t lo = 0u, hi = A.n_sub;
        while (hi - lo > 1u) {
            const uint32_t mid = (lo + hi) >> 1;
            if (A.sub_first[mid] <= h) lo = mid; else hi = mid;
        }
        k = lo;
        h0 = A.sub_first[k];
        const uint32_t nk = A.sub_first[k + 1] - h0;
        nb_small = nk / A.sub_batches;
        nb_rem = nk % A.sub_batches;
    }
    // batch b of history h and h's index within it (batches are contiguous;
    // the first nb_rem hold nb_small + 1 histories)
    const uint32_t hl = h - h0;
    const uint32_t big = nb_small + 1u, split = nb_rem * big;
    uint32_t b, local;
    if (hl < split) {
        b = hl / big;
        local = hl - b * big;
    } else {
        b = nb_rem + (hl - split) / nb_small;
        local = (hl - split) - (b - nb_rem) * nb_small;
    }
    const uint32_t slot = A.n_sub ? k * A.sub_batches + b : b;
    const uint32_t* prefix = (prefix_tab ? prefix_tab : A.bin_prefix) + size_t(slot) * (S.n_bins + 1);
    p.hist = h;
    p.pidlo = 1u; p.pidhi = 0u; p.ctr = 0u;
    p.flags = (slot << kBatchShift) & kBatchMask;
    const float4 r = draw(p, P.key0, P.key1);
    int lo = 0, hi = S.n_bins;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (prefix[mid] <= local) lo = mid; else hi = mid;
    }
    p.E = fmaf(S.edges[lo + 1] - S.edges[lo], r.z, S.edges[lo]);
    if (S.geometry == GDPM_GEO_PENCIL) {
        p.x = S.origin[0]; p.y = S.origin[1]; p.z = S.origin[2];
        p.u = S.direction[0]; p.v = S.direction[1]; p.w = S.direction[2];
    } else {
        float src[3], cen[3], au[3], av[3];
        float a0, a1, b0, b1;
        if (S.geometry == GDPM_GEO_POINT_FIELD) {
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                src[a] = S.origin[a]; cen[a] = S.center[a]; au[a] = S.axis_u[a]; av[a] = S.axis_v[a];
            }
            a0 = -S.half_u; a1 = S.half_u; b0 = -S.half_v; b1 = S.half_v;
        } else {
            // a dose-matrix sub-problem is its own beamlet; otherwise sample one
            const int kb = A.n_sub ? int(k)
                                   : pick_beamlet(S, A, idx, h, r.w, P.key0, P.key1, cdf_tab ? cdf_tab : S.bl_cdf);
            // a row is 16 floats, 64 bytes from a 16-byte aligned base: four vector loads
            const float4* row = reinterpret_cast<const float4*>(S.beamlets) +
                                size_t(GDPM_IDX(P.status, kb, S.n_beamlets, ST_B_TABLE)) * 4;
            const float4 q0 = __ldg(row), q1 = __ldg(row + 1), q2 = __ldg(row + 2), q3 = __ldg(row + 3);
            src[0] = q0.x; src[1] = q0.y; src[2] = q0.z;
            cen[0] = q0.w; cen[1] = q1.x; cen[2] = q1.y;
            au[0] = q1.z; au[1] = q1.w; au[2] = q2.x;
            av[0] = q2.y; av[1] = q2.z; av[2] = q2.w;
            a0 = q3.x; a1 = q3.y; b0 = q3.z; b1 = q3.w;
        }
        const float su = fmaf(a1 - a0, r.x, a0), sv = fmaf(b1 - b0, r.y, b0);
        const float ax = cen[0] + su * au[0] + sv * av[0];
        const float ay = cen[1] + su * au[1] + sv * av[1];
        const float az = cen[2] + su * au[2] + sv * av[2];
        p.x = src[0]; p.y = src[1]; p.z = src[2];
        const float dx = ax - p.x, dy = ay - p.y, dz = az - p.z;
        const float n = rsqrtf(dx * dx + dy * dy + dz * dz);
        p.u = dx * n; p.v = dy * n; p.w = dz * n;
    }
    acc.src += p.E;
    if (!enter_box(P, p)) {
        acc.esc += p.E;
        hist_add(P, p.hist, 0, p.E);
        return false;
    }
    voxel_of(P, p);
    return true;
}

// ---------------------------------------------------------------- photon step
// Woodcock flights a photon takes per iteration of the phase loop.  A photon
// crossing air or lung makes many virtual flights against a majorant set by
// bone; past this many it continues in the next iteration, so it does not
// hold the warp while the other lanes interact and are refilled.  Between
// flights a photon carries nothing but its position and draw counter, so
// the cap changes no draw and no result.  3 was measured best against 2, 4,
// 5, 6, 8 and no cap (CT plan: photon phase -17 %).
constexpr int kFlightsPerTrip = 3;

struct PhSmem {
    const float* maj;
    const float* tot;
    const float2* cum;
};

__device__ void photon_step(const SimParams& P, const PhSmem& S, Part& p, bool& active, Acc& acc,
                            Ev& ev, Sec& sec) {
    const DevTables& T = P.T;
    if (p.E < T.eabs_ph) {   // only a source photon below the cutoff reaches here
        tally(P, p.flags, vox_of(P, p.ix, p.iy, p.iz), p.E);
        ev.b += EV_TERM;
        active = false;
        return;
    }
    // Woodcock flights at fixed energy until a real collision (or escape), so
    // that the interaction below runs with the warp's lanes together; at most
    // kFlightsPerTrip of them per iteration.
    int i;
    float f;
    grid_pos(T, p.E, i, f);
    const float mm = lerpf(S.maj[i], S.maj[i + 1], f);
    const float inv_mm = 1.f / mm;
    float4 r;
    uint32_t vox;
    float mt;
    int mi;
    for (int flight = 0;; ++flight) {
        // a photon still in virtual flights after kFlightsPerTrip of them
        // goes on in the next iteration (the same draws: one block a flight)
        if (flight == kFlightsPerTrip) return;
        r = draw(p, P.key0, P.key1);
        const float s = -__logf(r.x) * inv_mm;
        p.x = fmaf(s, p.u, p.x);
        p.y = fmaf(s, p.v, p.y);
        p.z = fmaf(s, p.w, p.z);
        if (!inside(P, p.x, p.y, p.z)) {
            acc.esc += p.E;
            hist_add(P, p.hist, 0, p.E);
            ev.b += EV_TERM;
            active = false;
            return;
        }
        ++ev.n;
        voxel_of(P, p);
        vox = GDPM_IDX(P.status, vox_of(P, p.ix, p.iy, p.iz), n_voxels(P), ST_B_VOXEL);
        const int m = GDPM_IDX(P.status, int(__ldg(&P.mat[vox])), T.n_mat, ST_B_TABLE);
        const float rho = __ldg(&P.rho[vox]);
        mi = m * T.n_e + i;
        mt = lerpf(S.tot[mi], S.tot[mi + 1], f);
        if (r.y * mm < mt * rho) break;             // real; otherwise a virtual (delta) collision
    }
    ev.a += EV_REAL;
    hist_count(P, p.hist, 0);
    const float2 c0 = S.cum[mi], c1 = S.cum[mi + 1];
    const float rr = r.z * mt;
    sec.n = 1;
    sec.photon = false;
    sec.dx = p.u; sec.dy = p.v; sec.dz = p.w;
    if (rr < lerpf(c0.x, c1.x, f)) {
        // Compton (Klein-Nishina); recoil electron along E u - E' u'
        ev.a += EV_COMPTON;
        const float E = p.E;
        float eps, cost, rphi;
        sample_kn(p, P, E, eps, cost, rphi);
        float cp, sp;
        cossin_2pi(rphi, cp, sp);
        rotate(p.u, p.v, p.w, cost, cp, sp);
        const float Ep = eps * E;
        sec.E1 = E - Ep;
        float dx = E * sec.dx - Ep * p.u, dy = E * sec.dy - Ep * p.v, dz = E * sec.dz - Ep * p.w;
        const float en = rsqrtf(dx * dx + dy * dy + dz * dz);
        sec.dx = dx * en; sec.dy = dy * en; sec.dz = dz * en;
        sec.pos2 = false;
        if (Ep < T.eabs_ph) {
            tally(P, p.flags, vox, Ep);
            ev.b += EV_LOCAL + EV_TERM;
            active = false;
        } else {
            p.E = Ep;
        }
    } else if (rr < lerpf(c0.y, c1.y, f)) {
        // photoelectric: photon absorbed, photoelectron along the photon (or
        // at Sauter's angle to it, physics variant)
        ev.a += EV_PHOTO;
        ev.b += EV_TERM;
        sec.E1 = p.E;
        sec.pos2 = false;
        active = false;
        if (T.flags & GDPM_FLAG_SAUTER) {
            float mu, rphi, cp, sp;
            sample_sauter(p, P, p.E, mu, rphi);
            cossin_2pi(rphi, cp, sp);
            rotate(sec.dx, sec.dy, sec.dz, mu, cp, sp);
        }
    } else {
        // pair: electron takes r.w of the kinetic energy, positron the rest
        ev.a += EV_PAIR;
        ev.b += EV_TERM;
        const float tav = p.E - 2.f * kMC2f;
        sec.E1 = r.w * tav;
        sec.E2 = tav - sec.E1;
        sec.n = 2;
        sec.pos2 = true;
        active = false;
    }
}

// ---------------------------------------------------------------- electron step
struct ElSmem {
    const float4* el;
    const float* rinv;
    const float* atab;
};

// The electron phase runs in one of two forms with identical arithmetic
// (GDPM_PARAM_ELECTRON_WALK): a lane takes a whole condensed-history step
// per iteration of the phase loop (kernel k_phase<1>), or a resumable step
// whose voxel walk takes at most kWalkTrips trips of the DDA loop per
// iteration and resumes in the next (k_phase<2>).  The resumable form keeps
// a lane with many voxel crossings from holding its warp while the other
// lanes' steps end and they are refilled; it pays for that with step state
// that lives across the loop top.
constexpr int kWalkTrips = 3;

// An electron step in progress: the CH step of Sec. 2.1 is set up once
// (limits, end energy, hinge deflection), then its straight legs are walked
// through the voxels over one or more loop iterations.
struct ElStep {
    float left;        // mass thickness left in the current leg (g/cm2)
    float m1;          // mass thickness of the second leg
    float dpm;         // energy loss per unit mass thickness along the step
    float u1, v1, w1;  // resumable form: the direction after the hinge; whole-step
                       // form: the deflection cos(theta), cos(phi), sin(phi)
    float Tend;        // energy at the end of the step
    float dep;         // energy of the step tallied or owed to a voxel so far
    float rho;         // density of the particle's current voxel
    int leg;           // 0: no step in progress; 1 or 2: walking that leg
    int lim_m;         // what ends the step (bits 0-1), start material (bits 2+)
};

// Voxel walk (3-D DDA) of the step in progress, depositing dpm MeV per
// g/cm2 in each voxel: along leg 1 (zeta x_s), turn to the deflected
// direction at the hinge, along leg 2 ((1 - zeta) x_s).  pend is energy
// already owed to the current voxel but not yet tallied: it goes out with
// the first piece tallied on leaving the voxel, so a track issues one atomic
// per voxel it visits rather than one per piece; the last piece of leg 2 is
// left to the caller.  Returns 0 when the trip budget ran out (resumable
// form), 1 at the end of leg 2, 2 when the particle left the phantom.
//
// One DDA trip: the particle either ends its leg inside the current voxel
// (1) or moves to the voxel's exit face, tallies, and crosses (0, or 2 when
// it leaves the phantom).
__device__ __forceinline__ int walk_trip(const SimParams& P, Part& p, ElStep& s, float iu, float iv,
                                         float iw, int sx, int sy, int sz, uint32_t& vox,
                                         uint32_t& crossings, float& pend) {
    const float tx = p.u != 0.f ? (float(p.ix + (sx > 0)) * P.dx - p.x) * iu : kInf;
    const float ty = p.v != 0.f ? (float(p.iy + (sy > 0)) * P.dy - p.y) * iv : kInf;
    const float tz = p.w != 0.f ? (float(p.iz + (sz > 0)) * P.dz - p.z) * iw : kInf;
    float tb;
    int ab;
    if (tx <= ty && tx <= tz) { tb = tx; ab = 0; }
    else if (ty <= tz) { tb = ty; ab = 1; }
    else { tb = tz; ab = 2; }
    tb = fmaxf(tb, 0.f);
    const float rho = s.rho;
    if (rho * tb >= s.left) {
        // the leg ends in this voxel
        const float t = s.left / rho;
        p.x = fmaf(t, p.u, p.x);
        p.y = fmaf(t, p.v, p.y);
        p.z = fmaf(t, p.w, p.z);
        return 1;
    }
    p.x = fmaf(tb, p.u, p.x);
    p.y = fmaf(tb, p.v, p.y);
    p.z = fmaf(tb, p.w, p.z);
    const float piece = rho * tb;
    const float e = s.dpm * piece;
    if (e + pend > 0.f) tally(P, p.flags, vox, e + pend);
    s.dep += e;
    pend = 0.f;
    s.left -= piece;
    ++crossings;
    if (ab == 0) {
        p.ix += sx;
        if (p.ix < 0 || p.ix >= P.nx) return 2;
        vox += sx;
    } else if (ab == 1) {
        p.iy += sy;
        if (p.iy < 0 || p.iy >= P.ny) return 2;
        vox = sy > 0 ? vox + P.nx : vox - P.nx;
    } else {
        p.iz += sz;
        if (p.iz < 0 || p.iz >= P.nz) return 2;
        const uint32_t plane = uint32_t(P.nx) * uint32_t(P.ny);
        vox = sz > 0 ? vox + plane : vox - plane;
    }
    vox = GDPM_IDX(P.status, uint32_t(vox), n_voxels(P), ST_B_VOXEL);
    s.rho = __ldg(&P.rho[vox]);
    return 0;
}

// The hinge: the rest of leg 1 stays owed to the current voxel, then the
// particle turns to the deflected direction (precomputed by the resumable
// form, rotated here by the whole-step form) and starts leg 2.
template <bool RESUME>
__device__ __forceinline__ void hinge(Part& p, ElStep& s, float& pend) {
    pend += s.dpm * s.left;
    s.dep += s.dpm * s.left;
    if (RESUME) {
        p.u = s.u1; p.v = s.v1; p.w = s.w1;
    } else {
        rotate(p.u, p.v, p.w, s.u1, s.v1, s.w1);
    }
    s.leg = 2;
    s.left = s.m1;
}

// Whole-step form: the legs one after another, with the warp's lanes
// finishing leg 1 together before any turns.  The trip loop ends by
// construction: within a leg the signs sx, sy, sz are fixed, so every trip
// either ends the leg or moves one voxel index one step in its fixed
// direction (a NaN position falls to the z branch), and the walk leaves the
// grid within nx + ny + nz trips.  (A counted guard here cost 8-14 % of the
// electron phase in code generation, for no case it could catch.)
__device__ int walk_whole(const SimParams& P, Part& p, ElStep& s, uint32_t& crossings, float& pend) {
#pragma unroll 1
    for (;;) {
        const float iu = p.u != 0.f ? 1.f / p.u : 0.f;
        const float iv = p.v != 0.f ? 1.f / p.v : 0.f;
        const float iw = p.w != 0.f ? 1.f / p.w : 0.f;
        const int sx = p.u > 0.f ? 1 : -1, sy = p.v > 0.f ? 1 : -1, sz = p.w > 0.f ? 1 : -1;
        uint32_t vox = vox_of(P, p.ix, p.iy, p.iz);
        int res;
#pragma unroll 1
        do {
            res = walk_trip(P, p, s, iu, iv, iw, sx, sy, sz, vox, crossings, pend);
        } while (res == 0);
        if (res == 2 || s.leg == 2) return res;
        hinge<false>(p, s, pend);
    }
}

// Resumable form: at most kWalkTrips trips, turning at the hinge within the
// budget.
__device__ int walk_resumable(const SimParams& P, Part& p, ElStep& s, uint32_t& crossings,
                              float& pend) {
    float iu = p.u != 0.f ? 1.f / p.u : 0.f;
    float iv = p.v != 0.f ? 1.f / p.v : 0.f;
    float iw = p.w != 0.f ? 1.f / p.w : 0.f;
    int sx = p.u > 0.f ? 1 : -1, sy = p.v > 0.f ? 1 : -1, sz = p.w > 0.f ? 1 : -1;
    uint32_t vox = vox_of(P, p.ix, p.iy, p.iz);
#pragma unroll 1
    for (int trip = 0; trip < kWalkTrips; ++trip) {
        const int res = walk_trip(P, p, s, iu, iv, iw, sx, sy, sz, vox, crossings, pend);
        if (res == 2 || (res == 1 && s.leg == 2)) return res;
        if (res == 1) {
            hinge<true>(p, s, pend);
            iu = p.u != 0.f ? 1.f / p.u : 0.f;
            iv = p.v != 0.f ? 1.f / p.v : 0.f;
            iw = p.w != 0.f ? 1.f / p.w : 0.f;
            sx = p.u > 0.f ? 1 : -1; sy = p.v > 0.f ? 1 : -1; sz = p.w > 0.f ? 1 : -1;
        }
    }
    return 0;
}

__device__ void electron_escape(const SimParams& P, Part& p, float energy, Acc& acc) {
    double e = energy;
    if (p.flags & kPositron) {
        if (P.S.annihilation) e += 2.0 * kMC2;
        else acc.disc += 2.0 * kMC2;
    }
    acc.esc += e;
    hist_add(P, p.hist, 0, e);
}

// One condensed-history step of an electron or positron (Sec. 2.1), or its
// absorption.  Whole-step form (RESUME false): set up, walk and end in one
// call.  Resumable form: the step is set up when none is in progress, its
// voxel walk may take several calls (several iterations of the phase loop),
// and the step's end (escape, absorption, hard-event candidate) runs in the
// call whose walk reaches it.
template <bool RESUME>
__device__ __forceinline__ void electron_step(const SimParams& P, const ElSmem& S, Part& p, bool& active,
                                              Acc& acc, Ev& ev, Sec& sec, float& pend, ElStep& carried) {
    const DevTables& T = P.T;
    // the whole-step form keeps its step state local to this call
    ElStep local;
    ElStep& st = RESUME ? carried : local;
    if (!RESUME) st.leg = 0;
    bool absorb = false;
    if (st.leg == 0) {
        absorb = p.E < T.eabs_el;
        if (!absorb) {
            const float4 r = draw(p, P.key0, P.key1);
            ev.b += EV_STEP;
            hist_count(P, p.hist, 1);
            // material and density of the start voxel, loaded together
            const uint32_t vox0 = GDPM_IDX(P.status, vox_of(P, p.ix, p.iy, p.iz), n_voxels(P), ST_B_VOXEL);
            const int m = GDPM_IDX(P.status, int(__ldg(&P.mat[vox0])), T.n_mat, ST_B_TABLE);
            st.rho = __ldg(&P.rho[vox0]);
            int i;
            float f;
            grid_pos(T, p.E, i, f);
            const int mi = m * T.n_e + i;
            const float4 a0 = S.el[mi], a1 = S.el[mi + 1];
            // step limits as mass thickness in the start material: reach E_abs,
            // hard-event candidate, or the multiple-scattering step
            const float R0 = lerpf(a0.x, a1.x, f);
            const float xms = lerpf(a0.y, a1.y, f);
            const float xcut = R0 - T.r_eabs[m];
            const float xhard = (T.flags & GDPM_FLAG_NO_HARD) ? kInf : -__logf(r.x) * T.inv_sigmax[m];
            int lim;   // what ends the step: 0 reach E_abs, 1 hard candidate, 2 MS step
            float xs;
            if (xcut <= xms && xcut <= xhard) { lim = 0; xs = xcut; }
            else if (xhard <= xms) { lim = 1; xs = xhard; }
            else { lim = 2; xs = xms; }
            xs = fmaxf(xs, 0.f);
            float Tend;
            if (lim == 0) {
                Tend = T.eabs_el;
            } else {
                const float rr = (R0 - xs - T.rinv_lo[m]) * T.rinv_idr[m];
                const int j = min(max(int(floorf(rr)), 0), T.n_r - 2);
                const float g = fminf(fmaxf(rr - float(j), 0.f), 1.f);
                const float* ri = S.rinv + m * T.n_r;
                Tend = fminf(lerpf(ri[j], ri[j + 1], g), p.E);
            }
            const float Tk = p.E;
            const float dT = Tk - Tend;
            if (P.hrec) hist_add(P, p.hist, 1, double(xs));
            // multiple scattering at the mid-step energy
            const float Tm = 0.5f * (Tk + Tend);
            const float pbc = Tm * (Tm + 2.f * kMC2f) / (Tm + kMC2f);
            const float q = kEs / pbc;
            const float G1 = xs * q * q * 0.5f * T.inv_x0[m];
            float mu;
            if (G1 >= 1.f) {
                mu = 2.f * r.z - 1.f;
            } else {
                const float Asc = screening_A(T, S.atab, G1);
                mu = 1.f - 2.f * Asc * r.z / (1.f - r.z + Asc);
            }
            float cp, sp;
            cossin_2pi(r.w, cp, sp);
            if (RESUME) {
                // the direction after the hinge: leg 1 keeps the step's start
                // direction, so the deflection is applied to it here, with all
                // lanes that start a step together
                st.u1 = p.u; st.v1 = p.v; st.w1 = p.w;
                rotate(st.u1, st.v1, st.w1, mu, cp, sp);
            } else {
                st.u1 = mu; st.v1 = cp; st.w1 = sp;
            }
            st.dpm = xs > 0.f ? dT / xs : 0.f;
            st.dep = 0.f;
            st.Tend = Tend;
            // random hinge: zeta x_s straight, deflect, (1 - zeta) x_s straight
            st.left = r.y * xs;
            st.m1 = (1.f - r.y) * xs;
            st.leg = 1;
            st.lim_m = lim | (m << 2);
        }
    }
    if (!absorb) {
        const int res = RESUME ? walk_resumable(P, p, st, ev.n, pend) : walk_whole(P, p, st, ev.n, pend);
        if (res == 0) return;            // the walk goes on in the next iteration
        st.leg = 0;
        const float Tk = p.E;
        if (res == 2) {
            electron_escape(P, p, Tk - st.dep, acc);
            ev.b += EV_TERM;
            active = false;
            return;
        }
        // the step's remainder stays owed to the voxel the step ends in
        pend += (Tk - st.Tend) - st.dep;
        p.E = st.Tend;
        const int lim = st.lim_m & 3, m = st.lim_m >> 2;
        if (lim == 0) {
            absorb = true;
        } else if (lim == 1) {
            // hard-event candidate: accept with Sigma_h(T)/Sigma_max (start material)
            const float4 v = draw(p, P.key0, P.key1);
            const float Tn = p.E, wcc = T.eabs_el, wcb = T.eabs_ph;
            float sm = 0.f, sb = 0.f;
            if (Tn > wcb || Tn > 2.f * wcc) {
                int i;
                float f;
                grid_pos(T, Tn, i, f);
                const int mj = m * T.n_e + i;
                const float4 a0 = S.el[mj], a1 = S.el[mj + 1];
                if (Tn > 2.f * wcc) sm = lerpf(a0.z, a1.z, f);
                if (Tn > wcb) sb = lerpf(a0.w, a1.w, f);
            }
            const float sh = sm + sb;
            if (v.x * T.sigmax[m] < sh) {
                hist_count(P, p.hist, 2);
                sec.n = 1;
                sec.pos2 = false;
                if (v.y * sh < sm) {
                    ev.b += EV_MOLLER;
                    float eps, rphi;
                    sample_moller(p, P, Tn, wcc, eps, rphi);
                    float c, sn;
                    cossin_2pi(rphi, c, sn);
                    const float W = eps * Tn, Tp = Tn - W;
                    const float cd = sqrtf(W * (Tn + 2.f * kMC2f) / (Tn * (W + 2.f * kMC2f)));
                    const float cpr = sqrtf(Tp * (Tn + 2.f * kMC2f) / (Tn * (Tp + 2.f * kMC2f)));
                    sec.dx = p.u; sec.dy = p.v; sec.dz = p.w;
                    rotate(sec.dx, sec.dy, sec.dz, cd, c, sn);
                    sec.photon = false;
                    sec.E1 = W;
                    rotate(p.u, p.v, p.w, cpr, -c, -sn);
                    p.E = Tp;
                } else {
                    ev.c += EV_BREMS;
                    const float k = wcb * exp2f(v.z * __log2f(Tn / wcb));
                    sec.photon = true;
                    sec.E1 = k;
                    sec.dx = p.u; sec.dy = p.v; sec.dz = p.w;
                    p.E = Tn - k;
                }
            }
        }
    }
    if (absorb) {
        // end of track: residual energy deposited here; a positron then
        // annihilates into two back-to-back 0.511 MeV photons (isotropic),
        // or its rest energy is discarded (Sec. 2.1, Sec. 4)
        tally(P, p.flags, vox_of(P, p.ix, p.iy, p.iz), p.E + pend);
        pend = 0.f;
        ev.b += EV_TERM;
        active = false;
        if (p.flags & kPositron) {
            if (!P.S.annihilation) {
                acc.disc += 2.0 * kMC2;
            } else {
                const float4 a = draw(p, P.key0, P.key1);
                const float cost = 2.f * a.x - 1.f;
                const float sint = sqrtf(fmaxf(0.f, 1.f - cost * cost));
                float cp, sp;
                cossin_2pi(a.y, cp, sp);
                ev.c += EV_ANNIHIL;
                sec.n = 2;
                sec.photon = true;
                sec.pos2 = false;
                sec.E1 = sec.E2 = kMC2f;
                sec.dx = sint * cp; sec.dy = sint * sp; sec.dz = cost;
            }
        }
    }
}

// ---------------------------------------------------------------- warp-uniform parts
// Fold the lanes' event counters into the block's (call with the whole warp).
template <int PT>
__device__ __forceinline__ void flush_events(Ev& ev, uint32_t* s_cnt) {
    const bool lead = lane_id() == 0;
    const uint32_t n = __reduce_add_sync(kFull, ev.n);
    if (lead && n) atomicAdd(&s_cnt[PT == 0 ? C_PH_FLIGHTS : C_CROSS], n);
    const uint32_t w[3] = {ev.a, ev.b, ev.c};
    const int slots[10] = {C_PH_REAL, C_COMPTON, C_PHOTO, C_PAIR,
                           PT == 0 ? C_PH_TERMINATED : C_EL_TERMINATED, C_LOCAL_DEP,
                           C_EL_STEPS, C_MOLLER, C_BREMS, C_ANNIHIL};
#pragma unroll
    for (int k = 0; k < 10; ++k) {
        const uint32_t c = __reduce_add_sync(kFull, (w[k >> 2] >> (8 * (k & 3))) & 0xFFu);
        if (lead && c) atomicAdd(&s_cnt[slots[k]], c);
    }
    ev = Ev{0u, 0u, 0u, 0u};
}

// Warp-uniform tallies of the loop top (identical in every lane), two
// 16-bit counts to a word: (local deposits, electron pushes), (photon
// pushes, primaries), (pops, primaries that miss the phantom).  At most 32
// per count and iteration, folded with the event counters.
struct WarpCnt {
    uint32_t w0, w1, w2;
};

template <int PT>
__device__ __forceinline__ void flush_warp_counts(WarpCnt& wc, uint32_t* s_cnt) {
    if (lane_id() == 0) {
        const uint32_t local = wc.w0 & 0xFFFFu, push_el = wc.w0 >> 16;
        const uint32_t push_ph = wc.w1 & 0xFFFFu, primary = wc.w1 >> 16;
        const uint32_t pop = wc.w2 & 0xFFFFu, missed = wc.w2 >> 16;
        if (local) atomicAdd(&s_cnt[C_LOCAL_DEP], local);
        if (push_el) {
            atomicAdd(&s_cnt[C_PUSH_EL], push_el);
            atomicAdd(&s_cnt[C_EL_CREATED], push_el);
        }
        if (push_ph) {
            atomicAdd(&s_cnt[C_PUSH_PH], push_ph);
            atomicAdd(&s_cnt[C_PH_CREATED], push_ph);
        }
        if (primary) {
            atomicAdd(&s_cnt[C_PRIMARY], primary);
            atomicAdd(&s_cnt[PT == 0 ? C_PH_CREATED : C_EL_CREATED], primary);
        }
        if (pop) atomicAdd(&s_cnt[PT == 0 ? C_POP_PH : C_POP_EL], pop);
        if (missed) atomicAdd(&s_cnt[PT == 0 ? C_PH_TERMINATED : C_EL_TERMINATED], missed);
    }
    wc = WarpCnt{0u, 0u, 0u};
}

// Queue slots a warp holds: [base, base + left) reserved but not yet written.
struct Slots {
    uint32_t base, left;
};

// `c` consecutive slots for the warp's pushes to one queue: from the
// reservation first, then a new reservation of max(missing, block) slots
// (one atomic).  Returns the first slot of the new reservation (or of the
// old one when it sufficed); a lane of rank r < old left writes slot
// old.base + r, the others new + (r - old left).
__device__ __forceinline__ uint32_t reserve(Slots& sl, uint32_t c, uint32_t* count, uint32_t block,
                                            int leader) {
    if (c <= sl.left) {
        const uint32_t b = sl.base;
        sl.base += c;
        sl.left -= c;
        return b;
    }
    const uint32_t miss = c - sl.left, want = max(miss, block);
    uint32_t nb = 0;
    if (int(lane_id()) == leader) nb = atomicAdd(count, want);
    nb = __shfl_sync(kFull, nb, leader);
    sl.base = nb + miss;
    sl.left = want - miss;
    return nb;
}

// Bank the secondaries the lanes' last steps created (call with the whole
// warp): below-cutoff electrons and photons deposit on the spot, the rest
// get slots in the warp's reservations and counter-derived ids.
__device__ __forceinline__ void bank_pending(const SimParams& P, const PhaseArgs& A, Part& p,
                                             const Sec& sec, Slots (&sl)[2], WarpCnt& wc) {
    const uint32_t lane = lane_id();
    for (int k = 0; k < 2; ++k) {
        const bool want = k < sec.n;
        if (!__any_sync(kFull, want)) return;
        const bool pos = k == 1 && sec.pos2;
        const float E = k ? sec.E2 : sec.E1;
        const float sg = (k == 1 && sec.photon) ? -1.f : 1.f;
        const bool push = want && (pos || E >= (sec.photon ? P.T.eabs_ph : P.T.eabs_el));
        if (want && !push) tally(P, p.flags, vox_of(P, p.ix, p.iy, p.iz), E);
        wc.w0 += __popc(__ballot_sync(kFull, want && !push));
#pragma unroll
        for (int q = 0; q < 2; ++q) {           // q = 0 electron queue, 1 photon queue
            const bool mine = push && (sec.photon == (q == 1));
            const uint32_t m = __ballot_sync(kFull, mine);
            if (!m) continue;
            const uint32_t c = __popc(m);
            const uint32_t left0 = sl[q].left, base0 = sl[q].base;
            const uint32_t nb = reserve(sl[q], c, q ? A.out_ph_count : A.out_el_count, A.bank_block,
                                        __ffs(m) - 1);
            if (mine) {
                Part ch;
                ch.x = p.x; ch.y = p.y; ch.z = p.z;
                ch.u = sg * sec.dx; ch.v = sg * sec.dy; ch.w = sg * sec.dz;
                ch.E = E;
                ch.ix = p.ix; ch.iy = p.iy; ch.iz = p.iz;
                ch.hist = p.hist;
                const uint64_t id = child_id(uint64_t(p.pidlo) | (uint64_t(p.pidhi) << 32), p.flags & kChildMask);
                // the child index cannot wrap into the slot bits (no particle
                // comes near 65535 secondaries; flag it if one ever did)
                if ((p.flags & kChildMask) == kChildMask) atomicOr(P.status, ST_QUEUE_OVERFLOW);
                ch.pidlo = uint32_t(id);
                ch.pidhi = uint32_t(id >> 32);
                ch.ctr = 0;
                ch.flags = (p.flags & kBatchMask) | (pos ? kPositron : 0u);
                ++p.flags;
                const uint32_t r = __popc(m & lanemask_lt());
                const uint32_t slot = c <= left0 ? base0 + r : (r < left0 ? base0 + r : nb + (r - left0));
                const Queue& Q = q ? A.out_ph : A.out_el;
                if (slot < Q.capacity) queue_store(Q, slot, ch);
                else atomicOr(P.status, ST_QUEUE_OVERFLOW);
                hist_count(P, p.hist, 3);
            }
            if (q) wc.w1 += c; else wc.w0 += c << 16;
        }
    }
}

// ---------------------------------------------------------------- phase kernel
__device__ __forceinline__ void copy_to_smem(void* dst, const void* src, size_t bytes) {
    const float4* s = static_cast<const float4*>(src);
    float4* d = static_cast<float4*>(dst);
    const size_t n4 = bytes / 16;
    for (size_t k = threadIdx.x; k < n4; k += blockDim.x) d[k] = __ldg(&s[k]);
    const size_t rem = bytes - n4 * 16;
    const unsigned char* sb = static_cast<const unsigned char*>(src) + n4 * 16;
    unsigned char* db = static_cast<unsigned char*>(dst) + n4 * 16;
    for (size_t k = threadIdx.x; k < rem; k += blockDim.x) db[k] = sb[k];
}

__host__ __device__ inline size_t align16(size_t b) { return (b + 15) & ~size_t(15); }

// Indices of this phase's work a warp takes at a time (primaries first,
// then queued particles): one atomic per block instead of one per refill.
// Every block boundary costs the warp a round trip to the shared counter,
// so blocks are several refills deep (128: measured best against 32, 64
// and 256); near the end of a phase the grabs turn exact.
constexpr uint32_t kGrab = 128u;

// One transport phase (Sec. 2.2.1 Step 3): a persistent loop per warp.
// Loop top (whole warp): fold event counters now and then, bank the
// secondaries of the last step, refill lanes whose particle ended.  Then
// each lane takes one step of its own particle.  PT: 0 photons, 1 electrons
// a whole step per iteration, 2 electrons with resumable steps.
template <int PT>
__device__ __forceinline__ void phase_run(const SimParams& P, const PhaseArgs& A) {
    extern __shared__ __align__(16) unsigned char smem[];
    const uint32_t n_in = A.in_count ? min(*A.in_count, A.in.capacity) : 0u;
    const uint32_t total = A.n_src + n_in;
    if (total == 0u || blockIdx.x * blockDim.x >= total) return;

    const DevTables& T = P.T;
    const size_t ne = size_t(T.n_mat) * T.n_e;
    PhSmem ps{};
    ElSmem es{};
    uint32_t* s_cnt;
    if (PT == 0) {
        float2* cum = reinterpret_cast<float2*>(smem);
        float* tot = reinterpret_cast<float*>(smem + align16(ne * 8));
        float* maj = reinterpret_cast<float*>(smem + align16(ne * 8) + align16(ne * 4));
        s_cnt = reinterpret_cast<uint32_t*>(smem + align16(ne * 8) + align16(ne * 4) +
                                            align16(size_t(T.n_e) * 4));
        copy_to_smem(cum, T.ph_cum, ne * 8);
        copy_to_smem(tot, T.ph_tot, ne * 4);
        copy_to_smem(maj, P.maj, size_t(T.n_e) * 4);
        ps.maj = maj; ps.tot = tot; ps.cum = cum;
    } else {
        float4* el = reinterpret_cast<float4*>(smem);
        float* rinv = reinterpret_cast<float*>(smem + ne * 16);
        const size_t nr = size_t(T.n_mat) * T.n_r;
        float* atab = reinterpret_cast<float*>(smem + ne * 16 + align16(nr * 4));
        s_cnt = reinterpret_cast<uint32_t*>(smem + ne * 16 + align16(nr * 4) +
                                            align16(size_t(T.n_a) * 4));
        copy_to_smem(el, T.el, ne * 16);
        copy_to_smem(rinv, T.rinv, nr * 4);
        copy_to_smem(atab, T.atab, size_t(T.n_a) * 4);
        es.el = el; es.rinv = rinv; es.atab = atab;
    }
    for (int k = threadIdx.x; k < C_NCOUNT; k += blockDim.x) s_cnt[k] = 0u;
    __syncthreads();

    Acc acc{0.0, 0.0, 0.0};
    Part p{};
    Sec sec{};
    Ev ev{0u, 0u, 0u, 0u};
    WarpCnt wc{0u, 0u, 0u};
    Slots sl[2] = {{0u, 0u}, {0u, 0u}};
    bool active = false, exhausted = false;
    float pend = 0.f;   // electron energy owed to its current voxel (see walk)
    ElStep est{};       // electron step in progress (leg 0: none)
    // the warp's block of work indices [st_base, st_base + st_left); near
    // the end of the phase (less than two per lane of the grid left) the
    // warp takes exactly what it needs, so no warp sits on spare work
    uint32_t st_base = 0u, st_left = 0u;
    bool st_exact = false;
    const uint32_t lane = lane_id();
    for (uint32_t it = 0;; ++it) {
        // ---- whole warp: account and bank the last step, then refill
        if ((it % kFlushEvery) == kFlushEvery - 1u) {
            flush_events<PT>(ev, s_cnt);
            flush_warp_counts<PT>(wc, s_cnt);
        }
        bank_pending(P, A, p, sec, sl, wc);
        sec.n = 0;
        const bool need = !active && !exhausted;
        const uint32_t nm = __ballot_sync(kFull, need);
        if (nm) {
            const uint32_t k = __popc(nm);
            const uint32_t left0 = st_left, base0 = st_base;
            uint32_t nb = 0u;
            if (k > st_left) {
                const uint32_t miss = k - st_left, want = st_exact ? miss : max(miss, kGrab);
                if (lane == 0) nb = atomicAdd(A.head, want);
                nb = __shfl_sync(kFull, nb, 0);
                st_base = nb + miss;
                st_left = want - miss;
                if (nb >= total || total - nb < 2u * gridDim.x * blockDim.x) st_exact = true;
            } else {
                st_base += k;
                st_left -= k;
            }
            bool from_queue = false;
            if (need) {
                const uint32_t r = __popc(nm & lanemask_lt());
                const uint32_t idx = r < left0 ? base0 + r : nb + (r - left0);
                if (idx < A.n_src) {
                    // made by k_sources; a primary that missed the phantom
                    // left its slot empty (E < 0) and is accounted there
                    source_load(A.src, GDPM_IDX(P.status, idx, A.src.capacity, ST_B_QUEUE), p);
                    active = p.E >= 0.f;
                    if (active) {
                        p.hist = A.src_first + idx;
                        p.pidlo = 1u;
                        p.pidhi = 0u;
                        voxel_of(P, p);
                    }
                } else if (idx < total) {
                    queue_load(A.in, GDPM_IDX(P.status, idx - A.n_src, A.in.capacity, ST_B_QUEUE), p);
                    // a slot reserved but never written holds E < 0
                    from_queue = p.E >= 0.f;
                    active = from_queue;
                } else {
                    exhausted = true;
                }
            }
            wc.w2 += __popc(__ballot_sync(kFull, from_queue));
        }
        if (__all_sync(kFull, exhausted)) break;
        if (it >= P.max_iters) {
            if (lane == 0) atomicOr(P.status, ST_ITER_CAP);
            break;
        }
        // ---- each lane on its own: one step
        if (active) {
            if (PT == 0) photon_step(P, ps, p, active, acc, ev, sec);
            else electron_step<PT == 2>(P, es, p, active, acc, ev, sec, pend, est);
        }
    }
    // only a phase stopped by its iteration cap leaves a track unfinished
    if (PT != 0 && pend != 0.f) tally(P, p.flags, vox_of(P, p.ix, p.iy, p.iz), pend);
    flush_events<PT>(ev, s_cnt);
    flush_warp_counts<PT>(wc, s_cnt);
    // reserved queue slots never written: mark them empty for the consumer
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        const Queue& Q = q ? A.out_ph : A.out_el;
        const uint32_t slot = sl[q].base + lane;
        if (lane < sl[q].left && slot < Q.capacity) Q.E[slot] = -1.f;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        acc.src += __shfl_down_sync(kFull, acc.src, o);
        acc.esc += __shfl_down_sync(kFull, acc.esc, o);
        acc.disc += __shfl_down_sync(kFull, acc.disc, o);
    }
    if (lane == 0) {
        if (acc.src != 0.0) atomicAdd(&P.ledger[L_SOURCE], acc.src);
        if (acc.esc != 0.0) atomicAdd(&P.ledger[L_ESCAPED], acc.esc);
        if (acc.disc != 0.0) atomicAdd(&P.ledger[L_DISCARDED], acc.disc);
    }
    __syncthreads();
    for (int k = threadIdx.x; k < C_NCOUNT; k += blockDim.x)
        if (s_cnt[k]) atomicAdd(&P.counters[k], (unsigned long long)s_cnt[k]);
}

template <int PT>
__global__ void __launch_bounds__(PhaseShape<PT>::threads, PhaseShape<PT>::ctas)
k_phase(const SimParams P, const PhaseArgs A) {
    phase_run<PT>(P, A);
}


// ---------------------------------------------------------------- sources
// The primaries of one source phase (Sec. 2.3), made with every lane busy
// before the phase runs: primary idx goes to slot idx of A.src.  One that
// misses the phantom leaves its slot empty (E < 0) and is accounted here:
// source and escaped energy, a created and a terminated particle.
// The spectrum prefix counts of the batches and the cumulative beamlet
// weights are searched for every primary: a CTA copies them to shared
// memory when they fit (n_prefix, n_cdf of them; see sources_smem).
template <int PT>
__device__ __forceinline__ void make_sources(const SimParams& P, const PhaseArgs& A, uint32_t n_prefix,
                                             uint32_t n_cdf) {
    extern __shared__ __align__(16) unsigned char smem[];
    float* s_cdf = reinterpret_cast<float*>(smem);
    uint32_t* s_prefix = reinterpret_cast<uint32_t*>(smem + size_t(n_cdf) * 4);
    for (uint32_t i = threadIdx.x; i < n_cdf; i += blockDim.x) s_cdf[i] = P.S.bl_cdf[i];
    for (uint32_t i = threadIdx.x; i < n_prefix; i += blockDim.x) s_prefix[i] = A.bin_prefix[i];
    __syncthreads();
    const uint32_t* ptab = n_prefix ? s_prefix : nullptr;
    const float* ctab = n_cdf ? s_cdf : nullptr;
    Acc acc{0.0, 0.0, 0.0};
    uint32_t made = 0u, missed = 0u;
    for (uint32_t idx = blockIdx.x * blockDim.x + threadIdx.x; idx < A.n_src;
         idx += gridDim.x * blockDim.x) {
        Part p{};
        if (make_primary(P, A, idx, p, acc, ptab, ctab)) {
            source_store(A.src, GDPM_IDX(P.status, idx, A.src.capacity, ST_B_QUEUE), p);
        } else {
            A.src.E[GDPM_IDX(P.status, idx, A.src.capacity, ST_B_QUEUE)] = -1.f;
            ++missed;
        }
        ++made;
    }
    made = __reduce_add_sync(kFull, made);
    missed = __reduce_add_sync(kFull, missed);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        acc.src += __shfl_down_sync(kFull, acc.src, o);
        acc.esc += __shfl_down_sync(kFull, acc.esc, o);
    }
    if (lane_id() == 0) {
        if (acc.src != 0.0) atomicAdd(&P.ledger[L_SOURCE], acc.src);
        if (acc.esc != 0.0) atomicAdd(&P.ledger[L_ESCAPED], acc.esc);
        if (made) {
            atomicAdd(&P.counters[C_PRIMARY], (unsigned long long)made);
            atomicAdd(&P.counters[PT == 0 ? C_PH_CREATED : C_EL_CREATED], (unsigned long long)made);
        }
        if (missed) atomicAdd(&P.counters[PT == 0 ? C_PH_TERMINATED : C_EL_TERMINATED], (unsigned long long)missed);
    }
}

template <int PT>
__global__ void __launch_bounds__(256) k_sources(const SimParams P, const PhaseArgs A, uint32_t n_prefix,
                                                 uint32_t n_cdf) {
    make_sources<PT>(P, A, n_prefix, n_cdf);
}

// Cumulative-weight entries the sources search (the cumulative sampler of a
// sampled fluence map; none otherwise).
inline uint32_t cdf_entries(const SimParams& P, const PhaseArgs& A) {
    return (P.S.geometry == GDPM_GEO_BEAMLETS && P.S.sampler == GDPM_SAMPLE_CDF && A.n_sub == 0)
               ? uint32_t(P.S.n_beamlets) : 0u;
}

// Entries of the prefix and cumulative-weight tables a source CTA stages in
// shared memory (0: read from global memory), within a 40 KB budget.
__host__ __device__ inline void sources_smem(uint32_t prefix_entries, uint32_t cdf_entries,
                                             uint32_t& n_prefix, uint32_t& n_cdf) {
    const size_t budget = 40u << 10;
    n_cdf = size_t(cdf_entries) * 4 <= budget ? cdf_entries : 0u;
    n_prefix = size_t(n_cdf) * 4 + size_t(prefix_entries) * 4 <= budget ? prefix_entries : 0u;
}

// ---------------------------------------------------------------- device-driven phase loop
// Phase k's arguments from k alone, as the host loop sets them: photon
// phase k (even) reads photons P[k] and banks electrons into E[k+1];
// electron phase k (odd) reads E[k] and banks photons into P[k+1] and
// electrons into E[k+2].  Row k of ctl holds (pop head, P[k] count, E[k]
// count, -).  The source particle's j-th phase takes primaries
// [first + j*chunk, first + min((j+1)*chunk, n_src)).
__device__ __forceinline__ PhaseArgs phase_args(const LoopArgs& L, uint32_t k) {
    PhaseArgs A{};
    A.nb_small = L.nb_small;
    A.nb_rem = L.nb_rem;
    A.bin_prefix = L.bin_prefix;
    A.prefix_n = L.prefix_n;
    A.n_sub = L.n_sub;
    A.sub_batches = L.sub_batches;
    A.sub_first = L.sub_first;
    A.bank_block = L.bank_block;
    A.src = L.qsrc;
    const bool ph = (k % 2u) == 0u;
    const bool src_phase = ph == (L.src_particle == GDPM_PHOTON);
    if (src_phase) {
        const uint32_t j = L.src_particle == GDPM_PHOTON ? k / 2u : (k - 1u) / 2u;
        const uint64_t off = uint64_t(j) * L.chunk;
        if (off < L.n_src) {
            A.n_src = uint32_t(min(uint64_t(L.chunk), uint64_t(L.n_src) - off));
            A.src_first = L.first + uint32_t(off);
            A.bl_pick = L.pick;
        }
    }
    uint32_t* ctl = L.ctl;
    A.head = ctl + size_t(k) * 4;
    if (ph) {
        A.in = L.qph;
        A.in_count = k >= 1u ? ctl + size_t(k) * 4 + 1 : nullptr;
        A.out_el = ((k + 1u) / 2u) % 2u ? L.qe1 : L.qe0;
        A.out_el_count = ctl + size_t(k + 1) * 4 + 2;
        A.out_ph = L.qph;
        A.out_ph_count = ctl + size_t(k + 2) * 4 + 1;
    } else {
        A.in = (k / 2u) % 2u ? L.qe1 : L.qe0;
        A.in_count = ctl + size_t(k) * 4 + 2;
        A.out_ph = L.qph;
        A.out_ph_count = ctl + size_t(k + 1) * 4 + 1;
        A.out_el = ((k + 2u) / 2u) % 2u ? L.qe1 : L.qe0;
        A.out_el_count = ctl + size_t(k + 2) * 4 + 2;
    }
    return A;
}

// One pass of the device-driven loop runs photon phase k and electron
// phase k+1, k = *L.k (even); PT selects which of the two this launch is
// (0 the photon phase; 1 or 2 the electron phase in its whole-step or
// resumable form).
// The phase's arguments are derived in shared memory from k.  (A kernel of
// its own: the host loop's k_phase takes them as kernel parameters, which
// keeps more registers for the transport loop.)
template <int PT>
__global__ void __launch_bounds__(PhaseShape<PT>::threads, PhaseShape<PT>::ctas)
k_phase_loop(const SimParams P, const LoopArgs L) {
    __shared__ PhaseArgs sA;
    if (threadIdx.x == 0) sA = phase_args(L, *L.k + (PT == 0 ? 0u : 1u));
    __syncthreads();
    phase_run<PT>(P, sA);
}

// Primaries of this pass's source phase (before it runs).
template <int PT>
__global__ void __launch_bounds__(256) k_sources_loop(const SimParams P, const LoopArgs L, uint32_t n_prefix,
                                                      uint32_t n_cdf) {
    const PhaseArgs A = phase_args(L, *L.k + uint32_t(PT));
    if (A.n_src) make_sources<PT>(P, A, n_prefix, n_cdf);
}

// Metropolis picks for this pass's source phase (before it runs).
__global__ void k_metropolis_loop(const SimParams P, const LoopArgs L) {
    const uint32_t k = *L.k + (L.src_particle == GDPM_PHOTON ? 0u : 1u);
    const PhaseArgs A = phase_args(L, k);
    const uint32_t c = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t C = P.S.n_chains;
    if (A.n_src == 0u || c >= C) return;
    const uint32_t nf = uint32_t(P.S.n_beamlets);
    const double* f = P.S.bl_f;
    uint32_t I = L.chains[c];
    double fI = f[I];
    const uint64_t end = uint64_t(A.src_first) + A.n_src;
    for (uint64_t h = uint64_t(A.src_first) + (uint64_t(c) + C - A.src_first % C) % C; h < end; h += C) {
        const uint4 w = philox_block(uint32_t(h), 0u, 0u, 0u, P.key0, P.key1);
        const uint32_t J = __umulhi(w.x, nf);
        const double fJ = f[J];
        const double u = (double(w.y) + 0.5) * 0x1p-32;
        if (u * fI < fJ) {
            I = J;
            fI = fJ;
        }
        L.pick[h - A.src_first] = I;
    }
    L.chains[c] = I;
}

// After a pass: go on while primaries remain or the pass left particles for
// the next one (photons P[k+2], electrons E[k+3]); stop at the phase cap
// with a status bit.  One thread.
__global__ void k_loop_ctl(const LoopArgs L, cudaGraphConditionalHandle h) {
    const uint32_t k = *L.k, k2 = k + 2u;
    const uint32_t j_next = k2 / 2u;        // index of the next pass's source phase
    const bool src_left = uint64_t(j_next) * L.chunk < uint64_t(L.n_src);
    const uint32_t pending = L.ctl[size_t(k2) * 4 + 1] + L.ctl[size_t(k2 + 1) * 4 + 2];
    bool more = src_left || pending > 0u;
    if (more && int(k2) + 3 >= L.max_phases) {
        atomicOr(L.status, ST_PHASE_CAP);
        more = false;
    }
    *L.k = k2;
    cudaGraphSetConditional(h, more ? 1u : 0u);
}

// ---------------------------------------------------------------- checks
__global__ void k_debug_philox(const uint32_t* ctr, uint32_t k0, uint32_t k1, uint32_t* out,
                               uint64_t n) {
    for (uint64_t s = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; s < n;
         s += uint64_t(gridDim.x) * blockDim.x) {
        const uint4 c = make_uint4(ctr[4 * s], ctr[4 * s + 1], ctr[4 * s + 2], ctr[4 * s + 3]);
        const uint4 o = philox4x32_10(c, k0, k1);
        out[4 * s] = o.x; out[4 * s + 1] = o.y; out[4 * s + 2] = o.z; out[4 * s + 3] = o.w;
    }
}

__global__ void k_debug_sample(int kind, float a, float b, uint64_t n, uint32_t k0, uint32_t k1,
                               double* out1, double* out2) {
    SimParams P{};
    P.key0 = k0;
    P.key1 = k1;
    for (uint64_t s = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; s < n;
         s += uint64_t(gridDim.x) * blockDim.x) {
        Part p{};
        p.hist = uint32_t(s);
        p.pidlo = 1u;
        double o1 = 0, o2 = 0;
        if (kind == 0) {
            float eps, cost, rphi;
            sample_kn(p, P, a, eps, cost, rphi);
            o1 = eps; o2 = cost;
        } else if (kind == 1) {
            float eps, rphi;
            sample_moller(p, P, a, b, eps, rphi);
            const float W = eps * a;
            o1 = eps;
            o2 = sqrtf(W * (a + 2.f * kMC2f) / (a * (W + 2.f * kMC2f)));
        } else if (kind == 2) {
            const float4 v = draw(p, k0, k1);
            o1 = b * exp2f(v.z * __log2f(a / b));
        } else if (kind == 3) {
            const float4 r = draw(p, k0, k1);
            o1 = 1.f - 2.f * a * r.z / (1.f - r.z + a);
        } else if (kind == 5) {
            float mu, rphi;
            sample_sauter(p, P, a, mu, rphi);
            o1 = mu;
            o2 = kTwoPi * rphi;
        } else {
            const float4 r = draw(p, k0, k1);
            o1 = 2.f * r.x - 1.f;
            o2 = kTwoPi * r.y;
        }
        out1[s] = o1;
        if (out2) out2[s] = o2;
    }
}

// Metropolis chains of Algorithm A1, one thread per chain c.  Chain c starts
// at a uniform beamlet from the Philox block at (c, 0, 1, 0).
__global__ void k_metropolis_init(const SimParams P, uint32_t* chains) {
    const uint32_t c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= P.S.n_chains) return;
    const uint4 w = philox_block(c, 0u, 1u, 0u, P.key0, P.key1);
    chains[c] = __umulhi(w.x, uint32_t(P.S.n_beamlets));
}

// Advance every chain through the histories of [first, first+n) that belong
// to it (h = c, c + C, c + 2C, ...), in order: propose J uniform, accept
// when u f_I < f_J (u < f_J / f_I without the division), record the state
// as the beamlet of history h.
__global__ void k_metropolis(const SimParams P, uint32_t first, uint32_t n, uint32_t* chains,
                             uint32_t* pick) {
    const uint32_t c = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t C = P.S.n_chains;
    if (c >= C) return;
    const uint32_t nf = uint32_t(P.S.n_beamlets);
    const double* f = P.S.bl_f;
    uint32_t I = chains[c];
    double fI = f[I];
    const uint64_t end = uint64_t(first) + n;
    for (uint64_t h = uint64_t(first) + (uint64_t(c) + C - first % C) % C; h < end; h += C) {
        const uint4 w = philox_block(uint32_t(h), 0u, 0u, 0u, P.key0, P.key1);
        const uint32_t J = __umulhi(w.x, nf);
        const double fJ = f[J];
        const double u = (double(w.y) + 0.5) * 0x1p-32;
        if (u * fI < fJ) {
            I = J;
            fI = fJ;
        }
        pick[h - first] = I;
    }
    chains[c] = I;
}

// Beamlet rows of histories [first, first+n) (checks of the samplers).
__global__ void k_debug_beamlets(const SimParams P, uint32_t first, uint32_t n,
                                 const uint32_t* pick, int32_t* out) {
    for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
        Part p{};
        p.hist = first + s;
        p.pidlo = 1u;
        const float4 r = draw(p, P.key0, P.key1);
        PhaseArgs A{};
        A.bl_pick = pick;
        out[s] = P.S.bl_row[pick_beamlet(P.S, A, s, first + s, r.w, P.key0, P.key1, P.S.bl_cdf)];
    }
}

__global__ void k_debug_sources(const SimParams P, const PhaseArgs A, uint64_t n, double* out) {
    for (uint64_t s = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; s < n;
         s += uint64_t(gridDim.x) * blockDim.x) {
        Part p{};
        Acc acc{0, 0, 0};
        const bool in = make_primary(P, A, uint32_t(s), p, acc);
        double* o = out + 8 * s;
        o[0] = p.x; o[1] = p.y; o[2] = p.z; o[3] = p.u; o[4] = p.v; o[5] = p.w; o[6] = p.E;
        o[7] = in ? 1.0 : 0.0;
    }
}

}  // namespace

static size_t smem_of(const DevTables& T, int particle) {
    const size_t ne = size_t(T.n_mat) * T.n_e;
    const size_t cnt = align16(C_NCOUNT * 4);
    if (particle == GDPM_PHOTON)
        return align16(ne * 8) + align16(ne * 4) + align16(size_t(T.n_e) * 4) + cnt;
    return ne * 16 + align16(size_t(T.n_mat) * T.n_r * 4) + align16(size_t(T.n_a) * 4) + cnt;
}

int transport_smem(const gdpm_tables* t, int particle) { return int(smem_of(t->dev, particle)); }

// Persistent grid: SM count x resident CTAs per SM for this shared-memory size.
// share_eighths < 8 gives the grid that many eighths of the GPU: a large
// request that runs while small ones are active leaves SMs free for them,
// since persistent CTAs do not yield until their phase's input is drained.
int launch_phase(gdpm_ctx* ctx, cudaStream_t st, int particle, const SimParams& P,
                 const PhaseArgs& A, uint32_t n_items_hint, uint32_t share_eighths) {
    const size_t smem = smem_of(P.T, particle);
    const bool resumable = particle != GDPM_PHOTON && P.walk_resumable;
    const int thr = phase_threads(ctx, particle == GDPM_PHOTON ? 0 : resumable ? 2 : 1);
    const void* fn = particle == GDPM_PHOTON ? (const void*)k_phase<0>
                     : resumable              ? (const void*)k_phase<2>
                                              : (const void*)k_phase<1>;
    GDPM_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
    int bps = ctx->blocks_per_sm;
    if (bps <= 0) {
        GDPM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, fn, thr, smem));
        if (bps < 1) return GDPM_E_ARG;
    }
    uint32_t grid = uint32_t(ctx->sm_count) * uint32_t(bps);
    if (share_eighths < 8) grid = std::max<uint32_t>(uint32_t(ctx->sm_count), grid * share_eighths / 8);
    if (n_items_hint > 0) {
        const uint32_t need = (n_items_hint + thr - 1) / thr;
        grid = need < grid ? need : grid;
    }
    if (grid == 0) grid = 1;
    // queue slots a warp reserves at a time: up to 32, while all warps'
    // spare slots stay below an eighth of the queue; exact below 8
    PhaseArgs B = A;
    const uint64_t warps = uint64_t(grid) * uint64_t(thr / 32);
    const uint64_t cap = std::min(A.out_el.capacity, A.out_ph.capacity);
    const uint64_t bb = std::min<uint64_t>(32u, cap / (8u * warps));
    B.bank_block = bb >= 8u ? uint32_t(bb) : 0u;
    if (particle == GDPM_PHOTON)
        k_phase<0><<<grid, thr, smem, st>>>(P, B);
    else if (resumable)
        k_phase<2><<<grid, thr, smem, st>>>(P, B);
    else
        k_phase<1><<<grid, thr, smem, st>>>(P, B);
    GDPM_CUDA_TRY(cudaGetLastError());
    return GDPM_OK;
}

int launch_debug_philox(gdpm_ctx* ctx, const uint32_t* ctr, uint32_t k0, uint32_t k1,
                        uint32_t* out, uint64_t n) {
    const uint32_t grid = uint32_t(ctx->sm_count) * 4u;
    k_debug_philox<<<grid, 256, 0, ctx->stream>>>(ctr, k0, k1, out, n);
    GDPM_CUDA_TRY(cudaGetLastError());
    return GDPM_OK;
}

int launch_debug_sample(gdpm_ctx* ctx, int kind, double a, double b, uint64_t n, uint64_t seed,
                        double* out1, double* out2) {
    const uint32_t grid = uint32_t(ctx->sm_count) * 4u;
    k_debug_sample<<<grid, 256, 0, ctx->stream>>>(kind, float(a), float(b), n, uint32_t(seed),
                                                   uint32_t(seed >> 32), out1, out2);
    GDPM_CUDA_TRY(cudaGetLastError());
    return GDPM_OK;
}

int launch_debug_sources(gdpm_ctx* ctx, const SimParams& P, const PhaseArgs& A, uint64_t n,
                         double* out) {
    const uint32_t grid = uint32_t(ctx->sm_count) * 2u;
    k_debug_sources<<<grid, 256, 0, ctx->stream>>>(P, A, n, out);
    GDPM_CUDA_TRY(cudaGetLastError());
    return GDPM_OK;
}

// The device-driven phase loop: a graph holding one conditional WHILE node
// whose body runs [Metropolis picks ->] photon phase -> electron phase ->
// control kernel; the control kernel advances the phase index and ends the
// loop when nothing is left (or at the phase cap).  The phase kernels use
// the persistent grids of launch_phase; L.bank_block is set here.
int build_loop_graph(gdpm_ctx* ctx, const SimParams& P, LoopArgs& L, bool metropolis,
                     cudaGraph_t* graph, cudaGraphExec_t* exec) {
    *graph = nullptr;
    *exec = nullptr;
    uint32_t grid[2];
    size_t smem[2];
    const void* fn[2] = {(const void*)k_phase_loop<0>,
                         P.walk_resumable ? (const void*)k_phase_loop<2>
                                          : (const void*)k_phase_loop<1>};
    const int thr[2] = {phase_threads(ctx, 0), phase_threads(ctx, P.walk_resumable ? 2 : 1)};
    uint64_t warps = 0;
    for (int t = 0; t < 2; ++t) {
        smem[t] = smem_of(P.T, t == 0 ? GDPM_PHOTON : GDPM_ELECTRON);
        GDPM_CUDA_TRY(cudaFuncSetAttribute(fn[t], cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem[t])));
        int bps = ctx->blocks_per_sm;
        if (bps <= 0) {
            GDPM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, fn[t], thr[t], smem[t]));
            if (bps < 1) return GDPM_E_ARG;
        }
        grid[t] = uint32_t(ctx->sm_count) * uint32_t(bps);
        warps = std::max<uint64_t>(warps, uint64_t(grid[t]) * uint64_t(thr[t] / 32));
    }
    const uint64_t cap = std::min(L.qph.capacity, L.qe0.capacity);
    const uint64_t bb = std::min<uint64_t>(32u, cap / (8u * warps));
    L.bank_block = bb >= 8u ? uint32_t(bb) : 0u;

    cudaGraph_t g = nullptr;
    GDPM_CUDA_TRY(cudaGraphCreate(&g, 0));
    cudaGraphConditionalHandle h;
    cudaError_t e = cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault);
    cudaGraphNodeParams cp{};
    cudaGraphNode_t wn = nullptr;
    if (e == cudaSuccess) {
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = h;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        e = cudaGraphAddNode(&wn, g, nullptr, nullptr, 0, &cp);
    }
    cudaGraph_t body = e == cudaSuccess ? cp.conditional.phGraph_out[0] : nullptr;
    SimParams Pc = P;
    LoopArgs Lc = L;
    void* phase_args_v[2] = {&Pc, &Lc};
    void* metro_args_v[2] = {&Pc, &Lc};
    uint32_t np, nc;
    {
        PhaseArgs probe{};
        probe.n_sub = L.n_sub;
        sources_smem(L.prefix_n, cdf_entries(P, probe), np, nc);
    }
    const size_t src_sm = size_t(nc) * 4 + size_t(np) * 4;
    void* src_args_v[4] = {&Pc, &Lc, &np, &nc};
    void* ctl_args_v[2] = {&Lc, &h};
    cudaGraphNode_t prev = nullptr;
    auto add = [&](const void* f, dim3 gd, dim3 bd, size_t sm, void** args) {
        if (e != cudaSuccess) return;
        cudaKernelNodeParams kp{};
        kp.func = const_cast<void*>(f);
        kp.gridDim = gd;
        kp.blockDim = bd;
        kp.sharedMemBytes = unsigned(sm);
        kp.kernelParams = args;
        cudaGraphNode_t n = nullptr;
        e = cudaGraphAddKernelNode(&n, body, prev ? &prev : nullptr, prev ? 1 : 0, &kp);
        prev = n;
    };
    if (metropolis)
        add((const void*)k_metropolis_loop, dim3((P.S.n_chains + 127) / 128), dim3(128), 0, metro_args_v);
    {
        const uint32_t sg = std::max(1u, std::min((L.chunk + 255u) / 256u, uint32_t(ctx->sm_count) * 8u));
        const void* sf = L.src_particle == GDPM_PHOTON ? (const void*)k_sources_loop<0> : (const void*)k_sources_loop<1>;
        if (e == cudaSuccess) e = cudaFuncSetAttribute(sf, cudaFuncAttributeMaxDynamicSharedMemorySize, int(src_sm));
        add(sf, dim3(sg), dim3(256), src_sm, src_args_v);
    }
    add(fn[0], dim3(grid[0]), dim3(thr[0]), smem[0], phase_args_v);
    add(fn[1], dim3(grid[1]), dim3(thr[1]), smem[1], phase_args_v);
    add((const void*)k_loop_ctl, dim3(1), dim3(1), 0, ctl_args_v);
    cudaGraphExec_t x = nullptr;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&x, g, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        last_cuda_error() = e;
        cudaGetLastError();
        return GDPM_E_CUDA;
    }
    *graph = g;
    *exec = x;
    return GDPM_OK;
}

int launch_sources(gdpm_ctx* ctx, cudaStream_t st, const SimParams& P, const PhaseArgs& A) {
    const uint32_t grid = std::max(1u, std::min((A.n_src + 255u) / 256u, uint32_t(ctx->sm_count) * 8u));
    uint32_t np, nc;
    sources_smem(A.prefix_n, cdf_entries(P, A), np, nc);
    const size_t sm = size_t(nc) * 4 + size_t(np) * 4;
    if (P.S.particle == GDPM_PHOTON) {
        GDPM_CUDA_TRY(cudaFuncSetAttribute(k_sources<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm)));
        k_sources<0><<<grid, 256, sm, st>>>(P, A, np, nc);
    } else {
        GDPM_CUDA_TRY(cudaFuncSetAttribute(k_sources<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm)));
        k_sources<1><<<grid, 256, sm, st>>>(P, A, np, nc);
    }
    GDPM_CUDA_TRY(cudaGetLastError());
    return GDPM_OK;
}

int launch_metropolis_init(cudaStream_t st, const SimParams& P, uint32_t* chains) {
    k_metropolis_init<<<(P.S.n_chains + 255) / 256, 256, 0, st>>>(P, chains);
    GDPM_CUDA_TRY(cudaGetLastError());
    return GDPM_OK;
}

int launch_metropolis(cudaStream_t st, const SimParams& P, uint32_t first, uint32_t n,
                      uint32_t* chains, uint32_t* pick) {
    // a chain's steps are sequential: one thread per chain, 128 per block to
    // spread a few thousand chains over all SMs
    k_metropolis<<<(P.S.n_chains + 127) / 128, 128, 0, st>>>(P, first, n, chains, pick);
    GDPM_CUDA_TRY(cudaGetLastError());
    return GDPM_OK;
}

int launch_debug_beamlets(cudaStream_t st, const SimParams& P, uint32_t first, uint32_t n,
                          const uint32_t* pick, int32_t* out) {
    const uint32_t grid = std::max(1u, std::min(1024u, (n + 255) / 256));
    k_debug_beamlets<<<grid, 256, 0, st>>>(P, first, n, pick, out);
    GDPM_CUDA_TRY(cudaGetLastError());
    return GDPM_OK;
}

}  // namespace gdpm
