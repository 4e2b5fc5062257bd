// Device-side building blocks of the GB300 gDPM engine: random numbers,
// geometry helpers and the data layouts shared by the transport kernels.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "gdpm.h"

namespace gdpm {

constexpr int kMaxMat = GDPM_MAX_MATERIALS;
constexpr int kMaxBins = GDPM_MAX_BINS;
constexpr double kMC2 = 0.51099895;           // electron rest energy, MeV
constexpr float kMC2f = 0.51099895f;
constexpr float kTwoPi = 6.28318530717958647f;

// ---------------------------------------------------------------- status bits
enum : uint32_t {
    ST_QUEUE_OVERFLOW = 1u,
    ST_ITER_CAP = 2u,
    ST_PHASE_CAP = 4u,          // the device-driven phase loop reached its phase cap
    ST_BOUNDS = 8u,             // checked build: an index was out of range (class below)
    ST_B_VOXEL = 1u << 8,       //   phantom voxel
    ST_B_TALLY = 1u << 9,       //   tally cell
    ST_B_TABLE = 1u << 10,      //   material / beamlet table row
    ST_B_QUEUE = 1u << 11,      //   queue slot
    ST_B_RECORD = 1u << 12,     //   per-history record
};

// Checked build (compiled with GDPM_CHECKED=1): an index is tested against
// its range before use.  One out of range sets ST_BOUNDS and its class bit
// and is replaced by 0, so the access stays in bounds and the call returns
// GDPM_E_BOUNDS.  In the normal build the check and its range expression
// vanish.
#ifndef GDPM_CHECKED
#define GDPM_CHECKED 0
#endif
#if GDPM_CHECKED
__device__ __noinline__ inline void bounds_fail(uint32_t* status, uint32_t cls) {
    atomicOr(status, ST_BOUNDS | cls);
}
#define GDPM_IDX(status, i, n, cls) ((i) < (n) ? (i) : (bounds_fail((status), (cls)), decltype(i)(0)))
#else
#define GDPM_IDX(status, i, n, cls) (i)
#endif

// ---------------------------------------------------------------- counters
// Slots of the device counter array (uint64).  Names follow gdpm_stats.
enum {
    C_PRIMARY = 0, C_PH_CREATED, C_PH_TERMINATED, C_PH_FLIGHTS, C_PH_REAL, C_COMPTON,
    C_PHOTO, C_PAIR, C_EL_CREATED, C_EL_TERMINATED, C_EL_STEPS, C_MOLLER, C_BREMS,
    C_ANNIHIL, C_LOCAL_DEP, C_PUSH_PH, C_PUSH_EL, C_POP_PH, C_POP_EL, C_CROSS, C_NCOUNT
};
// Slots of the device FP64 ledger.
enum { L_SOURCE = 0, L_DEPOSITED, L_ESCAPED, L_DISCARDED, L_DMAX, L_SIGSUM, L_SIGCNT, L_NLEDGER };

// ---------------------------------------------------------------- Philox4x32-10
// Salmon et al., SC'11: ten rounds; each round multiplies words 0 and 2 by
// fixed 32-bit constants (64-bit products), mixes the halves with words 1
// and 3 and the round key, and bumps the key by two Weyl constants.
__host__ __device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
#ifdef __CUDA_ARCH__
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
#else
        const uint64_t p0 = uint64_t(0xD2511F53u) * c.x, p1 = uint64_t(0xCD9E8D57u) * c.z;
        const uint32_t hi0 = uint32_t(p0 >> 32), lo0 = uint32_t(p0);
        const uint32_t hi1 = uint32_t(p1 >> 32), lo1 = uint32_t(p1);
#endif
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// 23-bit uniform in the open interval (0,1): (floor(x/2^9) + 1/2) / 2^23 is
// exactly representable in FP32, so it never rounds to 0 or 1.
__device__ __forceinline__ float u01(uint32_t x) {
    return (float(x >> 9) + 0.5f) * 1.1920928955078125e-07f;
}

// Id of the k-th banked secondary: the SplitMix64 output function
// (Steele, Lea, Flood 2014) applied to parent ^ (k+1)*golden.
__host__ __device__ __forceinline__ uint64_t child_id(uint64_t parent, uint32_t k) {
    const uint64_t golden = 0x9E3779B97F4A7C15ull;
    uint64_t z = (parent ^ (uint64_t(k + 1) * golden)) + golden;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// ---------------------------------------------------------------- particle state
// Register copy of one particle (flags as above).
struct Part {
    float x, y, z, u, v, w, E;
    int ix, iy, iz;
    uint32_t hist, pidlo, pidhi, ctr, flags;
};
constexpr uint32_t kPositron = 0x80000000u;
// flags: bits 0..15 count the secondaries a particle has banked (the child
// index of the next one), bits 16..30 its tally slot (the batch of its
// history when batches run side by side; beamlet x batch in a dose-matrix
// run), bit 31 marks a positron.
constexpr uint32_t kChildMask = 0xFFFFu;
constexpr uint32_t kBatchShift = 16, kBatchMask = 0x7FFF0000u;
constexpr int kMaxConcurrentBatches = 128;
constexpr int kMaxSlots = 32767;

// One Philox block for the transport kernels.  Out of line (it has no
// warp-synchronous operations), so its ten unrolled rounds exist once in
// the kernel instead of at every draw site.
#ifndef GDPM_PHILOX_ATTR
#define GDPM_PHILOX_ATTR __noinline__
#endif
static __device__ GDPM_PHILOX_ATTR uint4 philox_block(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                           uint32_t k0, uint32_t k1) {
    return philox4x32_10(make_uint4(c0, c1, c2, c3), k0, k1);
}

__device__ __forceinline__ float4 draw(Part& p, uint32_t k0, uint32_t k1) {
    const uint4 r = philox_block(p.hist, p.pidlo, p.pidhi, p.ctr, k0, k1);
    ++p.ctr;
    return make_float4(u01(r.x), u01(r.y), u01(r.z), u01(r.w));
}

// Structure-of-arrays particle queue: 13 words per slot, one array each.
struct Queue {
    float *x, *y, *z, *u, *v, *w, *E;
    uint32_t *vox, *hist, *pidlo, *pidhi, *ctr, *flags;
    uint32_t capacity;
};
constexpr int kQueueWords = 13;
// A phase's source queue holds only x y z u v w E, draw counter and flags
// (source_store); its other four arrays are null.
constexpr int kSourceWords = 9;

__device__ __forceinline__ void queue_store(const Queue& q, uint32_t s, const Part& p) {
    q.x[s] = p.x; q.y[s] = p.y; q.z[s] = p.z;
    q.u[s] = p.u; q.v[s] = p.v; q.w[s] = p.w; q.E[s] = p.E;
    q.vox[s] = uint32_t(p.ix) | (uint32_t(p.iy) << 10) | (uint32_t(p.iz) << 20);
    q.hist[s] = p.hist; q.pidlo[s] = p.pidlo; q.pidhi[s] = p.pidhi;
    q.ctr[s] = p.ctr; q.flags[s] = p.flags;
}
// A primary in its phase's source queue keeps 9 of the words: its history is
// the phase's first plus its slot, its particle id 1 and its voxel follows
// from its position.
__device__ __forceinline__ void source_store(const Queue& q, uint32_t s, const Part& p) {
    q.x[s] = p.x; q.y[s] = p.y; q.z[s] = p.z;
    q.u[s] = p.u; q.v[s] = p.v; q.w[s] = p.w; q.E[s] = p.E;
    q.ctr[s] = p.ctr; q.flags[s] = p.flags;
}
__device__ __forceinline__ void source_load(const Queue& q, uint32_t s, Part& p) {
    p.x = q.x[s]; p.y = q.y[s]; p.z = q.z[s];
    p.u = q.u[s]; p.v = q.v[s]; p.w = q.w[s]; p.E = q.E[s];
    p.ctr = q.ctr[s]; p.flags = q.flags[s];
}
__device__ __forceinline__ void queue_load(const Queue& q, uint32_t s, Part& p) {
    p.x = q.x[s]; p.y = q.y[s]; p.z = q.z[s];
    p.u = q.u[s]; p.v = q.v[s]; p.w = q.w[s]; p.E = q.E[s];
    const uint32_t vx = q.vox[s];
    p.ix = int(vx & 1023u); p.iy = int((vx >> 10) & 1023u); p.iz = int(vx >> 20);
    p.hist = q.hist[s]; p.pidlo = q.pidlo[s]; p.pidhi = q.pidhi[s];
    p.ctr = q.ctr[s]; p.flags = q.flags[s];
}

// ---------------------------------------------------------------- geometry
// Rotate (u,v,w) by polar cosine `cost` and azimuth phi given as (cp, sp).
// Azimuth reference: e1 = (u w, v w, -(1-w^2))/s, e2 = (-v, u, 0)/s with
// s = sqrt(1-w^2); for s^2 < 1e-10 the x and y axes.  The result is
// renormalised.
__device__ __forceinline__ void rotate(float& u, float& v, float& w, float cost, float cp,
                                       float sp) {
    const float sint = sqrtf(fmaxf(0.f, 1.f - cost * cost));
    const float s2 = 1.f - w * w;
    float un, vn, wn;
    if (s2 < 1e-10f) {
        un = cost * u + sint * cp;
        vn = cost * v + sint * sp;
        wn = cost * w;
    } else {
        const float s = sqrtf(s2);
        const float is = 1.f / s;
        un = cost * u + sint * (cp * u * w - sp * v) * is;
        vn = cost * v + sint * (cp * v * w + sp * u) * is;
        wn = cost * w - sint * cp * s;
    }
    const float n = rsqrtf(un * un + vn * vn + wn * wn);
    u = un * n; v = vn * n; w = wn * n;
}

// cos and sin of 2*pi*r for r in (0,1): evaluated at the angle 2*pi*r - pi in
// [-pi, pi] where the hardware approximations are accurate, then negated.
__device__ __forceinline__ void cossin_2pi(float r, float& c, float& s) {
    float sn, cs;
    __sincosf(kTwoPi * r - 3.14159265358979f, &sn, &cs);
    c = -cs;
    s = -sn;
}

// ---------------------------------------------------------------- device tables
struct DevTables {
    int n_mat, n_e, n_r, n_a;
    float l2min, inv_dl2;                // energy grid: u = (log2 E - l2min) * inv_dl2
    const float* ph_tot;                 // [m][i] total attenuation per unit density
    const float2* ph_cum;                // [m][i] {mu_c, mu_c + mu_pe}
    const float4* el;                    // [m][i] {R, x_ms, Sigma_moller, Sigma_brems}
    const float* rinv;                   // [m][j] T(r_j), r_j = rlo_m + j/rinv_idr_m
    const float* atab;                   // [k] ln A at ln G1 = a_l1lo + k/a_idl
    float a_l1lo, a_idl, a_g1hi;
    float x0[kMaxMat], inv_x0[kMaxMat], sigmax[kMaxMat], inv_sigmax[kMaxMat];
    float r_eabs[kMaxMat], rinv_lo[kMaxMat], rinv_idr[kMaxMat];
    float eabs_ph, eabs_el, ms_keep;      // ms_keep = 1 - ms_loss
    int flags;
};

// Energy -> table cell (i, f), linear interpolation in ln E (Sec. 2.2.2).
__device__ __forceinline__ void grid_pos(const DevTables& T, float E, int& i, float& f) {
    const float uu = (__log2f(E) - T.l2min) * T.inv_dl2;
    const float fl = floorf(uu);
    i = min(max(int(fl), 0), T.n_e - 2);
    f = fminf(fmaxf(uu - float(i), 0.f), 1.f);
}
__device__ __forceinline__ float lerpf(float a, float b, float f) { return fmaf(f, b - a, a); }

// ---------------------------------------------------------------- warp helpers
__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31u; }
__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

}  // namespace gdpm
