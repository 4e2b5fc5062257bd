// Batch statistics (Sec. 2.2.1: mean dose and uncertainty from N_b batches;
// Sec. 3.1: sigma/Dmax over the D > 0.5 Dmax region) and the per-phantom
// Woodcock majorant.  These kernels stream voxel arrays and are bound by
// HBM bandwidth: coalesced grid-stride loops sized to the SM count.
#include <algorithm>
#include <cstring>

#include "internal.h"

namespace gdpm {
namespace {

// Largest density per material index and the smallest density overall
// (positive floats order like their bit patterns, so integer atomicMax and
// atomicMin on the bits are exact); counts voxels whose density is not a
// positive finite number (zero, negative, NaN or infinite).
__global__ void k_rhomax(const uint8_t* __restrict__ mat, const float* __restrict__ rho, size_t V,
                         int* rmax_bits, unsigned int* n_bad, int* rmin_bits) {
    __shared__ int s_max[256];
    __shared__ int s_min;
    for (int k = threadIdx.x; k < 256; k += blockDim.x) s_max[k] = 0;
    if (threadIdx.x == 0) s_min = 0x7f7fffff;
    __syncthreads();
    unsigned int bad = 0;
    int mn = 0x7f7fffff;
    for (size_t v = blockIdx.x * size_t(blockDim.x) + threadIdx.x; v < V;
         v += size_t(gridDim.x) * blockDim.x) {
        const float r = rho[v];
        if (!(r > 0.f) || isinf(r)) { ++bad; continue; }
        atomicMax(&s_max[mat[v]], __float_as_int(r));
        mn = min(mn, __float_as_int(r));
    }
    if (bad) atomicAdd(n_bad, bad);
    atomicMin(&s_min, mn);
    __syncthreads();
    for (int k = threadIdx.x; k < 256; k += blockDim.x)
        if (s_max[k]) atomicMax(&rmax_bits[k], s_max[k]);
    if (threadIdx.x == 0) atomicMin(rmin_bits, s_min);
}

// mu_max(E_i) = (1 + 1e-6) max_m mu_m(E_i) rho_max,m over the materials
// present: the interpolated majorant then bounds every voxel's
// interpolated attenuation.
__global__ void k_majorant(const float* __restrict__ tot, const float* __restrict__ rmax, int n_mat,
                           int n_e, float* maj) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_e) return;
    float m = 0.f;
    for (int k = 0; k < n_mat; ++k) m = fmaxf(m, tot[k * n_e + i] * rmax[k]);
    maj[i] = m * (1.0f + 1e-6f);
}

__device__ __forceinline__ double block_sum(double v, double* s_red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x < 32) {
        t = threadIdx.x < (blockDim.x >> 5) ? s_red[threadIdx.x] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    }
    return t;
}

// End of batch: x = E_b(v)/n_b (energy per history), sum x and x^2, clear
// the batch tally; accumulate the deposited energy into the ledger.
// Streams 48 B per voxel; every thread issues the loads of its four voxel
// pairs before any store, and the grid covers the data once.
constexpr int kFoldPairs = 4;

__global__ void __launch_bounds__(256) k_fold(SimParams P, size_t V, double inv_nb,
                                              double* __restrict__ s1, double* __restrict__ s2) {
    __shared__ double s_red[32];
    double dep = 0.0;
    const size_t n2 = V / 2;
    const size_t base = size_t(blockIdx.x) * blockDim.x * kFoldPairs + threadIdx.x;
    double2* __restrict__ a2 = reinterpret_cast<double2*>(s1);
    double2* __restrict__ b2 = reinterpret_cast<double2*>(s2);
    double2 e[kFoldPairs], a[kFoldPairs], b[kFoldPairs];
    if (P.tally_mode == 0) {
        double2* __restrict__ e2 = reinterpret_cast<double2*>(P.edep);
#pragma unroll
        for (int u = 0; u < kFoldPairs; ++u) {
            const size_t i = base + size_t(u) * blockDim.x;
            if (i < n2) { e[u] = e2[i]; a[u] = a2[i]; b[u] = b2[i]; }
        }
#pragma unroll
        for (int u = 0; u < kFoldPairs; ++u) {
            const size_t i = base + size_t(u) * blockDim.x;
            if (i < n2) e2[i] = make_double2(0.0, 0.0);
        }
    } else {
        float2* __restrict__ h2 = reinterpret_cast<float2*>(P.edep_hi);
        float2* __restrict__ l2 = reinterpret_cast<float2*>(P.edep_lo);
#pragma unroll
        for (int u = 0; u < kFoldPairs; ++u) {
            const size_t i = base + size_t(u) * blockDim.x;
            if (i < n2) {
                const float2 h = h2[i], l = l2[i];
                e[u] = make_double2(double(h.x) + double(l.x), double(h.y) + double(l.y));
                a[u] = a2[i];
                b[u] = b2[i];
            }
        }
#pragma unroll
        for (int u = 0; u < kFoldPairs; ++u) {
            const size_t i = base + size_t(u) * blockDim.x;
            if (i < n2) { h2[i] = make_float2(0.f, 0.f); l2[i] = make_float2(0.f, 0.f); }
        }
    }
#pragma unroll
    for (int u = 0; u < kFoldPairs; ++u) {
        const size_t i = base + size_t(u) * blockDim.x;
        if (i < n2) {
            dep += e[u].x + e[u].y;
            const double x0 = e[u].x * inv_nb, x1 = e[u].y * inv_nb;
            a2[i] = make_double2(a[u].x + x0, a[u].y + x1);
            b2[i] = make_double2(fma(x0, x0, b[u].x), fma(x1, x1, b[u].y));
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0 && (V & 1)) {
        double ev;
        if (P.tally_mode == 0) {
            ev = P.edep[V - 1];
            P.edep[V - 1] = 0.0;
        } else {
            ev = double(P.edep_hi[V - 1]) + double(P.edep_lo[V - 1]);
            P.edep_hi[V - 1] = 0.f;
            P.edep_lo[V - 1] = 0.f;
        }
        dep += ev;
        const double x = ev * inv_nb;
        s1[V - 1] += x;
        s2[V - 1] = fma(x, x, s2[V - 1]);
    }
    const double t = block_sum(dep, s_red);
    if (threadIdx.x == 0 && t != 0.0) atomicAdd(&P.ledger[L_DEPOSITED], t);
}

// Sums of a voxel's batch tallies b in [b0, b1) of grids of V cells
// starting at slot `first`: sum e and sum e^2, two FP64 operations per
// tally.  GB300's FP64 rate (about 5e11 FMA/s), not HBM, bounds the fold,
// so the batch weights are applied once per voxel, not per tally.  CLEAR
// then zeroes the tallies, leaving the grids ready for the next
// calculation; the stores come after all the loads, which a store between
// them would serialise (the compiler cannot tell the addresses apart).
template <bool CLEAR>
__device__ __forceinline__ void batch_sums(const SimParams& P, size_t V, size_t first, size_t v,
                                           int b0, int b1, double& se, double& sq) {
    for (int b = b0; b < b1; ++b) {
        const size_t k = (first + size_t(b)) * V + v;
        const double e = P.tally_mode == 0 ? P.edep[k] : double(P.edep_hi[k]) + double(P.edep_lo[k]);
        se += e;
        sq = fma(e, e, sq);
    }
    if (CLEAR) {
        for (int b = b0; b < b1; ++b) {
            const size_t k = (first + size_t(b)) * V + v;
            if (P.tally_mode == 0) {
                P.edep[k] = 0.0;
            } else {
                P.edep_hi[k] = 0.f;
                P.edep_lo[k] = 0.f;
            }
        }
    }
}

// All batches at once (batches run side by side, one tally grid each):
// s1 += sum_b E_b/n_b, s2 += sum_b (E_b/n_b)^2 per voxel (the sums of a run
// in parts accumulate).  The first n_big batches hold one history more.
// The grids are left zeroed.
__global__ void __launch_bounds__(256) k_fold_batches(SimParams P, size_t V, int nbatch,
                                                      double inv_big, double inv_small, int n_big,
                                                      double* __restrict__ s1, double* __restrict__ s2) {
    __shared__ double s_red[32];
    double dep = 0.0;
    const int nbig = min(n_big, nbatch);
    for (size_t v = blockIdx.x * size_t(blockDim.x) + threadIdx.x; v < V;
         v += size_t(gridDim.x) * blockDim.x) {
        double eb = 0.0, qb = 0.0, es = 0.0, qs = 0.0;
        batch_sums<true>(P, V, 0, v, 0, nbig, eb, qb);
        batch_sums<true>(P, V, 0, v, nbig, nbatch, es, qs);
        dep += eb + es;
        s1[v] += fma(eb, inv_big, es * inv_small);
        s2[v] += fma(qb, inv_big * inv_big, qs * (inv_small * inv_small));
    }
    const double t = block_sum(dep, s_red);
    if (threadIdx.x == 0 && t != 0.0) atomicAdd(&P.ledger[L_DEPOSITED], t);
}

// Dose matrix: sub-problem k (row k of the fluence map; blockIdx.y) tallied
// into slots k*nb .. k*nb+nb-1.  Writes its mean dose and standard error per
// voxel (MeV/g per history of that sub-problem) to dose[(k-k0)*V + v] and
// sigma[...]; with one batch only the dose.  inv_n[2k], inv_n[2k+1] are
// 1/(histories of a long batch) and 1/(histories of a short batch) of
// sub-problem k, whose first nbig[k] batches are the long ones.
__global__ void __launch_bounds__(256) k_fold_sub(SimParams P, size_t V, uint32_t k0, int nb,
                                                  const double* __restrict__ inv_n,
                                                  const uint32_t* __restrict__ nbig, double dvol,
                                                  double* __restrict__ dose, double* __restrict__ sigma) {
    __shared__ double s_red[32];
    const uint32_t k = k0 + blockIdx.y;
    const double ib = inv_n[2 * k], is = inv_n[2 * k + 1];
    const uint32_t n_big = nbig[k];
    double dep = 0.0;
    const int nbg = int(min(n_big, uint32_t(nb)));
    for (size_t v = blockIdx.x * size_t(blockDim.x) + threadIdx.x; v < V;
         v += size_t(gridDim.x) * blockDim.x) {
        double eb = 0.0, qb = 0.0, es = 0.0, qs = 0.0;
        batch_sums<false>(P, V, size_t(k) * nb, v, 0, nbg, eb, qb);
        batch_sums<false>(P, V, size_t(k) * nb, v, nbg, nb, es, qs);
        dep += eb + es;
        const double a1 = fma(eb, ib, es * is);
        const double a2 = fma(qb, ib * ib, qs * (is * is));
        const double mass = double(P.rho[v]) * dvol;
        double im = double(1.0f / float(mass));
        im = im * fma(-mass, im, 2.0);                       // Newton step for 1/mass
        const size_t o = size_t(blockIdx.y) * V + v;
        const double mean = a1 / nb;
        dose[o] = mean * im;
        if (sigma && nb > 1) {
            const double var = fmax(0.0, (a2 - nb * mean * mean) / (double(nb) * (nb - 1)));
            double sd = 0.0;
            if (var > 0.0) {
                double y = double(rsqrtf(float(var)));
                y = y * fma(-0.5 * var * y, y, 1.5);         // Newton step for 1/sqrt(var)
                sd = var * y;
            }
            sigma[o] = sd * im;
        }
    }
    const double t = block_sum(dep, s_red);
    if (threadIdx.x == 0 && t != 0.0) atomicAdd(&P.ledger[L_DEPOSITED], t);
}

// Mean and standard error per voxel in MeV/g per history; Dmax.  FP64
// division and square root are slow on this part, so 1/mass and sqrt(var)
// start from FP32 estimates and take one FP64 Newton step each (relative
// error ~1e-14).
__global__ void k_finalize(const double* __restrict__ s1, const double* __restrict__ s2,
                           const float* __restrict__ rho, size_t V, int nb, double dvol,
                           double* __restrict__ dose, double* __restrict__ sigma,
                           unsigned long long* dmax_bits, float metric_min_rho) {
    double mx = 0.0;
    const double inv_n = 1.0 / nb;
    const double inv_nn1 = 1.0 / (double(nb) * (nb - 1));
    for (size_t v = blockIdx.x * size_t(blockDim.x) + threadIdx.x; v < V;
         v += size_t(gridDim.x) * blockDim.x) {
        const double mean = s1[v] * inv_n;
        const double var = fmax(0.0, (s2[v] - nb * mean * mean) * inv_nn1);
        const float r = rho[v];
        const double mass = double(r) * dvol;
        double im = double(1.0f / float(mass));
        im = im * fma(-mass, im, 2.0);                       // Newton step for 1/mass
        const double d = mean * im;
        double sd = 0.0;
        if (var > 0.0) {
            double y = double(rsqrtf(float(var)));
            y = y * fma(-0.5 * var * y, y, 1.5);             // Newton step for 1/sqrt(var)
            sd = var * y;
        }
        if (dose) dose[v] = d;
        if (sigma) sigma[v] = sd * im;
        if (r >= metric_min_rho) mx = fmax(mx, d);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0 && mx > 0.0)
        atomicMax(dmax_bits, (unsigned long long)__double_as_longlong(mx));
}

// Sec. 3.1 precision metric: mean of sigma over voxels with D > 0.5 Dmax
// (both over voxels at least as dense as metric_min_rho: air voxels of tiny
// mass have meaningless dose noise).
__global__ void k_metric(const double* __restrict__ dose, const double* __restrict__ sigma,
                         const float* __restrict__ rho, size_t V,
                         const unsigned long long* dmax_bits, double* ledger, float metric_min_rho) {
    __shared__ double s_red[32];
    const double dmax = __longlong_as_double((long long)*dmax_bits);
    double acc = 0.0, cnt = 0.0;
    for (size_t v = blockIdx.x * size_t(blockDim.x) + threadIdx.x; v < V;
         v += size_t(gridDim.x) * blockDim.x) {
        if (dose[v] > 0.5 * dmax && rho[v] >= metric_min_rho) {
            acc += sigma[v];
            cnt += 1.0;
        }
    }
    const double a = block_sum(acc, s_red);
    __syncthreads();
    const double c = block_sum(cnt, s_red);
    if (threadIdx.x == 0) {
        if (a != 0.0) atomicAdd(&ledger[L_SIGSUM], a);
        if (c != 0.0) atomicAdd(&ledger[L_SIGCNT], c);
    }
}

}  // namespace

int phantom_density_max(gdpm_ctx* ctx, gdpm_phantom* ph) {
    const size_t V = size_t(ph->nx) * ph->ny * ph->nz;
    int rc = ensure(ph->rhomax, 256 * sizeof(float) + 16);
    if (rc) return rc;
    GDPM_CUDA_TRY(cudaMemsetAsync(ph->rhomax.p, 0, 256 * sizeof(float) + 16, ctx->stream));
    int* bits = static_cast<int*>(ph->rhomax.p);
    unsigned int* bad = reinterpret_cast<unsigned int*>(bits + 256);
    int* rmin = bits + 257;
    const int big = 0x7f7fffff;                 // FLT_MAX: the minimum's starting value
    GDPM_CUDA_TRY(cudaMemcpyAsync(rmin, &big, 4, cudaMemcpyHostToDevice, ctx->stream));
    k_rhomax<<<ctx->sm_count * 4, 256, 0, ctx->stream>>>(static_cast<const uint8_t*>(ph->mat.p),
                                                          static_cast<const float*>(ph->rho.p), V,
                                                          bits, bad, rmin);
    GDPM_CUDA_TRY(cudaGetLastError());
    unsigned int h[260];
    GDPM_CUDA_TRY(cudaMemcpyAsync(h, ph->rhomax.p, 258 * sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    GDPM_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    if (h[256] != 0) return GDPM_E_ARG;
    std::memcpy(&ph->rhomin_host, &h[257], 4);
    for (int k = 0; k < 256; ++k) {
        float f;
        std::memcpy(&f, &h[k], 4);
        ph->rhomax_host[k] = f;
    }
    return GDPM_OK;
}

}  // namespace gdpm

namespace gdpm {

// Launchers with every buffer and the stream explicit (a dose calculation's
// buffers belong to its runner, or to the no-allocation static array).
int launch_majorant_into(cudaStream_t st, gdpm_phantom* ph, gdpm_tables* t, float* maj) {
    k_majorant<<<(t->n_e + 127) / 128, 128, 0, st>>>(static_cast<const float*>(t->ph_tot.p),
                                                     static_cast<const float*>(ph->rhomax.p),
                                                     t->n_mat, t->n_e, maj);
    GDPM_CUDA_TRY(cudaGetLastError());
    return GDPM_OK;
}

int launch_fold_into(gdpm_ctx* ctx, cudaStream_t st, const SimParams& P, size_t V, uint32_t nb,
                     double* s1, double* s2) {
    const size_t per_block = size_t(256) * kFoldPairs;
    const unsigned grid = unsigned(std::max<size_t>(1, (V / 2 + per_block - 1) / per_block));
    k_fold<<<grid, 256, 0, st>>>(P, V, 1.0 / double(nb), s1, s2);
    GDPM_CUDA_TRY(cudaGetLastError());
    return GDPM_OK;
}

int launch_fold_batches(gdpm_ctx* ctx, cudaStream_t st, const SimParams& P, size_t V, int n_batches,
                        uint32_t nb_small, uint32_t nb_rem, double* s1, double* s2) {
    k_fold_batches<<<ctx->sm_count * 8, 256, 0, st>>>(P, V, n_batches, 1.0 / double(nb_small + 1),
                                                        1.0 / double(nb_small), int(nb_rem), s1, s2);
    GDPM_CUDA_TRY(cudaGetLastError());
    return GDPM_OK;
}

int launch_fold_sub(gdpm_ctx* ctx, cudaStream_t st, const SimParams& P, size_t V, uint32_t k0,
                    uint32_t nk, int nb, const double* inv_n, const uint32_t* nbig, double* dose,
                    double* sigma) {
    const double dvol = double(P.dx) * P.dy * P.dz;
    const uint32_t gx = uint32_t(std::min<size_t>((V + 255) / 256, size_t(ctx->sm_count) * 4));
    k_fold_sub<<<dim3(gx, nk), 256, 0, st>>>(P, V, k0, nb, inv_n, nbig, dvol, dose, sigma);
    GDPM_CUDA_TRY(cudaGetLastError());
    return GDPM_OK;
}

int launch_finalize_into(gdpm_ctx* ctx, cudaStream_t st, const SimParams& P, size_t V,
                         int n_batches, const double* s1, const double* s2, double* dose,
                         double* sigma) {
    const double dvol = double(P.dx) * P.dy * P.dz;
    unsigned long long* dmax_bits = reinterpret_cast<unsigned long long*>(&P.ledger[L_DMAX]);
    k_finalize<<<ctx->sm_count * 4, 256, 0, st>>>(s1, s2, P.rho, V, n_batches, dvol, dose, sigma,
                                                    dmax_bits, ctx->metric_min_rho);
    GDPM_CUDA_TRY(cudaGetLastError());
    if (dose && sigma) {
        k_metric<<<ctx->sm_count * 4, 256, 0, st>>>(dose, sigma, P.rho, V, dmax_bits, P.ledger,
                                                      ctx->metric_min_rho);
        GDPM_CUDA_TRY(cudaGetLastError());
    }
    return GDPM_OK;
}

}  // namespace gdpm
