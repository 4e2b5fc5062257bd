// Batch statistics (Sec. 2.2.1: mean dose and uncertainty from N_b batches;
// Sec. 3.1: sigma/Dmax over the D > 0.5 Dmax region) and the per-phantom
// Woodcock majorant.  These kernels stream voxel arrays and are bound by
// HBM bandwidth: coalesced grid-stride loops sized to the SM count.
#include "internal.h"

namespace gdpm {
namespace {

// Largest density per material index (positive floats order like their bit
// patterns, so an integer atomicMax on the bits is exact); counts voxels with
// non-positive density.
__global__ void k_rhomax(const uint8_t* __restrict__ mat, const float* __restrict__ rho, size_t V,
                         int* rmax_bits, unsigned int* n_bad) {
    __shared__ int s_max[256];
    for (int k = threadIdx.x; k < 256; k += blockDim.x) s_max[k] = 0;
    __syncthreads();
    unsigned int bad = 0;
    for (size_t v = blockIdx.x * size_t(blockDim.x) + threadIdx.x; v < V;
         v += size_t(gridDim.x) * blockDim.x) {
        const float r = rho[v];
        if (!(r > 0.f)) { ++bad; continue; }
        atomicMax(&s_max[mat[v]], __float_as_int(r));
    }
    if (bad) atomicAdd(n_bad, bad);
    __syncthreads();
    for (int k = threadIdx.x; k < 256; k += blockDim.x)
        if (s_max[k]) atomicMax(&rmax_bits[k], s_max[k]);
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
__global__ void k_fold(SimParams P, size_t V, double inv_nb, double* __restrict__ s1,
                       double* __restrict__ s2) {
    __shared__ double s_red[32];
    double dep = 0.0;
    for (size_t v = blockIdx.x * size_t(blockDim.x) + threadIdx.x; v < V;
         v += size_t(gridDim.x) * blockDim.x) {
        double e;
        if (P.tally_mode == 0) {
            e = P.edep[v];
            P.edep[v] = 0.0;
        } else {
            e = double(P.edep_hi[v]) + double(P.edep_lo[v]);
            P.edep_hi[v] = 0.f;
            P.edep_lo[v] = 0.f;
        }
        dep += e;
        const double x = e * inv_nb;
        s1[v] += x;
        s2[v] += x * x;
    }
    const double t = block_sum(dep, s_red);
    if (threadIdx.x == 0 && t != 0.0) atomicAdd(&P.ledger[L_DEPOSITED], t);
}

// Mean and standard error per voxel in MeV/g per history; Dmax.
__global__ void k_finalize(const double* __restrict__ s1, const double* __restrict__ s2,
                           const float* __restrict__ rho, size_t V, int nb, double dvol,
                           double* __restrict__ dose, double* __restrict__ sigma,
                           unsigned long long* dmax_bits) {
    double mx = 0.0;
    const double inv_n = 1.0 / nb;
    const double inv_nn1 = 1.0 / (double(nb) * (nb - 1));
    for (size_t v = blockIdx.x * size_t(blockDim.x) + threadIdx.x; v < V;
         v += size_t(gridDim.x) * blockDim.x) {
        const double mean = s1[v] * inv_n;
        const double var = fmax(0.0, (s2[v] - nb * mean * mean) * inv_nn1);
        const double inv_mass = 1.0 / (double(rho[v]) * dvol);
        const double d = mean * inv_mass;
        if (dose) dose[v] = d;
        if (sigma) sigma[v] = sqrt(var) * inv_mass;
        mx = fmax(mx, d);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0 && mx > 0.0)
        atomicMax(dmax_bits, (unsigned long long)__double_as_longlong(mx));
}

// Sec. 3.1 precision metric: mean of sigma over voxels with D > 0.5 Dmax.
__global__ void k_metric(const double* __restrict__ dose, const double* __restrict__ sigma, size_t V,
                         const unsigned long long* dmax_bits, double* ledger) {
    __shared__ double s_red[32];
    const double dmax = __longlong_as_double((long long)*dmax_bits);
    double acc = 0.0, cnt = 0.0;
    for (size_t v = blockIdx.x * size_t(blockDim.x) + threadIdx.x; v < V;
         v += size_t(gridDim.x) * blockDim.x) {
        if (dose[v] > 0.5 * dmax) {
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
    k_rhomax<<<ctx->sm_count * 4, 256, 0, ctx->stream>>>(static_cast<const uint8_t*>(ph->mat.p),
                                                          static_cast<const float*>(ph->rho.p), V,
                                                          bits, bad);
    GDPM_CUDA_TRY(cudaGetLastError());
    unsigned int h[260];
    GDPM_CUDA_TRY(cudaMemcpyAsync(h, ph->rhomax.p, 257 * sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    GDPM_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    if (h[256] != 0) return GDPM_E_ARG;
    for (int k = 0; k < 256; ++k) {
        float f;
        std::memcpy(&f, &h[k], 4);
        ph->rhomax_host[k] = f;
    }
    return GDPM_OK;
}

int build_majorant(gdpm_ctx* ctx, gdpm_phantom* ph, gdpm_tables* t) {
    if (ph->maj_tables_id == t->id && ph->maj.p) return GDPM_OK;
    int rc = ensure(ph->maj, sizeof(float) * t->n_e);
    if (rc) return rc;
    k_majorant<<<(t->n_e + 127) / 128, 128, 0, ctx->stream>>>(
        static_cast<const float*>(t->ph_tot.p), static_cast<const float*>(ph->rhomax.p), t->n_mat,
        t->n_e, static_cast<float*>(ph->maj.p));
    GDPM_CUDA_TRY(cudaGetLastError());
    ph->maj_tables_id = t->id;
    return GDPM_OK;
}

int launch_fold(gdpm_ctx* ctx, const SimParams& P, size_t V, uint32_t nb) {
    k_fold<<<ctx->sm_count * 4, 256, 0, ctx->stream>>>(P, V, 1.0 / double(nb),
                                                         static_cast<double*>(ctx->ws.s1.p),
                                                         static_cast<double*>(ctx->ws.s2.p));
    GDPM_CUDA_TRY(cudaGetLastError());
    return GDPM_OK;
}

int launch_finalize(gdpm_ctx* ctx, const SimParams& P, size_t V, int n_batches, double* dose,
                    double* sigma) {
    const double dvol = double(P.dx) * P.dy * P.dz;
    unsigned long long* dmax_bits = reinterpret_cast<unsigned long long*>(&P.ledger[L_DMAX]);
    k_finalize<<<ctx->sm_count * 4, 256, 0, ctx->stream>>>(
        static_cast<const double*>(ctx->ws.s1.p), static_cast<const double*>(ctx->ws.s2.p), P.rho, V,
        n_batches, dvol, dose, sigma, dmax_bits);
    GDPM_CUDA_TRY(cudaGetLastError());
    if (dose && sigma) {
        k_metric<<<ctx->sm_count * 4, 256, 0, ctx->stream>>>(dose, sigma, V, dmax_bits, P.ledger);
        GDPM_CUDA_TRY(cudaGetLastError());
    }
    return GDPM_OK;
}

}  // namespace gdpm

namespace gdpm {

// Variants of the launchers above that take every buffer explicitly (used by
// the no-allocation entry point, whose buffers live in a static array).
int launch_majorant_into(gdpm_ctx* ctx, gdpm_phantom* ph, gdpm_tables* t, float* maj) {
    k_majorant<<<(t->n_e + 127) / 128, 128, 0, ctx->stream>>>(
        static_cast<const float*>(t->ph_tot.p), static_cast<const float*>(ph->rhomax.p), t->n_mat,
        t->n_e, maj);
    GDPM_CUDA_TRY(cudaGetLastError());
    return GDPM_OK;
}

int launch_fold_into(gdpm_ctx* ctx, const SimParams& P, size_t V, uint32_t nb, double* s1, double* s2) {
    k_fold<<<ctx->sm_count * 4, 256, 0, ctx->stream>>>(P, V, 1.0 / double(nb), s1, s2);
    GDPM_CUDA_TRY(cudaGetLastError());
    return GDPM_OK;
}

int launch_finalize_into(gdpm_ctx* ctx, const SimParams& P, size_t V, int n_batches,
                         const double* s1, const double* s2, double* dose, double* sigma) {
    const double dvol = double(P.dx) * P.dy * P.dz;
    unsigned long long* dmax_bits = reinterpret_cast<unsigned long long*>(&P.ledger[L_DMAX]);
    k_finalize<<<ctx->sm_count * 4, 256, 0, ctx->stream>>>(s1, s2, P.rho, V, n_batches, dvol, dose,
                                                             sigma, dmax_bits);
    GDPM_CUDA_TRY(cudaGetLastError());
    if (dose && sigma) {
        k_metric<<<ctx->sm_count * 4, 256, 0, ctx->stream>>>(dose, sigma, V, dmax_bits, P.ledger);
        GDPM_CUDA_TRY(cudaGetLastError());
    }
    return GDPM_OK;
}

}  // namespace gdpm
