// Microbenchmarks of the resources the transport kernels lean on.
//
// The transport is not a dense contraction: its candidate bounds are the
// L2 atomic units that take the dose tally (one FP64 add per voxel a charged
// particle crosses, Sec. 2.2.2 tally into a per-batch grid), the FP32 issue
// rate, the MUFU unit (one log per Woodcock flight, sincos and rsqrt per
// deflection) and the FP64 pipe (the ledger and the batch fold).  Each kernel
// here saturates one of them with a persistent grid and reports operations
// per second, so that the rates the roofline divides by are measured on
// the GPU at hand rather than assumed.
#include "internal.h"

namespace gdpm {
namespace {

constexpr int kMbThreads = 256;

__device__ __forceinline__ uint32_t xorshift32(uint32_t x) {
    x ^= x << 13;
    x ^= x >> 17;
    x ^= x << 5;
    return x;
}

// Scattered atomic adds of 1 into n_slots cells: kind 0 FP64 without a
// returned value (RED), kind 1 FP32 RED, kind 2 FP32 with the returned old
// value consumed (ATOM, as in the compensated pair tally).
template <int KIND>
__global__ void __launch_bounds__(kMbThreads) k_mb_atomics(void* buf, uint32_t n_slots,
                                                           uint32_t per_thread) {
    uint32_t s = (blockIdx.x * kMbThreads + threadIdx.x) * 2654435761u + 0x9E3779B9u;
    if (s == 0) s = 1;
    float acc = 0.f;
#pragma unroll 4
    for (uint32_t i = 0; i < per_thread; ++i) {
        s = xorshift32(s);
        const uint32_t slot = __umulhi(s, n_slots);
        if (KIND == 0) {
            atomicAdd(static_cast<double*>(buf) + slot, 1.0);
        } else if (KIND == 1) {
            atomicAdd(static_cast<float*>(buf) + slot, 1.0f);
        } else {
            acc += atomicAdd(static_cast<float*>(buf) + slot, 1.0f);
        }
    }
    // never taken (counts are non-negative); keeps the returned values live
    if (KIND == 2 && acc < 0.f) static_cast<float*>(buf)[0] = acc;
}

// Eight independent dependency chains per thread, 64 operations per trip.
// Kind 3: FP32 FMA; kind 4: FP64 FMA; kind 5: MUFU base-2 logarithm (plus
// one FP32 add to keep the argument positive, far below the MUFU rate).
template <int KIND>
__global__ void __launch_bounds__(kMbThreads) k_mb_alu(float* sink, uint32_t trips) {
    const float t = float(threadIdx.x & 31) * 1e-3f;
    if (KIND == 3) {
        float a[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) a[k] = 1.0f + t + 0.01f * k;
        for (uint32_t i = 0; i < trips; ++i) {
#pragma unroll
            for (int j = 0; j < 8; ++j) {
#pragma unroll
                for (int k = 0; k < 8; ++k) a[k] = fmaf(a[k], 0.999f, 1e-3f);
            }
        }
        float sum = 0.f;
#pragma unroll
        for (int k = 0; k < 8; ++k) sum += a[k];
        if (sum == -1.f) sink[0] = sum;
    } else if (KIND == 4) {
        double a[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) a[k] = 1.0 + t + 0.01 * k;
        for (uint32_t i = 0; i < trips; ++i) {
#pragma unroll
            for (int j = 0; j < 8; ++j) {
#pragma unroll
                for (int k = 0; k < 8; ++k) a[k] = fma(a[k], 0.999, 1e-3);
            }
        }
        double sum = 0.0;
#pragma unroll
        for (int k = 0; k < 8; ++k) sum += a[k];
        if (sum == -1.0) sink[0] = float(sum);
    } else {
        float a[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) a[k] = 2.0f + t + 0.01f * k;
        for (uint32_t i = 0; i < trips; ++i) {
#pragma unroll
            for (int j = 0; j < 8; ++j) {
#pragma unroll
                for (int k = 0; k < 8; ++k) a[k] = __log2f(a[k]) + 2.0f;
            }
        }
        float sum = 0.f;
#pragma unroll
        for (int k = 0; k < 8; ++k) sum += a[k];
        if (sum == -1.f) sink[0] = sum;
    }
}

template <typename K>
int resident_grid(const gdpm_ctx* ctx, K kernel, int& grid) {
    int per_sm = 0;
    GDPM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kMbThreads, 0));
    grid = ctx->sm_count * (per_sm > 0 ? per_sm : 1);
    return GDPM_OK;
}

int launch_mb(gdpm_ctx* ctx, int kind, void* buf, uint32_t n_slots, uint32_t per, int grid) {
    cudaStream_t s = ctx->stream;
    switch (kind) {
        case GDPM_MB_RED_F64: k_mb_atomics<0><<<grid, kMbThreads, 0, s>>>(buf, n_slots, per); break;
        case GDPM_MB_RED_F32: k_mb_atomics<1><<<grid, kMbThreads, 0, s>>>(buf, n_slots, per); break;
        case GDPM_MB_ATOM_F32: k_mb_atomics<2><<<grid, kMbThreads, 0, s>>>(buf, n_slots, per); break;
        case GDPM_MB_FFMA: k_mb_alu<3><<<grid, kMbThreads, 0, s>>>(static_cast<float*>(buf), per); break;
        case GDPM_MB_DFMA: k_mb_alu<4><<<grid, kMbThreads, 0, s>>>(static_cast<float*>(buf), per); break;
        default: k_mb_alu<5><<<grid, kMbThreads, 0, s>>>(static_cast<float*>(buf), per); break;
    }
    GDPM_CUDA_TRY(cudaGetLastError());
    return GDPM_OK;
}

}  // namespace
}  // namespace gdpm

using namespace gdpm;

extern "C" int gdpm_microbench(gdpm_ctx* ctx, int kind, void* buf, uint64_t n_slots, uint64_t n_ops,
                               double* ops_done, double* ms) {
    if (!ctx || !buf || !ops_done || !ms || kind < GDPM_MB_RED_F64 || kind > GDPM_MB_MUFU_LG2)
        return GDPM_E_ARG;
    if (n_slots < 1 || n_slots > 0xFFFFFFFFull || n_ops < 1) return GDPM_E_ARG;
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, buf) != cudaSuccess || at.type != cudaMemoryTypeDevice) {
        cudaGetLastError();
        return GDPM_E_ARG;
    }
    GDPM_CUDA_TRY(cudaSetDevice(ctx->device));
    const bool atomics = kind <= GDPM_MB_ATOM_F32;
    int grid = 0, rc = 0;
    switch (kind) {
        case GDPM_MB_RED_F64: rc = resident_grid(ctx, k_mb_atomics<0>, grid); break;
        case GDPM_MB_RED_F32: rc = resident_grid(ctx, k_mb_atomics<1>, grid); break;
        case GDPM_MB_ATOM_F32: rc = resident_grid(ctx, k_mb_atomics<2>, grid); break;
        case GDPM_MB_FFMA: rc = resident_grid(ctx, k_mb_alu<3>, grid); break;
        case GDPM_MB_DFMA: rc = resident_grid(ctx, k_mb_alu<4>, grid); break;
        default: rc = resident_grid(ctx, k_mb_alu<5>, grid); break;
    }
    if (rc) return rc;
    // per-thread work: atomics count one add each, the ALU kernels 64 per trip
    const uint64_t threads = uint64_t(grid) * kMbThreads;
    const uint64_t unit = atomics ? 1 : 64;
    const uint64_t per = (n_ops + threads * unit - 1) / (threads * unit);
    if (per > 0xFFFFFFFFull) return GDPM_E_ARG;
    const size_t elem = kind == GDPM_MB_RED_F64 ? 8 : 4;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    GDPM_CUDA_TRY(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return GDPM_E_CUDA;
    }
    float t = 0.f;
    auto run = [&]() -> int {
        // warm-up launch, then the buffer is cleared so that it holds the
        // timed launch's adds only
        if ((rc = launch_mb(ctx, kind, buf, uint32_t(n_slots), uint32_t(per), grid))) return rc;
        GDPM_CUDA_TRY(cudaMemsetAsync(buf, 0, atomics ? size_t(n_slots) * elem : 4, ctx->stream));
        GDPM_CUDA_TRY(cudaEventRecord(e0, ctx->stream));
        if ((rc = launch_mb(ctx, kind, buf, uint32_t(n_slots), uint32_t(per), grid))) return rc;
        GDPM_CUDA_TRY(cudaEventRecord(e1, ctx->stream));
        GDPM_CUDA_TRY(cudaEventSynchronize(e1));
        GDPM_CUDA_TRY(cudaEventElapsedTime(&t, e0, e1));
        return GDPM_OK;
    };
    rc = run();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    *ops_done = double(threads) * double(per) * double(unit);
    *ms = double(t);
    return GDPM_OK;
}
