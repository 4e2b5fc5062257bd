// Test helper: outputs of cuRAND's device-side Philox4_32_10 generator, used
// as an independent library reference for the Philox implementations.
#include <cstdint>
#include <curand_kernel.h>

__global__ void k_ref(unsigned long long seed, unsigned long long subseq, int n_calls,
                      uint32_t* out) {
    curandStatePhilox4_32_10_t st;
    curand_init(seed, subseq, 0, &st);
    for (int i = 0; i < n_calls; ++i) {
        const uint4 v = curand4(&st);
        out[4 * i] = v.x; out[4 * i + 1] = v.y; out[4 * i + 2] = v.z; out[4 * i + 3] = v.w;
    }
}

extern "C" int curand_philox_ref(unsigned long long seed, unsigned long long subseq, int n_calls,
                                 uint32_t* host_out) {
    uint32_t* d = nullptr;
    if (cudaMalloc(&d, sizeof(uint32_t) * 4 * n_calls) != cudaSuccess) return -1;
    k_ref<<<1, 1>>>(seed, subseq, n_calls, d);
    cudaError_t e = cudaMemcpy(host_out, d, sizeof(uint32_t) * 4 * n_calls, cudaMemcpyDeviceToHost);
    cudaFree(d);
    return e == cudaSuccess ? 0 : -2;
}
