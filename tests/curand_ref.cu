// Test helper: Philox-4x32-10 blocks from cuRAND's curand_Philox4x32_10, used
// as an independent reference for the library's device generator.
#include <cuda_runtime.h>
#include <curand_kernel.h>
#include <stdint.h>

__global__ void ref_kernel(const uint32_t* in, uint32_t* out, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const uint32_t* a = in + 6 * i;
        uint4 o = curand_Philox4x32_10(make_uint4(a[0], a[1], a[2], a[3]), make_uint2(a[4], a[5]));
        out[4 * i + 0] = o.x;
        out[4 * i + 1] = o.y;
        out[4 * i + 2] = o.z;
        out[4 * i + 3] = o.w;
    }
}

extern "C" int curand_ref_philox(const uint32_t* in, uint32_t* out, long long n) {
    ref_kernel<<<1024, 256>>>(in, out, n);
    return (int)cudaDeviceSynchronize();
}
