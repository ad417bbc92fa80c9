// Test kernel: evaluates the library's device math helpers (rsqrt_nr,
// rcp_nr, atan_over of bpm_devmath.cuh) on arrays of inputs, so that a test
// can compare them with correctly rounded references.  Test code only.
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../paper_2603_27279_gb300/csrc/bpm_devmath.cuh"

namespace {
__global__ void k_devmath(int64_t n, const double* a, const double* c, double* rs, double* rc, double* at) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    rs[i] = bpm::rsqrt_nr(a[i]);
    rc[i] = bpm::rcp_nr(a[i]);
    at[i] = bpm::atan_over(a[i], c[i]);
}
}  // namespace

// a, c inputs and rs = rsqrt_nr(a), rc = rcp_nr(a), at = atan_over(a, c),
// all device arrays of n doubles; returns a cudaError_t after synchronising.
extern "C" int devmath_eval(int64_t n, const double* a, const double* c, double* rs, double* rc, double* at) {
    if (n <= 0) return 0;
    k_devmath<<<(unsigned)((n + 255) / 256), 256>>>(n, a, c, rs, rc, at);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    return (int)e;
}
