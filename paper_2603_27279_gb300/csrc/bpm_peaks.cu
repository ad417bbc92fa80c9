// Throughput probe of the arithmetic pipes that bound this library's
// kernels: FP64 fused multiply-add and add, FP32 fused multiply-add (scalar
// and the packed two-lane form) and the FP32 reciprocal square root of the
// special-function unit.  The paper has no counterpart; the measured rates are
// the denominators of the roofline fractions of the ALU-bound kernels.
//
// Each thread runs eight independent dependency chains of one operation, the
// SMs are filled (256-thread blocks, eight per SM), and the kernel runs for
// about 50 ms.  The time comes from CUDA events; the SM clock of the run from
// the cycle counter and the global timer read by each block's first thread,
// so that the rate per SM per clock does not depend on the clock the run
// happened to get.
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/bpm.h"

namespace bpm {
void set_handleless_error(const std::string& msg);

namespace {

constexpr int kProbeThreads = 256;
constexpr int kProbeBlocksPerSm = 8;
constexpr int kChains = 8;

enum ProbeOp { OP_DFMA = 0, OP_FFMA = 1, OP_FFMA2 = 2, OP_RSQRT = 3, OP_DADD = 4, OP_COUNT = 5 };

// the chains' multiplier and addend: compile-time constants, so that every
// operation reads one register and two constant operands (no register bank
// conflicts between the chains)
constexpr double kMulD = 0.999999, kAddD = 1e-6;
constexpr float kMulF = 0.9999f, kAddF = 1e-4f;

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

template <int OP>
__global__ void __launch_bounds__(kProbeThreads, kProbeBlocksPerSm) k_probe(int iters, double* sink, unsigned long long* clk) {
    unsigned long long c0 = 0, t0 = 0;
    if (threadIdx.x == 0) {
        c0 = clock64();
        t0 = global_ns();
    }
    const float s = 1.0f + 1e-7f * (float)(threadIdx.x & 15);
    double out = 0.0;
    if (OP == OP_DFMA) {
        double a[kChains];
        for (int k = 0; k < kChains; ++k) a[k] = 0.5 + 0.01 * k + 1e-9 * threadIdx.x;
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int k = 0; k < kChains; ++k) a[k] = fma(a[k], kMulD, kAddD);
        }
        for (int k = 0; k < kChains; ++k) out += a[k];
    } else if (OP == OP_DADD) {
        double a[kChains];
        for (int k = 0; k < kChains; ++k) a[k] = 0.5 + 0.01 * k + 1e-9 * threadIdx.x;
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int k = 0; k < kChains; ++k) a[k] = a[k] + kAddD;
        }
        for (int k = 0; k < kChains; ++k) out += a[k];
    } else if (OP == OP_FFMA) {
        float a[kChains];
        for (int k = 0; k < kChains; ++k) a[k] = 0.5f + 0.01f * k + 1e-6f * threadIdx.x;
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int k = 0; k < kChains; ++k) a[k] = fmaf(a[k], kMulF, kAddF);
        }
        for (int k = 0; k < kChains; ++k) out += a[k];
    } else if (OP == OP_FFMA2) {
        float2 a[kChains];
        for (int k = 0; k < kChains; ++k) a[k] = make_float2(0.5f + 0.01f * k, 0.25f + 1e-6f * threadIdx.x);
        const float2 m = make_float2(kMulF, kMulF), b = make_float2(kAddF * s, kAddF);
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int k = 0; k < kChains; ++k) a[k] = __ffma2_rn(a[k], m, b);
        }
        for (int k = 0; k < kChains; ++k) out += a[k].x + a[k].y;
    } else {
        float a[kChains];
        for (int k = 0; k < kChains; ++k) a[k] = (1.0f + 0.1f * k) * s;
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int k = 0; k < kChains; ++k) asm volatile("rsqrt.approx.ftz.f32 %0, %0;" : "+f"(a[k]));
        }
        for (int k = 0; k < kChains; ++k) out += a[k];
    }
    sink[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = out;
    if (threadIdx.x == 0) {
        clk[2 * blockIdx.x] = clock64() - c0;
        clk[2 * blockIdx.x + 1] = global_ns() - t0;
    }
}

typedef void (*ProbeKernel)(int, double*, unsigned long long*);

ProbeKernel probe_kernel(int op) {
    switch (op) {
        case OP_DFMA: return k_probe<OP_DFMA>;
        case OP_FFMA: return k_probe<OP_FFMA>;
        case OP_FFMA2: return k_probe<OP_FFMA2>;
        case OP_DADD: return k_probe<OP_DADD>;
        default: return k_probe<OP_RSQRT>;
    }
}

// lane operations per chain step: the packed FMA works on two lanes
double lanes_per_step(int op) { return op == OP_FFMA2 ? 2.0 : 1.0; }

int probe_fail(const std::string& msg) {
    set_handleless_error("bpm_measure_pipes: " + msg);
    return BPM_ERR_CUDA;
}

}  // namespace
}  // namespace bpm

extern "C" int bpm_measure_pipes(double out[20]) {
    using namespace bpm;
    if (!out) {
        set_handleless_error("bpm_measure_pipes: out is NULL");
        return BPM_ERR_ARG;
    }
    int dev = 0;
    cudaDeviceProp prop;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess)
        return probe_fail("no device");
    const int n_sm = prop.multiProcessorCount;
    const int blocks = n_sm * kProbeBlocksPerSm;
    double* sink = nullptr;
    unsigned long long* clk = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    unsigned long long* hclk = new unsigned long long[2 * (size_t)blocks];
    int rc = BPM_OK;
    auto ck = [&](cudaError_t e, const char* what) {
        if (e != cudaSuccess && rc == BPM_OK) rc = probe_fail(std::string(what) + ": " + cudaGetErrorString(e));
        return rc == BPM_OK;
    };
    if (ck(cudaMalloc(&sink, sizeof(double) * (size_t)blocks * kProbeThreads), "cudaMalloc") &&
        ck(cudaMalloc(&clk, sizeof(unsigned long long) * 2 * (size_t)blocks), "cudaMalloc") &&
        ck(cudaEventCreate(&e0), "cudaEventCreate") && ck(cudaEventCreate(&e1), "cudaEventCreate")) {
        for (int op = 0; op < OP_COUNT && rc == BPM_OK; ++op) {
            ProbeKernel kern = probe_kernel(op);
            // calibrate the iteration count to about 50 ms
            int iters = 1024;
            float ms = 0.f;
            for (int pass = 0; pass < 3 && rc == BPM_OK; ++pass) {
                ck(cudaEventRecord(e0), "cudaEventRecord");
                kern<<<blocks, kProbeThreads>>>(iters, sink, clk);
                ck(cudaGetLastError(), "launch");
                ck(cudaEventRecord(e1), "cudaEventRecord");
                ck(cudaEventSynchronize(e1), "cudaEventSynchronize");
                ck(cudaEventElapsedTime(&ms, e0, e1), "cudaEventElapsedTime");
                if (pass < 2) {
                    const double scale = 50.0 / (ms > 1e-3f ? ms : 1e-3);
                    double next = iters * (scale < 256.0 ? scale : 256.0);
                    if (next > 1e8) next = 1e8;
                    iters = next < 64 ? 64 : (int)next;
                }
            }
            if (rc != BPM_OK) break;
            ck(cudaMemcpy(hclk, clk, sizeof(unsigned long long) * 2 * (size_t)blocks, cudaMemcpyDeviceToHost),
               "cudaMemcpy");
            double cyc = 0.0, ns = 0.0;
            for (int b = 0; b < blocks; ++b) {
                cyc += (double)hclk[2 * b];
                ns += (double)hclk[2 * b + 1];
            }
            const double ghz = ns > 0 ? cyc / ns : 0.0;
            const double lane_ops = (double)blocks * kProbeThreads * kChains * (double)iters * lanes_per_step(op);
            const double per_s = lane_ops / (ms * 1e-3);
            out[4 * op + 0] = (ghz > 0) ? per_s / (n_sm * ghz * 1e9) : 0.0;  // lane operations per SM per clock
            out[4 * op + 1] = per_s;                                          // lane operations per second
            out[4 * op + 2] = ghz * 1e3;                                      // SM clock of the run, MHz
            out[4 * op + 3] = ms;                                             // kernel time, ms
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (sink) cudaFree(sink);
    if (clk) cudaFree(clk);
    delete[] hclk;
    return rc;
}
