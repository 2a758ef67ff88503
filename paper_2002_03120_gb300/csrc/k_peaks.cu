// k_peaks.cu -- throughput of the three arithmetic pipes the pair kernels
// run on, measured on the GPU at hand: FP32 fused multiply-add, FP64 fused
// multiply-add and 32-bit integer multiply-add (the multiply of the Philox
// rounds).  These are the denominators of the pair kernels' rooflines, which
// are bound by arithmetic issue, not by memory.
//
// Each kernel keeps ILP independent dependency chains per thread in
// registers (no memory traffic in the loop) on a grid of several resident
// blocks per SM, so the pipe, not latency, sets the time; the chains'
// results are folded into one store that the compiler cannot drop.  The rate
// is taken from CUDA events around a launch long enough (tens of ms) that
// launch overhead does not matter, at whatever clock the GPU runs.
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace sdpd {

constexpr int PK_ILP = 8;
constexpr int PK_THREADS = 256;

__global__ void __launch_bounds__(PK_THREADS) k_peak_ffma(float *out, int iters, float a, float b)
{
    float x[PK_ILP];
#pragma unroll
    for (int k = 0; k < PK_ILP; ++k) x[k] = (float)(threadIdx.x + k) * 1e-3f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 8; ++u)
#pragma unroll
            for (int k = 0; k < PK_ILP; ++k) x[k] = __fmaf_rn(x[k], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < PK_ILP; ++k) s += x[k];
    if (s == 1234.5f) out[blockIdx.x] = s;   // never true for the inputs used; keeps the work
}

__global__ void __launch_bounds__(PK_THREADS) k_peak_dfma(double *out, int iters, double a, double b)
{
    double x[PK_ILP];
#pragma unroll
    for (int k = 0; k < PK_ILP; ++k) x[k] = (double)(threadIdx.x + k) * 1e-3;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 8; ++u)
#pragma unroll
            for (int k = 0; k < PK_ILP; ++k) x[k] = __fma_rn(x[k], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < PK_ILP; ++k) s += x[k];
    if (s == 1234.5) out[blockIdx.x] = s;
}

__global__ void __launch_bounds__(PK_THREADS) k_peak_imad(uint32_t *out, int iters, uint32_t a, uint32_t b)
{
    uint32_t x[PK_ILP];
#pragma unroll
    for (int k = 0; k < PK_ILP; ++k) x[k] = threadIdx.x * 7919u + (uint32_t)k;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 8; ++u)
#pragma unroll
            for (int k = 0; k < PK_ILP; ++k) x[k] = x[k] * x[k] + b;   // not affine: no closed form
    }
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < PK_ILP; ++k) s ^= x[k];
    if (s == a) out[blockIdx.x] = s;   // the stored value is irrelevant; keeps the work
}

}  // namespace sdpd

namespace {

// Operations per second of one launch: lanes x chains x 8 x iters FMAs
// (two operations each for the floating-point pipes, one for IMAD).
template <class Launch>
double time_rate(Launch launch, double ops, cudaEvent_t e0, cudaEvent_t e1, sdpd_status &st)
{
    launch();   // warm-up (clocks up, code loaded)
    if (cudaEventRecord(e0, 0) != cudaSuccess) st = SDPD_E_CUDA;
    launch();
    if (cudaEventRecord(e1, 0) != cudaSuccess) st = SDPD_E_CUDA;
    if (cudaEventSynchronize(e1) != cudaSuccess) { st = SDPD_E_CUDA; return 0.0; }
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess || ms <= 0.f) { st = SDPD_E_CUDA; return 0.0; }
    return ops / (ms * 1e-3);
}

}  // namespace

extern "C" sdpd_status sdpd_alu_peaks(double *out)
{
    using namespace sdpd;
    if (!out) {
        set_last_error("sdpd_alu_peaks: NULL output");
        return SDPD_E_INVALID;
    }
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        set_last_error("sdpd_alu_peaks: no CUDA device");
        return SDPD_E_CUDA;
    }
    (void)cudaGetLastError();
    const int blocks = nsm * 8;   // 2048 threads per SM: full occupancy at <= 32 registers
    void *buf = nullptr;
    if (cudaMalloc(&buf, (size_t)blocks * sizeof(double)) != cudaSuccess) {
        set_last_error("sdpd_alu_peaks: cudaMalloc");
        return SDPD_E_OOM;
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    sdpd_status st = SDPD_OK;
    const double lanes = (double)blocks * PK_THREADS * PK_ILP * 8.0;
    // iteration counts sized for some tens of ms per launch at the nominal
    // rates (FP64 is a small fraction of FP32 on this part)
    const int it32 = 20000, it64 = 400, iti = 10000;
    const double ffma = time_rate([&] { k_peak_ffma<<<blocks, PK_THREADS>>>((float *)buf, it32, 0.999999f, 1e-7f); },
                                  lanes * it32 * 2.0, e0, e1, st);
    const double dfma = time_rate([&] { k_peak_dfma<<<blocks, PK_THREADS>>>((double *)buf, it64, 0.999999, 1e-9); },
                                  lanes * it64 * 2.0, e0, e1, st);
    const double imad = time_rate([&] { k_peak_imad<<<blocks, PK_THREADS>>>((uint32_t *)buf, iti, 1664525u, 1013904223u); },
                                  lanes * iti, e0, e1, st);
    if (cudaGetLastError() != cudaSuccess) st = SDPD_E_CUDA;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(buf);
    if (st != SDPD_OK) {
        set_last_error("sdpd_alu_peaks: a timing launch failed");
        return st;
    }
    out[0] = ffma / 1e12;   // FP32 TFLOP/s (FMA = 2 flops)
    out[1] = dfma / 1e12;   // FP64 TFLOP/s
    out[2] = imad / 1e12;   // INT32 multiply-adds, tera-operations/s (one per IMAD)
    out[3] = (double)nsm;
    return SDPD_OK;
}
