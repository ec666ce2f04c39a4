// probe.cu -- pmmf_probe_fp64: the FP64 FMA throughput of the current GPU,
// the denominator of the roofline fraction of the FP64-bound kernels (the
// rotation search, the FP64 Gram).  No counterpart in the paper.
#include <string>

#include "common.cuh"

namespace pmmf {
namespace {

constexpr int PROBE_CHAINS = 8;      // independent dependent-FMA chains per thread
constexpr int PROBE_THREADS = 256;

// Every thread runs PROBE_CHAINS independent chains of `iters` dependent
// fmas (x <- x * a + b), enough independent work per warp to keep the SM's
// FP64 pipe busy.  The result is written only when it equals a value no chain
// reaches, so nothing is stored but the work cannot be removed.
__global__ void __launch_bounds__(PROBE_THREADS) k_probe_fp64(int iters, double a, double b,
                                                              double *sink) {
    double x[PROBE_CHAINS];
#pragma unroll
    for (int c = 0; c < PROBE_CHAINS; ++c) x[c] = (double)(threadIdx.x + c) * 1e-3;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int c = 0; c < PROBE_CHAINS; ++c) x[c] = __fma_rn(x[c], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < PROBE_CHAINS; ++c) s += x[c];
    if (s == -1.0) *sink = s;
}

}  // namespace
}  // namespace pmmf

using namespace pmmf;

extern "C" pmmf_status pmmf_probe_fp64(double *tflops, void *stream) {
    set_error("");
    if (!tflops) {
        set_error("NULL output");
        return PMMF_ERR_INVALID_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    PMMF_CUDA_TRY(cudaGetDevice(&dev));
    PMMF_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    DBuf<double> sink;
    PMMF_TRY(sink.alloc(1, st));
    const int iters = 4096;
    const unsigned blocks = (unsigned)sms * 8u;   // 8 resident CTAs of 256 threads per SM
    // a, b keep every chain finite and away from -1 (|x| stays below 2)
    const double a = 0.5, b = 0.75;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    PMMF_CUDA_TRY(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        set_error("cudaEventCreate failed");
        return PMMF_ERR_CUDA;
    }
    pmmf_status rc = PMMF_OK;
    float best = 0.0f;
    for (int rep = 0; rep < 4 && rc == PMMF_OK; ++rep) {   // the first run warms up
        cudaEventRecord(e0, st);
        k_probe_fp64<<<blocks, PROBE_THREADS, 0, st>>>(iters, a, b, sink.p);
        rc = launched("probe_fp64");
        cudaEventRecord(e1, st);
        if (rc != PMMF_OK) break;
        if (cudaEventSynchronize(e1) != cudaSuccess) {
            set_error("probe: event synchronize failed");
            rc = PMMF_ERR_CUDA;
            break;
        }
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0 && (best == 0.0f || ms < best)) best = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    PMMF_TRY(rc);
    const double flops = 2.0 * PROBE_CHAINS * (double)iters * (double)blocks * PROBE_THREADS;
    *tflops = best > 0.0f ? flops / ((double)best * 1e-3) / 1e12 : 0.0;
    return PMMF_OK;
}
