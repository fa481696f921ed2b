// measure.cu -- rates of the device's FP64 units, the denominators of the plain FP64 path's
// roofline (GB300 has no FP64 rate of its own in the measured peaks beside the HBM copy and the
// bf16 tensor rate).  Each thread runs eight independent dependency chains so that the pipeline,
// not the latency of one chain, sets the rate.
#include "runtime.h"

namespace npb {

__global__ void k_fp64_fma(double *out, int iters, double a, double b) {
    double x[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) x[j] = 1e-3 * (threadIdx.x + j);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < 8; ++j) x[j] = fma(x[j], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < 8; ++j) s += x[j];
    if (s == -1.0) out[0] = s;  // never true (x stays near b/(1-a) > 0): keeps the chains live
}

__global__ void k_fp64_div(double *out, int iters, double b) {
    double x[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) x[j] = 1.5 + 1e-3 * (threadIdx.x + j);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < 8; ++j) x[j] = b / x[j] + 0.5;  // stays in [1.5, 2]
    }
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < 8; ++j) s += x[j];
    if (s == -1.0) out[0] = s;
}

}  // namespace npb

using namespace npb;

extern "C" int npb_measure_fp64(npb_ctx *ctx, double *dfma_per_s, double *ddiv_per_s) {
    if (!ctx || !dfma_per_s || !ddiv_per_s) return fail(NPB_EINVAL, "NULL argument");
    CU(cudaSetDevice(ctx->device));
    cudaStream_t st = ctx->stream;
    void *buf = nullptr;
    int rc = ctx->alloc(&buf, 64);
    if (rc) return rc;
    const int blocks = ctx->sm_count * 8, threads = 256;
    const int it_fma = 4096, it_div = 256;
    cudaEvent_t a, b;
    cudaError_t e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    float ms_fma = 0.f, ms_div = 0.f;
    for (int pass = 0; pass < 2 && e == cudaSuccess; ++pass) {  // the first pass warms the clocks up
        k_fp64_fma<<<blocks, threads, 0, st>>>((double *)buf, it_fma, 0.999, 1e-3);
        e = cudaEventRecord(a, st);
        if (e == cudaSuccess) k_fp64_fma<<<blocks, threads, 0, st>>>((double *)buf, it_fma, 0.999, 1e-3);
        if (e == cudaSuccess) e = cudaEventRecord(b, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(b);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms_fma, a, b);
        if (e == cudaSuccess) e = cudaEventRecord(a, st);
        if (e == cudaSuccess) k_fp64_div<<<blocks, threads, 0, st>>>((double *)buf, it_div, 0.75);
        if (e == cudaSuccess) e = cudaEventRecord(b, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(b);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms_div, a, b);
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaStreamSynchronize(st);
    ctx->release(buf, 64);
    if (e != cudaSuccess) return fail(NPB_ECUDA, "FP64 rate measurement failed: %s", cudaGetErrorString(e));
    const double n = (double)blocks * threads * 8;
    *dfma_per_s = n * it_fma / (ms_fma * 1e-3);
    *ddiv_per_s = n * it_div / (ms_div * 1e-3);
    return NPB_OK;
}
