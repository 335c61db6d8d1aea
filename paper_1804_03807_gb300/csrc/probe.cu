// probe.cu -- the FP64 issue rate of the GPU the library runs on.  The
// trackers are bound by double precision arithmetic; their roofline divides
// by a peak derived from the FP64 units and the clock, and this probe
// measures the same peak on the device: independent fused multiply-add
// chains in every thread of a grid that fills every SM.
#include "phc_internal.h"

namespace phc {

int set_error(int code, const char *msg);  // phc_api.cpp

namespace {

constexpr int PROBE_CHAINS = 8;  // independent chains per thread (hides the FMA latency)

__device__ double g_probe_sink;

__global__ void fp64_chains(int64_t iters)
{
    double a[PROBE_CHAINS];
#pragma unroll
    for (int c = 0; c < PROBE_CHAINS; c++) a[c] = 1e-3 * (threadIdx.x + c);
    const double m = 0.99999999, e = 1e-12;
    for (int64_t k = 0; k < iters; k++) {
#pragma unroll
        for (int c = 0; c < PROBE_CHAINS; c++) a[c] = fma(a[c], m, e);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < PROBE_CHAINS; c++) s += a[c];
    if (s == -1.0) g_probe_sink = s;  // never true (the chains stay positive); keeps them live
}

}  // namespace
}  // namespace phc

extern "C" int phc_fp64_probe(int warps_per_block, int64_t iters, double *tflops_out, void *stream)
{
    if (!tflops_out) return phc::set_error(PHC_EINVAL, "phc_fp64_probe: tflops_out is NULL");
    *tflops_out = 0.0;
    if (warps_per_block < 1 || warps_per_block > 32)
        return phc::set_error(PHC_EINVAL, "phc_fp64_probe: warps_per_block outside 1..32");
    if (iters < 1 || iters > 100000000) return phc::set_error(PHC_EINVAL, "phc_fp64_probe: iters outside 1..1e8");
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return phc::set_error(PHC_ECUDA, "phc_fp64_probe: device query failed");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return phc::set_error(PHC_ECUDA, "phc_fp64_probe: cudaEventCreate failed");
    }
    const int blocks = 2 * sms, threads = 32 * warps_per_block;
    cudaEventRecord(e0, s);
    phc::fp64_chains<<<blocks, threads, 0, s>>>(iters);
    cudaError_t err = cudaGetLastError();
    cudaEventRecord(e1, s);
    if (err == cudaSuccess) err = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (err != cudaSuccess) return phc::set_error(PHC_ECUDA, cudaGetErrorString(err));
    const double flops = 2.0 * phc::PROBE_CHAINS * (double)iters * threads * blocks;
    *tflops_out = ms > 0.0f ? flops / (ms * 1e-3) / 1e12 : 0.0;
    return PHC_OK;
}
