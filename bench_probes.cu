// bench_probes.cu -- throughput probes of the plain arithmetic pipes and of
// device memory, used by bench.py as context for the roofline denominators of
// kernels bound by FP32/integer issue, the special-function unit or HBM (none
// of the force step is tensor-core work).  Built by bench.py into its own
// shared object; not part of librbe.so.  Each probe runs independent
// dependency chains in every thread of a grid that fills the GPU, so the
// pipe, not latency, limits it; the result is the best of three timed
// launches after one warm-up (CUDA events on the caller's stream).
#include <cuda_runtime.h>

#define PROBE_FFMA 0
#define PROBE_DFMA 1
#define PROBE_SFU  2
#define PROBE_ALU  3
#define PROBE_COPY 4
#define PROBE_OK      0
#define PROBE_EINVAL -1
#define PROBE_ECUDA  -6
#define PROBE_ENOMEM -7

namespace {

constexpr int PB_THREADS = 256;
constexpr int PB_CHAINS = 8;

// Sinks keep the chains alive: the store happens only for a value the inputs
// never produce, but the compiler cannot know that.
__global__ void __launch_bounds__(PB_THREADS) k_probe_ffma(int iters, float x0, float* sink)
{
    float a[PB_CHAINS];
#pragma unroll
    for (int c = 0; c < PB_CHAINS; ++c) a[c] = x0 + 1e-7f * (float)(threadIdx.x + c);
    for (int t = 0; t < iters; ++t) {
#pragma unroll
        for (int c = 0; c < PB_CHAINS; ++c) a[c] = fmaf(a[c], 0.99999994f, 1e-8f);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < PB_CHAINS; ++c) s += a[c];
    if (s == -1.2345f) sink[blockIdx.x] = s;
}

__global__ void __launch_bounds__(PB_THREADS) k_probe_dfma(int iters, double x0, double* sink)
{
    double a[PB_CHAINS];
#pragma unroll
    for (int c = 0; c < PB_CHAINS; ++c) a[c] = x0 + 1e-9 * (double)(threadIdx.x + c);
    for (int t = 0; t < iters; ++t) {
#pragma unroll
        for (int c = 0; c < PB_CHAINS; ++c) a[c] = fma(a[c], 0.9999999999, 1e-12);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < PB_CHAINS; ++c) s += a[c];
    if (s == -1.2345) sink[blockIdx.x] = s;
}

// One __sinf per chain step: the hardware sine of the special-function unit
// (the FP32 sincos of the mixed Fourier kernels issues two such operations).
__global__ void __launch_bounds__(PB_THREADS) k_probe_sfu(int iters, float x0, float* sink)
{
    float a[PB_CHAINS];
#pragma unroll
    for (int c = 0; c < PB_CHAINS; ++c) a[c] = x0 + 1e-3f * (float)(threadIdx.x + c);
    for (int t = 0; t < iters; ++t) {
#pragma unroll
        for (int c = 0; c < PB_CHAINS; ++c) a[c] = __sinf(a[c]) + 0.5f;
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < PB_CHAINS; ++c) s += a[c];
    if (s == -1.2345f) sink[blockIdx.x] = s;
}

// Integer add/xor/shift chains (the compare, select and bit operations of the
// list classification issue on the same integer pipe).
__global__ void __launch_bounds__(PB_THREADS) k_probe_alu(int iters, unsigned x0, unsigned* sink)
{
    unsigned a[PB_CHAINS];
#pragma unroll
    for (int c = 0; c < PB_CHAINS; ++c) a[c] = x0 + threadIdx.x * 2654435761u + c;
    for (int t = 0; t < iters; ++t) {
#pragma unroll
        for (int c = 0; c < PB_CHAINS; ++c) a[c] = (a[c] ^ (a[c] >> 3)) + 0x9e3779b9u;
    }
    unsigned s = 0;
#pragma unroll
    for (int c = 0; c < PB_CHAINS; ++c) s ^= a[c];
    if (s == 0x12345678u) sink[blockIdx.x] = s;
}

// Device-to-device copy of n float4 (read + write bytes counted).
__global__ void __launch_bounds__(PB_THREADS) k_probe_copy(long n, const float4* __restrict__ src,
                                                            float4* __restrict__ dst)
{
    for (long i = (long)blockIdx.x * PB_THREADS + threadIdx.x; i < n; i += (long)gridDim.x * PB_THREADS)
        dst[i] = src[i];
}

}  // namespace

// kind: PROBE_FFMA (FP32 fused multiply-adds per second, one per lane),
// PROBE_DFMA (FP64 fused multiply-adds per second), PROBE_SFU (hardware sines
// per second), PROBE_ALU (32-bit integer shift/xor/add operations per second),
// PROBE_COPY (device-to-device copy, bytes read + written per second, 2 GiB
// per launch).  Best of three timed launches after a warm-up on cuda_stream
// (the call waits).  Allocates and frees a small sink, and 2 GiB for the copy.
extern "C" int bench_peak_probe(int kind, double* ops_per_s, void* cuda_stream)
{
    if (!ops_per_s || kind < PROBE_FFMA || kind > PROBE_COPY) return PROBE_EINVAL;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return PROBE_ECUDA;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return PROBE_ECUDA;
    const int blocks = nsm * 8;
    const double threads = (double)blocks * PB_THREADS;
    void* sink = nullptr;
    void* buf = nullptr;
    const long ncopy = 64L << 20;   // float4 elements: 1 GiB read + 1 GiB written
    if (cudaMalloc(&sink, sizeof(double) * blocks) != cudaSuccess) return PROBE_ENOMEM;
    if (kind == PROBE_COPY && cudaMalloc(&buf, sizeof(float4) * 2 * (size_t)ncopy) != cudaSuccess) {
        cudaFree(sink);
        return PROBE_ENOMEM;
    }
    int iters = 0;
    double ops = 0.0;
    switch (kind) {
        case PROBE_FFMA: iters = 16384; ops = threads * iters * PB_CHAINS; break;
        case PROBE_DFMA: iters = 512; ops = threads * iters * PB_CHAINS; break;
        case PROBE_SFU: iters = 4096; ops = threads * iters * PB_CHAINS; break;
        case PROBE_ALU: iters = 8192; ops = threads * iters * PB_CHAINS * 3.0; break;  // shift, xor, add
        default: ops = 2.0 * sizeof(float4) * (double)ncopy; break;
    }
    auto launch = [&]() {
        switch (kind) {
            case PROBE_FFMA: k_probe_ffma<<<blocks, PB_THREADS, 0, st>>>(iters, 1.0f, (float*)sink); break;
            case PROBE_DFMA: k_probe_dfma<<<blocks, PB_THREADS, 0, st>>>(iters, 1.0, (double*)sink); break;
            case PROBE_SFU: k_probe_sfu<<<blocks, PB_THREADS, 0, st>>>(iters, 0.25f, (float*)sink); break;
            case PROBE_ALU: k_probe_alu<<<blocks, PB_THREADS, 0, st>>>(iters, 7u, (unsigned*)sink); break;
            default:
                k_probe_copy<<<blocks, PB_THREADS, 0, st>>>(ncopy, (const float4*)buf, (float4*)buf + ncopy);
                break;
        }
    };
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    launch();
    float best = 1e30f;
    for (int r = 0; r < 3; ++r) {
        cudaEventRecord(e0, st);
        launch();
        cudaEventRecord(e1, st);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        best = ms < best ? ms : best;
    }
    cudaError_t e = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sink);
    if (buf) cudaFree(buf);
    if (e != cudaSuccess || !(best > 0.f)) return PROBE_ECUDA;
    *ops_per_s = ops / (best * 1e-3);
    return PROBE_OK;
}
