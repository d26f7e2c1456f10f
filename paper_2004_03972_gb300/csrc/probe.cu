// probe.cu -- bandwidth microbenchmarks for the rooflines: shared memory (the
// resident sparse and batch MD kernels gather from it) and L2 (the streaming
// sparse kernel gathers from it).
//
// Every CTA fills 32 KB of shared memory, then each thread streams 128-bit
// ld.shared loads over it: thread t reads the 16-byte word (t + 32 i) mod 2048
// at iteration i, so a warp's request covers 512 consecutive bytes (four
// conflict-free wavefronts), the loads of one thread are independent of each
// other, and no two loads of a thread within 64 iterations read the same word
// (the assembler may merge repeated loads of one address).  The loaded values
// are summed into a per-thread accumulator that is written out, so no load
// can be dropped.
// Two CTAs of 1024 threads per SM keep the load pipe busy.
#include <algorithm>

#include "hqa_internal.cuh"

namespace {

constexpr int kProbeThreads = 1024;
constexpr int kProbeWords = 2048;   // 16-byte words: 32 KB

__global__ void __launch_bounds__(kProbeThreads, 2) k_smem_probe(int iters, float* sink)
{
    __shared__ __align__(16) float4 buf[kProbeWords];
    for (int i = threadIdx.x; i < kProbeWords; i += blockDim.x)
        buf[i] = make_float4((float)i, 1.f, 2.f, 3.f);
    __syncthreads();
    const uint32_t base = (uint32_t)__cvta_generic_to_shared(buf);
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    const uint32_t t = threadIdx.x;
#pragma unroll 8
    for (int it = 0; it < iters; ++it) {
        const uint32_t w = (t + 32u * (uint32_t)it) & (kProbeWords - 1);
        float4 v;
        asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                     : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(base + 16u * w));
        acc.x += v.x;
        acc.y += v.y;
        acc.z += v.z;
        acc.w += v.w;
    }
    sink[blockIdx.x * blockDim.x + t] = acc.x + acc.y + acc.z + acc.w;
}

// L2 probe: every thread reads 16-byte words of an L2-resident buffer with
// ld.global.cg (no L1), a grid-stride pass at a time, and sums them.
__global__ void __launch_bounds__(kProbeThreads, 2) k_l2_probe(const float4* buf, size_t words,
                                                              int passes, float* sink)
{
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (int ps = 0; ps < passes; ++ps)
        for (size_t w = blockIdx.x * (size_t)blockDim.x + threadIdx.x; w < words; w += stride) {
            const float4 v = __ldcg(buf + w);
            acc.x += v.x;
            acc.y += v.y;
            acc.z += v.z;
            acc.w += v.w;
        }
    sink[blockIdx.x * blockDim.x + threadIdx.x] = acc.x + acc.y + acc.z + acc.w;
}

}  // namespace

extern "C" hqa_status hqa_probe_l2_bandwidth(double* gbps, void* stream)
{
    if (!gbps) return HQA_ERR_INVALID_ARG;
    if (hqa_capturing()) return hqa_capture_note(HQA_ERR_UNSUPPORTED);
    int dev = 0, sms = 0, l2 = 0;
    HQA_CUDA_TRY(cudaGetDevice(&dev));
    HQA_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    HQA_CUDA_TRY(cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev));
    // a buffer of half the L2 (64 MB on GB300): resident after the first pass
    const size_t bytes = std::max<size_t>((size_t)l2 / 2, (size_t)1 << 20) & ~(size_t)255;
    const size_t words = bytes / 16;
    const int blocks = 2 * sms;
    void* buf = nullptr;
    float* sink = nullptr;
    HQA_CUDA_TRY(cudaMalloc(&buf, bytes));
    if (cudaMalloc(&sink, (size_t)blocks * kProbeThreads * sizeof(float)) != cudaSuccess) {
        cudaFree(buf);
        (void)cudaGetLastError();
        return HQA_ERR_OOM;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    hqa_status s = HQA_OK;
    if (cudaMemsetAsync(buf, 0, bytes, st) != cudaSuccess) s = HQA_ERR_CUDA;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (s == HQA_OK && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess))
        s = HQA_ERR_CUDA;
    const int passes = 40;
    double best = 0.0;
    for (int rep = 0; rep < 4 && s == HQA_OK; ++rep) {
        cudaEventRecord(e0, st);
        k_l2_probe<<<blocks, kProbeThreads, 0, st>>>(static_cast<const float4*>(buf), words,
                                                     passes, sink);
        cudaEventRecord(e1, st);
        if (cudaEventSynchronize(e1) != cudaSuccess) {
            s = HQA_ERR_CUDA;
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0) best = std::max(best, (double)bytes * passes / (ms * 1e-3) / 1e9);
    }
    if (cudaGetLastError() != cudaSuccess) s = HQA_ERR_CUDA;
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(buf);
    cudaFree(sink);
    if (s == HQA_OK) *gbps = best;
    return s;
}

extern "C" hqa_status hqa_probe_smem_bandwidth(double* gbps, void* stream)
{
    if (!gbps) return HQA_ERR_INVALID_ARG;
    if (hqa_capturing()) return hqa_capture_note(HQA_ERR_UNSUPPORTED);
    int dev = 0, sms = 0;
    HQA_CUDA_TRY(cudaGetDevice(&dev));
    HQA_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int blocks = 2 * sms;
    const int iters = 16384;
    float* sink = nullptr;
    HQA_CUDA_TRY(cudaMalloc(&sink, (size_t)blocks * kProbeThreads * sizeof(float)));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    hqa_status s = HQA_OK;
    double best = 0.0;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) s = HQA_ERR_CUDA;
    for (int rep = 0; rep < 4 && s == HQA_OK; ++rep) {
        cudaEventRecord(e0, st);
        k_smem_probe<<<blocks, kProbeThreads, 0, st>>>(iters, sink);
        cudaEventRecord(e1, st);
        if (cudaEventSynchronize(e1) != cudaSuccess) {
            s = HQA_ERR_CUDA;
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        const double bytes = (double)blocks * kProbeThreads * (double)iters * 16.0;
        if (rep > 0) best = std::max(best, bytes / (ms * 1e-3) / 1e9);   // first run: warm-up
    }
    if (cudaGetLastError() != cudaSuccess) s = HQA_ERR_CUDA;
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(sink);
    if (s == HQA_OK) *gbps = best;
    return s;
}
