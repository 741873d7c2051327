// Throughput probes for the roofline denominators (FP32 FMA, instruction
// issue, shared-memory atomics). Each kernel runs a fixed, bounded number of
// iterations per thread and writes a value that depends on every operation so
// that nothing is optimised away.
#include <algorithm>

#include "sbp_internal.cuh"
#include "slingbag_probe.h"

namespace {

constexpr int kProbeThreads = 256;
constexpr int kFmaIters = 4096;
constexpr int kChains = 8;

__global__ void __launch_bounds__(kProbeThreads) probe_fma_kernel(float* out, float a, float b) {
    float v[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) v[c] = (float)(threadIdx.x + c);
#pragma unroll 4
    for (int it = 0; it < kFmaIters; ++it) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) v[c] = fmaf(v[c], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += v[c];
    if (s == 12345.678f) out[blockIdx.x] = s;  // practically never taken
}

// The same chains as packed pairs: one instruction performs two FP32 fused
// multiply-adds on the two halves of a float2.
__global__ void __launch_bounds__(kProbeThreads) probe_fma2_kernel(float* out, float a, float b) {
    float2 v[kChains / 2];
#pragma unroll
    for (int c = 0; c < kChains / 2; ++c)
        v[c] = make_float2((float)(threadIdx.x + 2 * c), (float)(threadIdx.x + 2 * c + 1));
    const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
#pragma unroll 4
    for (int it = 0; it < kFmaIters; ++it) {
#pragma unroll
        for (int c = 0; c < kChains / 2; ++c) v[c] = __ffma2_rn(v[c], a2, b2);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains / 2; ++c) s += v[c].x + v[c].y;
    if (s == 12345.678f) out[blockIdx.x] = s;  // practically never taken
}

__global__ void __launch_bounds__(kProbeThreads) probe_issue_kernel(unsigned* out, unsigned a) {
    unsigned v[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) v[c] = threadIdx.x * (c + 1);
#pragma unroll 4
    for (int it = 0; it < kFmaIters; ++it) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) v[c] = (v[c] ^ a) + (unsigned)c;
    }
    unsigned s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += v[c];
    if (s == 0x9e3779b9u) out[blockIdx.x] = s;
}

constexpr int kAtomIters = 1024;
constexpr int kAtomRows = 64;  // distinct words per lane

template <typename T>
__global__ void __launch_bounds__(kProbeThreads) probe_smem_atomic_kernel(T* out) {
    __shared__ T buf[kAtomRows * 32];
    for (int t = threadIdx.x; t < kAtomRows * 32; t += blockDim.x) buf[t] = T(0);
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // lane l always hits column l (its own bank for 32-bit words); rows rotate
    for (int it = 0; it < kAtomIters; ++it) {
        const int row = (it * 7 + warp * 13) & (kAtomRows - 1);
        atomicAdd(&buf[row * 32 + lane], T(1));
    }
    __syncthreads();
    if (threadIdx.x == 0) out[blockIdx.x] = buf[lane];
}

int time_launch(void (*launch)(cudaStream_t), double* ms_out) {
    cudaStream_t s;
    cudaEvent_t a, b;
    if (sbp_cuda_check(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking), "probe: stream"))
        return SBP_ERR_CUDA;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    launch(s);  // warm-up
    cudaEventRecord(a, s);
    for (int r = 0; r < 3; ++r) launch(s);
    cudaEventRecord(b, s);
    const cudaError_t e = cudaEventSynchronize(b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaStreamDestroy(s);
    if (sbp_cuda_check(e, "probe: kernel") || sbp_cuda_check(cudaGetLastError(), "probe: launch"))
        return SBP_ERR_CUDA;
    *ms_out = ms / 3.0;
    return SBP_OK;
}

int g_blocks = 0;
void* g_out = nullptr;

int probe_setup() {
    int dev = 0, sms = 0;
    if (sbp_cuda_check(cudaGetDevice(&dev), "probe: device")) return SBP_ERR_CUDA;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    g_blocks = std::max(1, sms) * 8;
    if (!g_out && sbp_cuda_check(cudaMalloc(&g_out, sizeof(double) * g_blocks * 4), "probe: alloc"))
        return SBP_ERR_CUDA;
    return SBP_OK;
}

}  // namespace

extern "C" int sbp_probe_fp32_fma(double* fma_per_s) {
    if (!fma_per_s) {
        sbp_set_error("probe_fp32_fma: null pointer");
        return SBP_ERR_ARG;
    }
    if (int e = probe_setup()) return e;
    double ms = 0;
    if (int e = time_launch(
            [](cudaStream_t s) {
                probe_fma_kernel<<<g_blocks, kProbeThreads, 0, s>>>((float*)g_out, 0.999f, 1e-3f);
            },
            &ms))
        return e;
    sbp_count_launches(4);
    *fma_per_s = (double)g_blocks * kProbeThreads * kFmaIters * kChains / (ms * 1e-3);
    return SBP_OK;
}

extern "C" int sbp_probe_fp32x2_fma(double* fma_per_s) {
    if (!fma_per_s) {
        sbp_set_error("probe_fp32x2_fma: null pointer");
        return SBP_ERR_ARG;
    }
    if (int e = probe_setup()) return e;
    double ms = 0;
    if (int e = time_launch(
            [](cudaStream_t s) {
                probe_fma2_kernel<<<g_blocks, kProbeThreads, 0, s>>>((float*)g_out, 0.999f, 1e-3f);
            },
            &ms))
        return e;
    sbp_count_launches(4);
    // kChains / 2 packed instructions per iteration, two FMAs each
    *fma_per_s = (double)g_blocks * kProbeThreads * kFmaIters * kChains / (ms * 1e-3);
    return SBP_OK;
}

extern "C" int sbp_probe_issue(double* warp_inst_per_s) {
    if (!warp_inst_per_s) {
        sbp_set_error("probe_issue: null pointer");
        return SBP_ERR_ARG;
    }
    if (int e = probe_setup()) return e;
    double ms = 0;
    if (int e = time_launch(
            [](cudaStream_t s) {
                probe_issue_kernel<<<g_blocks, kProbeThreads, 0, s>>>((unsigned*)g_out, 0x5bd1e995u);
            },
            &ms))
        return e;
    sbp_count_launches(4);
    // two dependent integer operations per chain and iteration
    *warp_inst_per_s =
        (double)g_blocks * (kProbeThreads / 32) * kFmaIters * kChains * 2 / (ms * 1e-3);
    return SBP_OK;
}

extern "C" int sbp_probe_smem_atomic(int kind, double* atomics_per_s) {
    if (!atomics_per_s || kind < 0 || kind > 2) {
        sbp_set_error("probe_smem_atomic: null pointer or unknown kind");
        return SBP_ERR_ARG;
    }
    if (int e = probe_setup()) return e;
    double ms = 0;
    int e = SBP_OK;
    if (kind == 0)
        e = time_launch(
            [](cudaStream_t s) {
                probe_smem_atomic_kernel<unsigned><<<g_blocks, kProbeThreads, 0, s>>>((unsigned*)g_out);
            },
            &ms);
    else if (kind == 1)
        e = time_launch(
            [](cudaStream_t s) {
                probe_smem_atomic_kernel<unsigned long long>
                    <<<g_blocks, kProbeThreads, 0, s>>>((unsigned long long*)g_out);
            },
            &ms);
    else
        e = time_launch(
            [](cudaStream_t s) {
                probe_smem_atomic_kernel<float><<<g_blocks, kProbeThreads, 0, s>>>((float*)g_out);
            },
            &ms);
    if (e) return e;
    sbp_count_launches(4);
    *atomics_per_s = (double)g_blocks * kProbeThreads * kAtomIters / (ms * 1e-3);
    return SBP_OK;
}
