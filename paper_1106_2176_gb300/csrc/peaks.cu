// Measured arithmetic peaks of the current GPU: the denominators of the
// roofline fractions of the P2P kernel (FP32 FMA on the CUDA cores) and of the
// tensor-core M2L (tcgen05.mma kind::tf32). The paper has no counterpart;
// this is measurement infrastructure (fmm_measure_peak in include/fmm.h).
//
// FP32: every thread runs 8 independent FMA chains (scalar fma.rn.ftz.f32, or
// packed fma.rn.ftz.f32x2 on register pairs, 4 flop per instruction) at full
// occupancy, so the FMA pipe, not latency, sets the rate.
// TF32: one CTA per SM, one thread issuing 128 x N x 8 MMAs back to back from
// two fixed shared-memory operands (128B-swizzled, K-major) into one tensor-
// memory accumulator; one commit at the end, waited for with a bound.
#include <algorithm>

#include "fmm_internal.cuh"
#include "ptx_sm100.cuh"

namespace fmm {

constexpr int PEAK_CHAINS = 8;
constexpr int PEAK_FMA_THREADS = 256;

__global__ void __launch_bounds__(PEAK_FMA_THREADS) peak_fma_k(int iters, float b, float c, float *sink)
{
    float a[PEAK_CHAINS];
#pragma unroll
    for (int i = 0; i < PEAK_CHAINS; i++) a[i] = (float)(threadIdx.x + i) * 1e-3f;
    for (int it = 0; it < iters; it++) {
#pragma unroll
        for (int i = 0; i < PEAK_CHAINS; i++) asm volatile("fma.rn.ftz.f32 %0, %0, %1, %2;" : "+f"(a[i]) : "f"(b), "f"(c));
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < PEAK_CHAINS; i++) s += a[i];
    if (s == -1.0f) sink[blockIdx.x] = s;  // never true; keeps the chains live
}

__global__ void __launch_bounds__(PEAK_FMA_THREADS) peak_fma2_k(int iters, float b, float c, float *sink)
{
    uint64_t a[PEAK_CHAINS];
    uint64_t bb, cc;
    asm("mov.b64 %0, {%1, %1};" : "=l"(bb) : "f"(b));
    asm("mov.b64 %0, {%1, %1};" : "=l"(cc) : "f"(c));
#pragma unroll
    for (int i = 0; i < PEAK_CHAINS; i++) {
        const float lo = (float)(threadIdx.x + i) * 1e-3f, hi = lo + 0.5f;
        asm("mov.b64 %0, {%1, %2};" : "=l"(a[i]) : "f"(lo), "f"(hi));
    }
    for (int it = 0; it < iters; it++) {
#pragma unroll
        for (int i = 0; i < PEAK_CHAINS; i++) asm volatile("fma.rn.ftz.f32x2 %0, %0, %1, %2;" : "+l"(a[i]) : "l"(bb), "l"(cc));
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < PEAK_CHAINS; i++) {
        float lo, hi;
        asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(a[i]));
        s += lo + hi;
    }
    if (s == -1.0f) sink[blockIdx.x] = s;
}

// shared memory: A 128 rows x 128 B, B up to 256 rows x 128 B, the mbarrier
// and the TMEM address; padded so that one CTA fills an SM
constexpr int PEAK_TC_A = 128 * 128, PEAK_TC_B = 256 * 128;
constexpr int PEAK_TC_SMEM = 160 * 1024;

__global__ void __launch_bounds__(128, 1) peak_tf32_k(int iters, int N, int *err)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *base = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    unsigned char *A = base, *B = base + PEAK_TC_A;
    uint64_t *bar = reinterpret_cast<uint64_t *>(B + PEAK_TC_B);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bar + 1);
    const int tid = threadIdx.x;
    // small nonzero operands (the contents do not change the MMA's rate, but
    // zero operands would understate its power draw)
    for (int i = tid; i < (PEAK_TC_A + PEAK_TC_B) / 4; i += blockDim.x)
        reinterpret_cast<float *>(A)[i] = (float)((i * 2654435761u) >> 22) * (1.0f / 1024.0f) - 0.5f;
    if (tid == 0) {
        mbar_init(bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    fence_proxy_async();
    if (tid < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(256));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    if (tid == 0) {
        const uint32_t id = idesc_tf32(128, N);
        const uint32_t a0 = smem_u32(A), b0 = smem_u32(B);
        for (int it = 0; it < iters; it++) {
#pragma unroll
            for (int k = 0; k < 4; k++)
                mma_tf32(tmem, sdesc(a0 + 32 * k), sdesc(b0 + 32 * k), id, (it | k) ? 1u : 0u);
        }
        mma_commit(bar);
        if (!mbar_wait(bar, 0)) atomicExch(err, 1);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (tid < 32) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(256));
}

}  // namespace fmm

extern "C" FMM_API int fmm_measure_peak(int kind, int param, int reps, double *tflops)
{
    using namespace fmm;
    if (!tflops) {
        set_error("fmm_measure_peak: NULL output");
        return FMM_EINVAL;
    }
    if (kind < FMM_PEAK_FP32_FMA || kind > FMM_PEAK_TF32_MMA || reps < 1 || reps > 100) {
        set_error("fmm_measure_peak: unknown kind or reps outside [1, 100]");
        return FMM_EINVAL;
    }
    if (kind == FMM_PEAK_TF32_MMA && param != 128 && param != 256) {
        set_error("fmm_measure_peak: the TF32 MMA width must be 128 or 256");
        return FMM_EINVAL;
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    float *sink = nullptr;
    int *err = nullptr;
    try {
        int dev = 0, nsm = 0, major = 0;
        FMM_CUDA_TRY(cudaGetDevice(&dev));
        FMM_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
        FMM_CUDA_TRY(cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev));
        if (major != 10) throw Error{FMM_ENODEV, "fmm_measure_peak: the library is built for sm_103 (Blackwell) only"};
        FMM_CUDA_TRY(cudaEventCreate(&e0));
        FMM_CUDA_TRY(cudaEventCreate(&e1));
        FMM_CUDA_TRY(cudaMalloc(&sink, sizeof(float) * 65536));
        FMM_CUDA_TRY(cudaMalloc(&err, sizeof(int)));
        FMM_CUDA_TRY(cudaMemset(err, 0, sizeof(int)));
        double flops = 0;
        auto launch = [&]() {
            if (kind == FMM_PEAK_TF32_MMA) {
                const int iters = 32768;
                ensure_smem((const void *)peak_tf32_k, PEAK_TC_SMEM);
                peak_tf32_k<<<nsm, 128, PEAK_TC_SMEM>>>(iters, param, err);
                flops = 2.0 * 128 * param * 8 * 4 * (double)iters * nsm;
            } else {
                const int blocks = nsm * (2048 / PEAK_FMA_THREADS), iters = 1 << 18;
                if (kind == FMM_PEAK_FP32_FMA) {
                    peak_fma_k<<<blocks, PEAK_FMA_THREADS>>>(iters, 0.999f, 1e-3f, sink);
                    flops = 2.0 * PEAK_CHAINS * (double)iters * blocks * PEAK_FMA_THREADS;
                } else {
                    peak_fma2_k<<<blocks, PEAK_FMA_THREADS>>>(iters, 0.999f, 1e-3f, sink);
                    flops = 4.0 * PEAK_CHAINS * (double)iters * blocks * PEAK_FMA_THREADS;
                }
            }
            FMM_CUDA_TRY(cudaGetLastError());
        };
        launch();  // warm-up (clocks, instruction cache)
        FMM_CUDA_TRY(cudaDeviceSynchronize());
        float best = 1e30f;
        for (int r = 0; r < reps; r++) {
            FMM_CUDA_TRY(cudaEventRecord(e0, 0));
            launch();
            FMM_CUDA_TRY(cudaEventRecord(e1, 0));
            FMM_CUDA_TRY(cudaEventSynchronize(e1));
            float ms = 0.f;
            FMM_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
            best = std::min(best, ms);
        }
        int herr = 0;
        FMM_CUDA_TRY(cudaMemcpy(&herr, err, sizeof(int), cudaMemcpyDeviceToHost));
        if (herr) throw Error{FMM_ECUDA, "fmm_measure_peak: the MMA commit was not seen within the wait bound"};
        *tflops = flops / (best * 1e-3) / 1e12;
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        cudaFree(sink);
        cudaFree(err);
        return FMM_OK;
    } catch (const Error &e) {
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        if (sink) cudaFree(sink);
        if (err) cudaFree(err);
        set_error(e.msg);
        return e.code;
    }
}
