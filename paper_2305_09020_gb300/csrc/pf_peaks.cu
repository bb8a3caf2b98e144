// Measured compute peaks of the current device: the denominators of the roofline fractions that
// the benchmark reports for the fast-diagonalisation transforms (the paper has no counterpart).
//
//   TF32 tensor: one CTA per SM, one thread issues back-to-back tcgen05.mma kind::tf32 of shape
//                M = 128, N = 256, K = 8 from shared memory into one TMEM accumulator; the
//                operands are zero, the rate does not depend on the values
//   FP32 / FP64: every thread runs eight independent FMA chains (FFMA / DFMA)
// Each is timed with CUDA events around one launch, best of five, after a warm-up launch.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>

#include "../../include/pf.h"
#define PF_TC_HELPERS_ONLY
#include "pf_tc.cuh"

void pf_internal_set_error(const std::string &msg);   // pf_api.cu: message for pf_last_error(NULL)

namespace {

constexpr int PEAK_N = 256;
constexpr int PEAK_SMEM = (128 + PEAK_N) * 128 + 1024 + 64;

__global__ void __launch_bounds__(128, 1) k_peak_tf32(int iters, int *err, unsigned long long wait_ns) {
    extern __shared__ __align__(1024) unsigned char raw[];
    unsigned char *base = (unsigned char *)(((uintptr_t)raw + 1023) & ~(uintptr_t)1023);
    uint64_t *mbar = (uint64_t *)(base + (128 + PEAK_N) * 128);
    uint32_t *slot = (uint32_t *)(mbar + 1);
    for (int i = threadIdx.x; i < (128 + PEAK_N) * 128 / 16; i += blockDim.x)
        ((float4 *)base)[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (threadIdx.x == 0) {
        pf::mbar_init(pf::smem_u32(mbar), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (threadIdx.x < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(pf::smem_u32(slot)),
                     "r"(PEAK_N)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *slot;
    if (threadIdx.x == 0) {
        const uint32_t a = pf::smem_u32(base), b = a + 128 * 128;
        const uint32_t idesc = pf::idesc_tf32(128, PEAK_N);
        for (int i = 0; i < iters; ++i) {
            const uint32_t o = (uint32_t)((i & 3) * 32);
            pf::mma_tf32(tmem, pf::sdesc_sw128(a + o), pf::sdesc_sw128(b + o), idesc, i > 0 ? 1u : 0u);
        }
        pf::mma_commit(pf::smem_u32(mbar));
        if (!pf::mbar_wait(pf::smem_u32(mbar), 0u, nullptr, wait_ns)) atomicExch(err, pf::TC_ERR_TIMEOUT);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (threadIdx.x < 32) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(PEAK_N) : "memory");
    }
}

template <typename T>
__global__ void __launch_bounds__(256) k_peak_fma(int iters, T a, T b, T *out) {
    T x[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) x[j] = (T)(threadIdx.x + j);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < 8; ++j) x[j] = x[j] * a + b;
    }
    T s = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) s += x[j];
    if (s == (T)-1.2345) out[0] = s;   // keeps the chains alive; never true for these inputs
}

template <typename F>
double best_ms(F launch, cudaEvent_t e0, cudaEvent_t e1) {
    launch();   // warm-up
    double best = 1e30;
    for (int r = 0; r < 5; ++r) {
        cudaEventRecord(e0);
        launch();
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        best = std::min(best, (double)ms);
    }
    return best;
}

}  // namespace

extern "C" int pf_measure_peaks(double out[3]) {
    if (!out) return PF_EINVAL;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        pf_internal_set_error("pf_measure_peaks: no CUDA device");
        return PF_ECUDA;
    }
    int *err = nullptr;
    double *dout = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaMalloc(&err, sizeof(int)) != cudaSuccess || cudaMalloc(&dout, sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(err);
        pf_internal_set_error("pf_measure_peaks: cudaMalloc failed");
        return PF_ENOMEM;
    }
    cudaMemset(err, 0, sizeof(int));
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaFuncSetAttribute(k_peak_tf32, cudaFuncAttributeMaxDynamicSharedMemorySize, PEAK_SMEM);
    const int iters = 4096;
    const double ms_tc = best_ms([&] { k_peak_tf32<<<sms, 128, PEAK_SMEM>>>(iters, err, 1000000000ull); }, e0, e1);
    const int fit = 16384;
    const double ms32 = best_ms([&] { k_peak_fma<float><<<sms * 8, 256>>>(fit, 0.999f, 1e-3f, (float *)dout); }, e0, e1);
    const int dit = 1024;
    const double ms64 = best_ms([&] { k_peak_fma<double><<<sms * 8, 256>>>(dit, 0.999, 1e-3, dout); }, e0, e1);
    int herr = 0;
    cudaError_t e = cudaMemcpy(&herr, err, sizeof(int), cudaMemcpyDeviceToHost);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(err);
    cudaFree(dout);
    if (e != cudaSuccess || cudaGetLastError() != cudaSuccess) {
        pf_internal_set_error("pf_measure_peaks: a measurement kernel failed");
        return PF_ECUDA;
    }
    if (herr) {
        pf_internal_set_error("pf_measure_peaks: the tensor-core loop gave up waiting");
        return PF_ETIMEOUT;
    }
    out[0] = (double)sms * iters * (2.0 * 128 * PEAK_N * 8) / (ms_tc * 1e-3) / 1e12;
    out[1] = (double)sms * 8 * 256 * fit * 8 * 2.0 / (ms32 * 1e-3) / 1e12;
    out[2] = (double)sms * 8 * 256 * dit * 8 * 2.0 / (ms64 * 1e-3) / 1e12;
    return PF_OK;
}
