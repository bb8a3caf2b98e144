// Tensor-core (tcgen05, sm_103a) GEMM for the single-precision fast-diagonalisation transforms.
//
// C[M x N] = A[M x Kd] * B[Kd x N] in "3xTF32": every operand is split into a TF32 head and a
// TF32 tail (x = hi + lo, both rounded to nearest), and the three products hi*hi, hi*lo, lo*hi
// accumulate in FP32 in tensor memory; the dropped lo*lo term is ~2^-22 relative, so the result
// has single-precision accuracy.  B (an eigenbasis, constant for the run) is split once on the
// host and stored transposed and zero-padded as Bt[Npad][Kpad]; A is split while it is staged.
//
// One CTA (4 warps) owns 128 rows of A and a tile of TN columns: per 32-wide K chunk the threads
// stage A (hi, lo) and Bt (hi, lo) into shared memory in the K-major 128-byte-swizzled layout,
// one thread issues the MMAs (M = 128, N = TN, K = 8 per instruction) and commits them to an
// mbarrier.  For every 8-wide K slice the hi*hi product goes to its own TMEM region and the two
// small correction products to another, so the tensor core never adds a large term to a
// running sum; the regions are read back with tcgen05.ld and summed in FP32 registers with
// round-to-nearest.  The epilogue divides by the eigenvalue sum and/or stores per plane.
// Every wait on the mbarrier is bounded; on time-out the kernel records an error code and
// returns after freeing its tensor memory.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace pf {

struct TcArgs {
    const float *A;           // M x Kd row-major
    const float *Bhi, *Blo;   // Npad x Kpad row-major (B transposed, split, zero padded)
    float *C;
    long long Mrows;
    int Kd, N, Npad, Kpad;
    int ntile, tile_n;        // unused by the column-tiled kernel (kept for the launch helper)
    int tmem_cols;
    int R, store;             // epilogue as in GemmArgs
    const float *lamN, *lamR, *cpl;
    int cpl_mod;
    int *err;                 // set to 1 when a bounded wait gives up
    float *C2;                // optional: C2 = -m2x[n] m2y[r] C (+ face2[p N + n] on row r == 0)
    const float *m2x, *m2y, *face2;
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// round to nearest TF32 (10 explicit mantissa bits), kept in an FP32 container
__device__ __forceinline__ float tf32_rna(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// K-major, 128-byte swizzle, 8-row atoms of 1024 bytes: descriptor of a tile starting at addr
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t addr) {
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFF);          // start address
    d |= (uint64_t)1 << 16;                         // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(1024 >> 4) << 32;               // stride byte offset: next 8-row group
    d |= (uint64_t)1 << 46;                         // descriptor version (sm_100 family)
    d |= (uint64_t)2 << 61;                         // swizzle: 128 bytes
    return d;
}

// instruction descriptor: D = F32, A = B = TF32, both K-major, shape M x N
__device__ __forceinline__ uint32_t idesc_tf32(int M, int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                 : "memory");
}

__device__ __forceinline__ bool mbar_wait_bounded(uint32_t mbar, uint32_t parity) {
    for (int it = 0; it < (1 << 24); ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(mbar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// byte offset of element (row r, k) in a 32-wide K chunk stored K-major with 128B swizzle
__device__ __forceinline__ uint32_t sw128_off(int r, int k) {
    return (uint32_t)((r >> 3) * 1024 + (r & 7) * 128 + ((((k >> 2) ^ (r & 7)) & 7) << 4) + (k & 3) * 4);
}

// One CTA: 128 rows of A x TN columns (blockIdx.y selects the column tile).  K is walked in
// 32-wide chunks, double-buffered: while the tensor core multiplies chunk c the threads stage
// chunk c+1.  Each chunk writes into one of two TMEM buffers (8 regions each) and is added to
// FP32 registers (round to nearest) after it completes.
template <int TN>
__global__ void __launch_bounds__(128, 1) k_gemm_tc(TcArgs g) {
    extern __shared__ __align__(1024) unsigned char tc_smem_raw[];
    unsigned char *base = (unsigned char *)(((uintptr_t)tc_smem_raw + 1023) & ~(uintptr_t)1023);
    constexpr int ABYTES = 128 * 32 * 4;          // one A chunk (hi or lo)
    constexpr int BBYTES = TN * 32 * 4;           // one Bt chunk (hi or lo)
    constexpr int STAGE = 2 * ABYTES + 2 * BBYTES;
    uint64_t *mbar = (uint64_t *)(base + 2 * STAGE);
    uint32_t *tslot = (uint32_t *)(mbar + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const long long m0 = (long long)blockIdx.x * 128;
    const int n0 = blockIdx.y * TN;
    // TMEM: 2 buffers x 4 K-slices x {hi*hi, lo*hi + hi*lo} regions of TN columns
    constexpr uint32_t NREG = 8;
    constexpr uint32_t TCOLS = (2 * NREG * TN < 32) ? 32 : 2 * NREG * TN;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(TCOLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mbar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;
    const uint32_t idesc = idesc_tf32(128, TN);
    const int nchunk = g.Kpad / 32;

    // stage chunk c: every load of the chunk is issued before the first dependent store
    auto stage = [&](int c) {
        unsigned char *sb = base + (c & 1) * STAGE;
        const int k0 = c * 32;
        const int kk = k0 + lane;            // warp w loads rows w, w+4, ..., column k0 + lane
        const bool kin = kk < g.Kd;
        float av[32];
#pragma unroll
        for (int i = 0; i < 32; ++i) {
            const long long m = m0 + warp + 4 * i;
            av[i] = (kin && m < g.Mrows) ? __ldg(g.A + m * g.Kd + kk) : 0.f;
        }
        constexpr int NB = TN * 8 / 128;     // float4 chunks of Bt per thread (hi and lo each)
        float4 bh[NB], bl[NB];
#pragma unroll
        for (int i = 0; i < NB; ++i) {
            const int idx = tid + 128 * i, r = idx >> 3, q = idx & 7;
            const long long row = n0 + r;    // < Npad: the column tiles cover Npad exactly
            bh[i] = __ldg((const float4 *)(g.Bhi + row * g.Kpad + k0 + q * 4));
            bl[i] = __ldg((const float4 *)(g.Blo + row * g.Kpad + k0 + q * 4));
        }
#pragma unroll
        for (int i = 0; i < 32; ++i) {
            const float hi = tf32_rna(av[i]);
            const float lo = tf32_rna(av[i] - hi);
            const uint32_t off = sw128_off(warp + 4 * i, lane);
            *(float *)(sb + off) = hi;
            *(float *)(sb + ABYTES + off) = lo;
        }
#pragma unroll
        for (int i = 0; i < NB; ++i) {
            const int idx = tid + 128 * i, r = idx >> 3, q = idx & 7;
            const uint32_t off = sw128_off(r, q * 4);
            *(float4 *)(sb + 2 * ABYTES + off) = bh[i];
            *(float4 *)(sb + 2 * ABYTES + BBYTES + off) = bl[i];
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    };
    auto issue = [&](int c) {   // thread 0 only
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t sb = smem_u32(base + (c & 1) * STAGE);
        const uint32_t aH = sb, aL = sb + ABYTES, bH = sb + 2 * ABYTES, bL = sb + 2 * ABYTES + BBYTES;
        const uint32_t d = tmem + (uint32_t)((c & 1) * NREG * TN);
        for (int kk = 0; kk < 4; ++kk) {
            const uint32_t o = (uint32_t)(kk * 32);
            const uint32_t dm = d + (uint32_t)(2 * kk * TN), dc = dm + (uint32_t)TN;
            mma_tf32(dc, sdesc_sw128(aL + o), sdesc_sw128(bH + o), idesc, 0u);   // corrections
            mma_tf32(dc, sdesc_sw128(aH + o), sdesc_sw128(bL + o), idesc, 1u);
            mma_tf32(dm, sdesc_sw128(aH + o), sdesc_sw128(bH + o), idesc, 0u);   // main term alone
        }
        mma_commit(smem_u32(mbar));
    };

    float acc[TN];
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[j] = 0.f;
    bool ok = true;
    stage(0);
    __syncthreads();
    if (tid == 0) issue(0);
    for (int c = 0; c < nchunk; ++c) {
        if (c + 1 < nchunk) stage(c + 1);   // overlaps the MMAs of chunk c
        const bool waited = mbar_wait_bounded(smem_u32(mbar), (uint32_t)(c & 1));
        ok = __syncthreads_and(waited ? 1 : 0) != 0;
        if (!ok) break;
        if (c + 1 < nchunk && tid == 0) issue(c + 1);
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t region = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)((c & 1) * NREG * TN);
        // sum the K-slices in FP32 (round to nearest): corrections first, then the main term
#pragma unroll
        for (int s = 0; s < 8; ++s) {
            const uint32_t rs = region + (uint32_t)((s ^ 1) * TN);   // order: corr0, main0, corr1, ...
#pragma unroll
            for (int j0 = 0; j0 < TN; j0 += 16) {
                uint32_t v[16];
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                    : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                      "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                      "=r"(v[15])
                    : "r"(rs + (uint32_t)j0));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                for (int j = 0; j < 16; ++j) acc[j0 + j] += __uint_as_float(v[j]);
            }
        }
        // region (c & 1) is rewritten by the MMAs of chunk c + 2, issued after the next barrier
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    }
    if (!ok) {
        if (lane == 0) atomicExch(g.err, 1);
        // give MMAs that may still be in flight a bounded chance to finish before freeing TMEM
        for (int c = 0; c < 2; ++c) mbar_wait_bounded(smem_u32(mbar), 0u);
    } else {
        const long long m = m0 + warp * 32 + lane;
        if (m < g.Mrows) {
            const long long p = m / g.R;
            const int r = (int)(m - p * g.R);
#pragma unroll
            for (int j = 0; j < TN; ++j) {
                const int n = n0 + j;
                if (n < g.N) {
                    float x = acc[j];
                    if (g.lamN) {
                        const float dd = g.lamN[n] + g.lamR[r] + g.cpl[p % g.cpl_mod];
                        x = (dd != 0.f) ? x / dd : 0.f;
                    }
                    if (g.store == 0) g.C[m * g.N + n] = x;
                    else g.C[(p * g.N + n) * g.R + r] = x;
                    if (g.C2) {
                        float w2 = -g.m2x[n] * g.m2y[r] * x;
                        if (g.face2 && r == 0) w2 += g.face2[p * g.N + n];
                        g.C2[m * g.N + n] = w2;
                    }
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TCOLS) : "memory");
    }
}

}  // namespace pf
