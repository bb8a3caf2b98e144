// Tensor-core (tcgen05, sm_103a) GEMM for the single-precision fast-diagonalisation transforms
// (the constant eigenbasis products of the Remark after Algorithm 2).
//
// C[M x N] = A[M x K] * B[K x N] in "3xTF32": A and B are split into TF32 heads and tails
// (x = hi + lo) and the tensor core accumulates hi*hi + hi*lo + lo*hi in FP32; the dropped lo*lo
// term is ~2^-21 relative, so the product has single-precision accuracy.  B (an eigenbasis,
// constant for the run) is split once on the host (both parts rounded to nearest) and stored
// transposed and zero padded as Bt[Npad][Kpad] (K-major).  A's head is the landed FP32 chunk
// itself, which the tensor core truncates to TF32; its tail, the exact remainder rounded to
// nearest, is written to shared memory after the chunk lands.
//
// Persistent, warp-specialised kernel; one CTA per SM walks tiles of 128 rows x BN columns:
//   warp 8      TMA producer: per 32-wide K chunk, A (128 x 32) and both halves of Bt (BN x 32)
//               into a ring of shared-memory stages (128-byte swizzle, the layout the MMA reads)
//   warps 10-11 write the TF32 tail of each landed A chunk into a second buffer (the landed chunk
//               is the head: the tensor core truncates FP32 words to TF32)
//   warp 9      one thread issues tcgen05.mma (M = 128, N = BN, K = 8) and commits to mbarriers
//   warps 0-7   drain the TMEM accumulators into FP32 registers (all of a thread's columns loaded
//               before one wait) and run the epilogue; setmaxnreg moves registers from warps 8-11
//               (producer, MMA, split) to them
// The tensor core's FP32 accumulation is not rounded to nearest, and the eigenvector sums cancel
// heavily, so a chain of MMAs in one accumulator loses digits (chunks of 32 in one region: phi of
// the 2D droplet drifted 4x further from the oracle in 50 steps than with one region per slice).
// Each group of `gs` 8-wide K slices therefore accumulates into its own TMEM region, taken from a
// ring of NR regions: the MMAs of later groups run while warps 0-7 add the finished groups into
// FP32 registers with round-to-nearest, in K order.  Two layouts (`sep`):
//   sep = 0  a group's region takes all three products of its slices (the two small correction
//            products first); every product added into a running sum is truncated against it
//   sep = 1  the main products hi*hi go to the group's region; the correction products of the
//            whole tile (2^-11 of the main term, so their truncations are 2^-11 smaller) chain into
//            one region per tile (two, alternating between tiles), drained once per tile: per
//            slice one truncation against a running main-term sum, as with sep = 0 and one slice
//            per group, at a fraction of the drains
// Every mbarrier wait is bounded (counted in SM cycles); on time-out the kernel records an error word, lets its own copies and MMAs finish (bounded), frees its
// tensor memory and returns.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace pf {

constexpr int TC_BM = 128;                          // rows per tile = TMEM lanes
constexpr int TC_KC = 32;                           // K per stage: one 128-byte row of FP32
constexpr int TC_EPI_WARPS = 8;                     // warpgroups 0-1: one per column half
constexpr int TC_CONV_WARPS = 2;                    // warps 10-11: the A split
constexpr int TC_THREADS = 12 * 32;                 // warpgroup 2: producer, MMA, converters
// register split (setmaxnreg): the launch holds 384 x 168 = 64512 registers; warpgroup 2 gives
// back down to 72 a thread and the epilogue warpgroups take 216: 256 x 216 + 128 x 72 = 64512
constexpr int TC_REG_EPI = 216, TC_REG_AUX = 72;
static_assert(TC_EPI_WARPS * 32 * TC_REG_EPI + (TC_THREADS - TC_EPI_WARPS * 32) * TC_REG_AUX <= 65536,
              "the setmaxnreg split must fit the launch's registers");
constexpr int TC_MAXH = 64;                         // accumulator columns per thread: BN <= 128
constexpr int TC_MAXR = 8;                          // TMEM regions in the ring at most
constexpr int TC_ERR_TIMEOUT = 1;                   // error word: a bounded wait gave up

struct TcArgs {
    int M;                    // rows of A and C (< 2^31)
    int N;                    // columns of C
    int BN;                   // column tile, multiple of 16, <= 2 TC_MAXH (128)
    int BNlast;               // width of the last column tile (multiple of 16, <= BN)
    int ntn;                  // column tiles
    int nchunk;               // K chunks of 32 (Kpad / 32)
    int gs;                   // 8-wide K slices per TMEM accumulation group (>= 1; a tile's last
                              // group may be shorter)
    int nr;                   // TMEM regions in the ring (nr <= TC_MAXR; (nr + 2 sep) BN <= tmem_cols)
    int sep;                  // 1: correction products in a per-tile region of their own (above)
    int stages;               // shared-memory stages
    int tmem_cols;            // allocated TMEM columns (power of two >= 2 BN)
    int ntiles;               // row tiles x column tiles
    // epilogue: row m = p R + r; store 0: C[m ldc + n]; store 1: C[(p N + n) ldr + r]
    int R, store, ldc, ldr;
    const float *lamN, *lamR, *cpl;   // optional division by lamN[n] + lamR[r] + cpl[p % cpl_mod]
    int cpl_mod;
    float *C;
    float *C2;                // optional C2[m ldc + n] = -m2x[n] m2y[r] C (+ face2[p N + n] on r == 0)
    const float *m2x, *m2y, *face2;
    int *err;                 // error word (TC_ERR_TIMEOUT)
    unsigned long long wait_ns;   // bound of every wait
    int stall;                // test hook: wait on a barrier that nothing arrives at, then report
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// round to the nearest TF32 value, ties away from zero, in integer arithmetic (full-rate ALU ops):
// add half a unit of the 10-bit mantissa's last place to the magnitude bits and clear the 13 low
// bits; a carry moves into the exponent as rounding requires; non-finite inputs stay non-finite
__device__ __forceinline__ float tf32_rna(float x) {
    return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}

// the TF32 value the tensor core takes from an FP32 word: its upper 19 bits
__device__ __forceinline__ float tf32_trunc(float x) { return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u); }

// K-major, 128-byte swizzle, 8-row atoms of 1024 bytes: matrix descriptor of a tile at addr
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t addr) {
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFF);          // start address
    d |= (uint64_t)1 << 16;                         // leading byte offset (unused: swizzled K-major)
    d |= (uint64_t)(1024 >> 4) << 32;               // stride byte offset: next 8-row group
    d |= (uint64_t)1 << 46;                         // descriptor version (sm_100 family)
    d |= (uint64_t)2 << 61;                         // 128-byte swizzle
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

// One test of the phase; a thread whose phase is not complete sleeps in hardware (up to a
// microsecond) until it completes instead of spinning: waiting warps leave the issue slots to the
// warps that work.
__device__ __forceinline__ bool mbar_try(uint32_t mbar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(mbar), "r"(parity), "r"(1000u)
        : "memory");
    return done != 0;
}

// Wait for the phase of `parity` to complete.  Gives up (false) after about limit_ns of waiting
// (counted in SM clock cycles at up to 2.5 GHz: the cycle counter is cheap to read, unlike the
// global timer), or at once when another thread of the CTA has raised the abort flag (abort may
// be null).
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity, const volatile int *abort,
                                          unsigned long long limit_ns) {
    if (mbar_try(mbar, parity)) return true;
    const long long t0 = clock64();
    const long long limit = (long long)(limit_ns * 5ull / 2ull);   // cycles
    for (;;) {
        if (mbar_try(mbar, parity)) return true;
        if (abort && *abort) return false;
        if (clock64() - t0 > limit) return false;
    }
}

__device__ __forceinline__ void mbar_init(uint32_t mbar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mbar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t mbar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(mbar) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t mbar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes) : "memory");
}

// 2D tiled TMA load of the box at (x = inner coordinate, y = row) into shared memory
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y, uint32_t mbar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            dst),
        "l"((unsigned long long)map), "r"(x), "r"(y), "r"(mbar)
        : "memory");
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float *v) {
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
#pragma unroll
    for (int j = 0; j < 8; ++j) v[j] = __uint_as_float(r[j]);
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float *v) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
#pragma unroll
    for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}

// the hbn (<= TC_MAXH, a multiple of 8) accumulator columns of this thread's lane at taddr into
// v: 32-column loads where whole, 8-column loads for the rest; the caller waits (wait::ld)
__device__ __forceinline__ void tmem_ld_cols(uint32_t taddr, int hbn, float *v) {
#pragma unroll
    for (int j0 = 0; j0 < TC_MAXH; j0 += 32) {
        if (j0 + 32 <= hbn) {
            tmem_ld32(taddr + (uint32_t)j0, v + j0);
        } else {
#pragma unroll
            for (int j1 = j0; j1 < j0 + 32; j1 += 8)
                if (j1 < hbn) tmem_ld8(taddr + (uint32_t)j1, v + j1);
        }
    }
}

// acc[j] += v[j] for j < hbn, two lanes of FP32 per instruction (round to nearest)
__device__ __forceinline__ void add_cols(float *acc, const float *v, int hbn) {
#pragma unroll
    for (int j = 0; j < TC_MAXH; j += 2)
        if (j < hbn) {
            unsigned long long x, y, z;
            asm("mov.b64 %0, {%1, %2};" : "=l"(x) : "f"(acc[j]), "f"(acc[j + 1]));
            asm("mov.b64 %0, {%1, %2};" : "=l"(y) : "f"(v[j]), "f"(v[j + 1]));
            asm("add.rn.f32x2 %0, %1, %2;" : "=l"(z) : "l"(x), "l"(y));
            asm("mov.b64 {%0, %1}, %2;" : "=f"(acc[j]), "=f"(acc[j + 1]) : "l"(z));
        }
}

#ifndef PF_TC_HELPERS_ONLY   // translation units that only need the helpers above
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_gemm_tc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmBh,
              const __grid_constant__ CUtensorMap tmBl, TcArgs g) {
    extern __shared__ __align__(1024) unsigned char tc_raw[];
    unsigned char *base = (unsigned char *)(((uintptr_t)tc_raw + 1023) & ~(uintptr_t)1023);
    const int S = g.stages, BN = g.BN;
    const uint32_t ABYTES = TC_BM * TC_KC * 4, BBYTES = (uint32_t)BN * TC_KC * 4;
    const uint32_t STAGE = 2 * ABYTES + 2 * BBYTES;
    uint64_t *bars = (uint64_t *)(base + (size_t)S * STAGE);
    // barriers: full[S] (TMA landed), conv[S] (A split), empty[S] (MMAs done with the stage),
    // rfull[TC_MAXR] (a group's MMAs done), rempty[TC_MAXR] (a group drained), stall,
    // cfull[2] (a tile's correction products done), cempty[2] (drained)
    const int NR = g.nr, SEP = g.sep;
    const uint32_t b_full = smem_u32(bars), b_conv = b_full + 8 * S, b_empty = b_conv + 8 * S;
    const uint32_t b_rfull = b_empty + 8 * S, b_rempty = b_rfull + 8 * TC_MAXR, b_stall = b_rempty + 8 * TC_MAXR;
    const uint32_t b_cfull = b_stall + 8, b_cempty = b_cfull + 16;
    const uint32_t rbase = SEP ? 2u * (uint32_t)BN : 0u;   // column of the ring's first region
    uint32_t *tslot = (uint32_t *)(bars + 3 * S + 2 * TC_MAXR + 5);
    volatile int *abort_flag = (volatile int *)(tslot + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    if (tid == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(b_full + 8 * s, 1);
            mbar_init(b_conv + 8 * s, TC_CONV_WARPS);
            mbar_init(b_empty + 8 * s, 1);
        }
        for (int r = 0; r < TC_MAXR; ++r) {
            mbar_init(b_rfull + 8 * r, 1);
            mbar_init(b_rempty + 8 * r, TC_EPI_WARPS);
        }
        mbar_init(b_stall, 1);
        for (int c = 0; c < 2; ++c) {
            mbar_init(b_cfull + 8 * c, 1);
            mbar_init(b_cempty + 8 * c, TC_EPI_WARPS);
        }
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (g.stall) {   // test hook: nothing arrives at b_stall; report the time-out and leave
        __syncthreads();
        if (tid == 0 && !mbar_wait(b_stall, 0u, abort_flag, g.wait_ns)) atomicExch(g.err, TC_ERR_TIMEOUT);
        return;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(g.tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;
    const int nchunk = g.nchunk;
    const int my_tiles = g.ntiles > (int)blockIdx.x ? (g.ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    const int Q = my_tiles * nchunk;   // K chunks this CTA walks (stage of chunk q: q mod S)
    auto fail = [&]() {
        if (!*abort_flag) atomicExch(g.err, TC_ERR_TIMEOUT);
        *abort_flag = 1;
    };

    if (warp >= TC_EPI_WARPS) asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(TC_REG_AUX));
    if (warp == TC_EPI_WARPS) {
        // ---- TMA producer -------------------------------------------------------------------
        if (lane == 0) {
            asm volatile("prefetch.tensormap [%0];" ::"l"((unsigned long long)&tmA) : "memory");
            asm volatile("prefetch.tensormap [%0];" ::"l"((unsigned long long)&tmBh) : "memory");
            asm volatile("prefetch.tensormap [%0];" ::"l"((unsigned long long)&tmBl) : "memory");
            // tile coordinates kept as running counters (no division per chunk)
            const int ntn = g.ntn, gstep = (int)gridDim.x % ntn, mstep = (int)gridDim.x / ntn;
            int issued = 0, s = 0, c = 0, mt = (int)blockIdx.x / ntn, nt = (int)blockIdx.x % ntn;
            uint32_t ph = 0;
            for (int q = 0; q < Q; ++q) {
                if (!mbar_wait(b_empty + 8 * s, ph ^ 1u, abort_flag, g.wait_ns)) { fail(); break; }
                const uint32_t sb = smem_u32(base + (size_t)s * STAGE);
                mbar_expect_tx(b_full + 8 * s, STAGE - ABYTES);   // A, Bt hi, Bt lo (A's lo buffer is ours)
                tma_load_2d(sb, &tmA, c * TC_KC, mt * TC_BM, b_full + 8 * s);
                tma_load_2d(sb + 2 * ABYTES, &tmBh, c * TC_KC, nt * BN, b_full + 8 * s);
                tma_load_2d(sb + 2 * ABYTES + BBYTES, &tmBl, c * TC_KC, nt * BN, b_full + 8 * s);
                issued = q + 1;
                if (++s == S) { s = 0; ph ^= 1u; }
                if (++c == nchunk) {
                    c = 0;
                    mt += mstep;
                    nt += gstep;
                    if (nt >= ntn) { nt -= ntn; ++mt; }
                }
            }
            // our copies still in flight (only after an abort) finish before the CTA leaves
            for (int q = issued - 1; q >= 0 && q >= issued - S; --q)
                mbar_wait(b_full + 8 * (q % S), (uint32_t)((q / S) & 1), nullptr, g.wait_ns);
        }
        __syncwarp();
    } else if (warp == TC_EPI_WARPS + 1) {
        // ---- MMA issuer -----------------------------------------------------------------------
        // One thread issues every MMA, so its loop is latency-bound: no divisions, descriptors
        // advanced by constants, group and ring positions kept as running counters.
        if (lane == 0) {
            const uint32_t idesc_full = idesc_tf32(TC_BM, BN), idesc_last = idesc_tf32(TC_BM, g.BNlast);
            // shared-memory descriptors advance in 16-byte units: stage, operand and K-slice offsets
            const uint64_t dbase = sdesc_sw128(smem_u32(base));
            const uint64_t dstage = STAGE >> 4, daL = ABYTES >> 4, dbH = (2 * ABYTES) >> 4,
                           dbL = (2 * ABYTES + BBYTES) >> 4;
            const int gs = g.gs, ntn = g.ntn, gstep = (int)gridDim.x % ntn;
            int nt = (int)blockIdx.x % ntn;   // column tile of the current tile
            int s = 0, c = 0, it = 0, r = 0, ing = 0;   // stage, chunk, tile, ring region, slice in group
            uint32_t ph = 0, rph = 0;                   // stage and ring phases
            uint64_t ds = dbase;
            bool ok = true;
            for (int q = 0; q < Q && ok; ++q) {
                // sep: the products with A's head start once the chunk has landed, the ones with its
                // tail once the split warps have written it; otherwise every product waits for them
                if (!mbar_wait((SEP ? b_full : b_conv) + 8 * s, ph, abort_flag, g.wait_ns)) { fail(); break; }
                // sep: the tile's correction region (it & 1) is free once its previous tile is drained
                if (SEP && c == 0 &&
                    !mbar_wait(b_cempty + 8 * (it & 1), (uint32_t)(((it >> 1) & 1) ^ 1), abort_flag, g.wait_ns)) {
                    fail();
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t idesc = nt == ntn - 1 ? idesc_last : idesc_full;
                const uint32_t dcor = tmem + (uint32_t)((it & 1) * BN);
                const bool last_chunk = c == nchunk - 1;
#pragma unroll
                for (int kk = 0; kk < TC_KC / 8; ++kk) {
                    // groups of gs slices counted from the tile's first slice; the tile's last
                    // slice closes its group
                    const bool first = ing == 0;
                    const bool last = ing == gs - 1 || (last_chunk && kk == TC_KC / 8 - 1);
                    if (first) {
                        if (!mbar_wait(b_rempty + 8 * r, rph ^ 1u, abort_flag, g.wait_ns)) {
                            fail();
                            ok = false;
                            break;
                        }
                        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    }
                    const uint32_t d = tmem + rbase + (uint32_t)(r * BN);
                    const uint64_t o = ds + 2 * kk;     // this 8-wide K slice: 32 bytes further
                    if (SEP) {   // head x tail of B into the tile's region, the main product into the group's
                        mma_tf32(dcor, o, o + dbL, idesc, (c == 0 && kk == 0) ? 0u : 1u);
                        mma_tf32(d, o, o + dbH, idesc, first ? 0u : 1u);
                    } else {     // the two small correction products first, then the main term
                        mma_tf32(d, o + daL, o + dbH, idesc, first ? 0u : 1u);
                        mma_tf32(d, o, o + dbL, idesc, 1u);
                        mma_tf32(d, o, o + dbH, idesc, 1u);
                    }
                    if (last) {
                        mma_commit(b_rfull + 8 * r);
                        ing = 0;
                        if (++r == NR) { r = 0; rph ^= 1u; }
                    } else {
                        ++ing;
                    }
                }
                if (!ok) break;
                if (SEP) {   // A's tail x head of B, once the split warps are done with the chunk
                    if (!mbar_wait(b_conv + 8 * s, ph, abort_flag, g.wait_ns)) { fail(); break; }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
                    for (int kk = 0; kk < TC_KC / 8; ++kk) mma_tf32(dcor, ds + 2 * kk + daL, ds + 2 * kk + dbH, idesc, 1u);
                    if (last_chunk) {
                        mma_commit(b_cfull + 8 * (it & 1));
                        ++it;
                    }
                }
                mma_commit(b_empty + 8 * s);   // the stage is free once these MMAs have read it
                if (++s == S) { s = 0; ph ^= 1u; ds = dbase; } else { ds += dstage; }
                if (++c == nchunk) {
                    c = 0;
                    nt += gstep;
                    if (nt >= ntn) nt -= ntn;
                }
            }
            // every MMA issued (also after an abort) finishes before the tensor memory is released:
            // one more commit, on the barrier the stall hook uses (idle on this path)
            mma_commit(b_stall);
            mbar_wait(b_stall, 0u, nullptr, g.wait_ns);
        }
        __syncwarp();
    } else if (warp < TC_EPI_WARPS) {
        // ---- drain the accumulators, epilogue (warps 0-7) ----------------------------------------
        asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(TC_REG_EPI));
        const int quarter = warp & 3, half = warp >> 2;
        float acc[TC_MAXH];
#pragma unroll
        for (int j = 0; j < TC_MAXH; ++j) acc[j] = 0.f;
        const int ngrp = ((TC_KC / 8) * nchunk + g.gs - 1) / g.gs;   // groups per tile
        int r = 0;           // ring region of the next group, and its phase
        uint32_t rph = 0;
        bool ok = true;
        for (int it = 0; it < my_tiles && ok; ++it) {
            // the tile's groups, in K order, into the registers
            const int td = (int)blockIdx.x + it * (int)gridDim.x;
            const int hbn = ((td % g.ntn == g.ntn - 1) ? g.BNlast : BN) >> 1;   // columns per thread
            for (int gi = 0; gi < ngrp; ++gi) {
                if (!mbar_wait(b_rfull + 8 * r, rph, abort_flag, g.wait_ns)) {
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t ta =
                    tmem + ((uint32_t)(quarter * 32) << 16) + rbase + (uint32_t)(r * BN + half * hbn);
                {   // every column of the group first, then one wait
                    float v[TC_MAXH];
                    tmem_ld_cols(ta, hbn, v);
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                    add_cols(acc, v, hbn);
                }
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                __syncwarp();
                if (lane == 0) mbar_arrive(b_rempty + 8 * r);
                if (++r == NR) { r = 0; rph ^= 1u; }
            }
            if (!ok) break;
            if (SEP) {   // the tile's correction products, once
                const int cr = it & 1;
                if (!mbar_wait(b_cfull + 8 * cr, (uint32_t)((it >> 1) & 1), abort_flag, g.wait_ns)) {
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t ta = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(cr * BN + half * hbn);
                float v[TC_MAXH];
                tmem_ld_cols(ta, hbn, v);
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                add_cols(acc, v, hbn);
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                __syncwarp();
                if (lane == 0) mbar_arrive(b_cempty + 8 * cr);
            }
            // ---- epilogue of tile td ------------------------------------------------------------
            const int mt = td / g.ntn, nt = td - mt * g.ntn;
            const int m = mt * TC_BM + quarter * 32 + lane;
            const int nb = nt * BN + half * hbn;
            if (m < g.M) {
                const int p = m / g.R;
                const int rr = m - p * g.R;
                const float lr = g.lamN ? g.lamR[rr] + g.cpl[p % g.cpl_mod] : 0.f;
                const float my = g.C2 ? g.m2y[rr] : 0.f;
                // store 1: lanes hold consecutive rows r, so each column's stores are coalesced;
                // store 0: a row's columns are contiguous (16-byte stores; ldc, nb multiples of 4)
                float *cb = g.store == 1 ? g.C + ((long long)p * g.N + nb) * g.ldr + rr : g.C + (long long)m * g.ldc + nb;
                float *c2b = g.C2 ? g.C2 + (long long)m * g.ldc + nb : nullptr;
                const float *fb = (g.face2 && rr == 0) ? g.face2 + (long long)p * g.N + nb : nullptr;
                const int ncol = min(hbn, g.N - nb);
                // eight columns at a time; the empty asm keeps the loads of one group from being
                // hoisted over the others (register pressure)
#pragma unroll
                for (int j0 = 0; j0 < TC_MAXH; j0 += 8) {
                    if (j0 < ncol) {
                        if (g.lamN) {
#pragma unroll
                            for (int u = 0; u < 8; ++u)
                                if (j0 + u < ncol) {
                                    const float dd = g.lamN[nb + j0 + u] + lr;
                                    acc[j0 + u] = (dd != 0.f) ? acc[j0 + u] / dd : 0.f;
                                }
                        }
                        if (g.store == 1) {
#pragma unroll
                            for (int u = 0; u < 8; ++u)
                                if (j0 + u < ncol) cb[(long long)(j0 + u) * g.ldr] = acc[j0 + u];
                        } else if (j0 + 8 <= ncol) {
                            *(float4 *)(cb + j0) = make_float4(acc[j0], acc[j0 + 1], acc[j0 + 2], acc[j0 + 3]);
                            *(float4 *)(cb + j0 + 4) = make_float4(acc[j0 + 4], acc[j0 + 5], acc[j0 + 6], acc[j0 + 7]);
                        } else {
#pragma unroll
                            for (int u = 0; u < 8; ++u)
                                if (j0 + u < ncol) cb[j0 + u] = acc[j0 + u];
                        }
                        if (c2b) {
#pragma unroll
                            for (int u = 0; u < 8; ++u)
                                if (j0 + u < ncol) {
                                    float w2 = -g.m2x[nb + j0 + u] * my * acc[j0 + u];
                                    if (fb) w2 += fb[j0 + u];
                                    c2b[j0 + u] = w2;
                                }
                        }
                    }
                    asm volatile("" ::: "memory");
                }
            }
#pragma unroll
            for (int j = 0; j < TC_MAXH; ++j) acc[j] = 0.f;
        }
        if (!ok) fail();
    } else {
        // ---- A's TF32 tail (warps 10-11: 64 floats a thread) ---------------------------------
        // The tensor core reads a TF32 operand by truncating the FP32 word to its upper 19 bits
        // (measured on the GB300: 1 + 3 2^-12 enters an MMA as 1), so the landed A serves as the
        // head as it is; the tail is the exact remainder x - trunc(x), rounded to nearest TF32.
        const int ct = tid - (TC_EPI_WARPS + 2) * 32;   // 0 .. 32 TC_CONV_WARPS - 1
        int s = 0;
        uint32_t ph = 0;
        for (int q = 0; q < Q; ++q) {
            if (!mbar_wait(b_full + 8 * s, ph, abort_flag, g.wait_ns)) {
                fail();
                break;
            }
            unsigned char *sa = base + (size_t)s * STAGE;
#pragma unroll 4
            for (int i = ct; i < (int)(ABYTES / 16); i += 32 * TC_CONV_WARPS) {
                const uint32_t off = (uint32_t)(16 * i);
                const float4 x = *(const float4 *)(sa + off);
                float4 l;
                l.x = tf32_rna(x.x - tf32_trunc(x.x));
                l.y = tf32_rna(x.y - tf32_trunc(x.y));
                l.z = tf32_rna(x.z - tf32_trunc(x.z));
                l.w = tf32_rna(x.w - tf32_trunc(x.w));
                *(float4 *)(sa + ABYTES + off) = l;
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(b_conv + 8 * s);
            if (++s == S) { s = 0; ph ^= 1u; }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(g.tmem_cols) : "memory");
    }
}

#endif  // PF_TC_HELPERS_ONLY

}  // namespace pf
