// Neural operator for warm-starting equilibrium runs (the paper has nothing like it).
//
// A multilayer perceptron maps the three run parameters (electrode voltage, permittivity
// ratio, drop area) to the phase field on a uniform n_gx x n_gy grid (x periodic on
// [x0, x1), y on [y0, y1] including both ends), which a fixed bilinear map carries to the GLL
// nodes of the run's mesh.  Hidden and output activations are tanh (phi lies in [-1, 1]).
// Weights are stored in BF16 for the forward and backward products (FP32 master copies and
// Adam moments are kept for the update); activations, accumulations and the loss are FP32.
// The loss is the mean squared difference to target phase fields at the nodes.
//
// Kernels: k_dense_fwd (Y = tanh(X W + b)), k_dense_bwd_x (dX = dZ W^T), k_dense_bwd_w
// (dW = X^T dZ, db = sum dZ), k_resample / k_resample_t (grid -> nodes and its transpose),
// k_loss (MSE and its gradient), k_adam, k_gather_rows.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <memory>
#include <random>
#include <string>
#include <vector>

#include "../../include/pf.h"
#define PF_TC_HELPERS_ONLY
#include "pf_tc.cuh"

void pf_internal_set_error(const std::string &msg);

namespace {

struct NoErr {
    cudaError_t code;
    std::string where;
};
#define NO_CU(call)                                                        \
    do {                                                                   \
        cudaError_t e_ = (call);                                           \
        if (e_ != cudaSuccess) throw NoErr{e_, std::string(#call)};        \
    } while (0)

__global__ void k_dense_fwd(const float *__restrict__ X, const __nv_bfloat16 *__restrict__ W,
                            const float *__restrict__ b, float *__restrict__ Y, int B, int K, int N,
                            const float *__restrict__ mean, const float *__restrict__ istd) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    const int r = blockIdx.y;
    if (n >= N || r >= B) return;
    float s = b[n];
    for (int k = 0; k < K; ++k) {
        float x = X[(long long)r * K + k];
        if (mean) x = (x - mean[k]) * istd[k];   // input standardisation (first layer)
        s += x * __bfloat162float(W[(long long)k * N + n]);
    }
    Y[(long long)r * N + n] = tanhf(s);
}

// The same dense layer on the tensor cores, for hidden and output layers with K % 64 == 0,
// K <= 384 and N % 128 == 0: one CTA per 128 outputs x 64 samples.  A = the layer's BF16 weights,
// transposed (Wt[N][K], K-major), B = the FP32 inputs split into BF16 head and tail (x = hi + lo,
// both rounded to nearest: the inputs keep ~16 bits, the weights are BF16 anyway);
// tcgen05.mma kind::f16 (M = 128, N = 64, K = 16) accumulates Wt (hi + lo) in FP32 in tensor memory,
// the epilogue adds the bias and applies tanh.  Operands are staged by the block's threads in the
// 128-byte-swizzled K-major layout (K in atoms of 64 BF16; rows of 128 bytes, 16-byte chunks
// permuted by row mod 8).  The wait is bounded: on time-out the error word is set and the
// results are not written.
constexpr int NO_TC_BN = 64;   // samples per CTA
__device__ __forceinline__ uint32_t sw128_off(int row, int k, int rows) {
    // byte offset of BF16 element (row, k) in a K-major, 128B-swizzled tile of `rows` rows
    const int atom = k >> 6, c = (k & 63) * 2;
    return (uint32_t)(atom * rows * 128 + row * 128 + ((((c >> 4) ^ (row & 7))) << 4) + (c & 15));
}
__global__ void __launch_bounds__(128, 1) k_dense_fwd_tc(const float *__restrict__ X, const __nv_bfloat16 *__restrict__ Wt,
                                                         const float *__restrict__ b, float *__restrict__ Y, int B, int K,
                                                         int N, int *err) {
    extern __shared__ __align__(1024) unsigned char no_raw[];
    unsigned char *base = (unsigned char *)(((uintptr_t)no_raw + 1023) & ~(uintptr_t)1023);
    unsigned char *sA = base;                                   // 128 x K
    unsigned char *sBh = sA + 128 * K * 2, *sBl = sBh + NO_TC_BN * K * 2;   // 64 x K each
    uint64_t *mbar = (uint64_t *)(sBl + NO_TC_BN * K * 2);
    uint32_t *slot = (uint32_t *)(mbar + 1);
    const int n0 = blockIdx.x * 128, r0 = blockIdx.y * NO_TC_BN, tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // weights: 16-byte chunks of Wt rows
    const int cpr = K / 8;   // chunks per row
    for (int i = tid; i < 128 * cpr; i += blockDim.x) {
        const int row = i / cpr, kc = (i - row * cpr) * 8;
        const uint4 v = *reinterpret_cast<const uint4 *>(Wt + (size_t)(n0 + row) * K + kc);
        *reinterpret_cast<uint4 *>(sA + sw128_off(row, kc, 128)) = v;
    }
    // inputs: head and tail in BF16 (rows past B are zero)
    for (int i = tid; i < NO_TC_BN * (K / 2); i += blockDim.x) {
        const int row = i / (K / 2), k = (i - row * (K / 2)) * 2;
        float2 x = make_float2(0.f, 0.f);
        if (r0 + row < B) x = *reinterpret_cast<const float2 *>(X + (size_t)(r0 + row) * K + k);
        const __nv_bfloat162 h = __floats2bfloat162_rn(x.x, x.y);
        const float2 hf = __bfloat1622float2(h);
        const __nv_bfloat162 l = __floats2bfloat162_rn(x.x - hf.x, x.y - hf.y);
        *reinterpret_cast<__nv_bfloat162 *>(sBh + sw128_off(row, k, NO_TC_BN)) = h;
        *reinterpret_cast<__nv_bfloat162 *>(sBl + sw128_off(row, k, NO_TC_BN)) = l;
    }
    if (tid == 0) {
        pf::mbar_init(pf::smem_u32(mbar), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // generic writes -> tensor core
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(pf::smem_u32(slot)),
                     "r"(NO_TC_BN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *slot;
    if (tid == 0) {
        // instruction descriptor: D = F32, A = B = BF16, both K-major, M = 128, N = 64
        const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(NO_TC_BN >> 3) << 17) |
                               ((uint32_t)(128 >> 4) << 24);
        const uint32_t a0 = pf::smem_u32(sA), bh0 = pf::smem_u32(sBh), bl0 = pf::smem_u32(sBl);
        for (int s = 0; s < K / 16; ++s) {   // 16 BF16 = 32 bytes per K step
            const uint32_t oa = (uint32_t)((s >> 2) * 128 * 128 + (s & 3) * 32);
            const uint32_t ob = (uint32_t)((s >> 2) * NO_TC_BN * 128 + (s & 3) * 32);
            const uint64_t da = pf::sdesc_sw128(a0 + oa);
            uint32_t acc = s > 0 ? 1u : 0u;
            asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                         "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
                         "l"(da), "l"(pf::sdesc_sw128(bh0 + ob)), "r"(idesc), "r"(acc));
            acc = 1u;
            asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                         "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
                         "l"(da), "l"(pf::sdesc_sw128(bl0 + ob)), "r"(idesc), "r"(acc));
        }
        pf::mma_commit(pf::smem_u32(mbar));
    }
    bool ok = pf::mbar_wait(pf::smem_u32(mbar), 0u, nullptr, 1000000000ull);
    if (!ok) {   // record the time-out, give the MMAs one more bounded wait before the memory goes
        if (lane == 0) atomicExch(err, pf::TC_ERR_TIMEOUT);
        pf::mbar_wait(pf::smem_u32(mbar), 0u, nullptr, 1000000000ull);
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (ok) {
        // warp w reads rows (outputs) 32 w .. 32 w + 31, all 64 samples
        float v[64];
        const uint32_t ta = tmem + ((uint32_t)(warp * 32) << 16);
        pf::tmem_ld32(ta, v);
        pf::tmem_ld32(ta + 32, v + 32);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        const int n = n0 + warp * 32 + lane;
        const float bn = b[n];
#pragma unroll
        for (int c = 0; c < NO_TC_BN; ++c)
            if (r0 + c < B) Y[(size_t)(r0 + c) * N + n] = tanhf(v[c] + bn);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(NO_TC_BN) : "memory");
    }
}

// Wt[n][k] = W[k][n] (BF16) for the tensor-core layers
__global__ void k_transpose_bf16(const __nv_bfloat16 *__restrict__ W, __nv_bfloat16 *__restrict__ Wt, int K, int N) {
    __shared__ __nv_bfloat16 t[32][33];
    const int k0 = blockIdx.y * 32, n0 = blockIdx.x * 32;
    for (int i = threadIdx.y; i < 32; i += blockDim.y)
        if (k0 + i < K && n0 + threadIdx.x < N) t[i][threadIdx.x] = W[(size_t)(k0 + i) * N + n0 + threadIdx.x];
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += blockDim.y)
        if (n0 + i < N && k0 + threadIdx.x < K) Wt[(size_t)(n0 + i) * K + k0 + threadIdx.x] = t[threadIdx.x][i];
}

// dZ = dY (1 - Y^2) in place on dY
__global__ void k_tanh_back(const float *__restrict__ Y, float *__restrict__ dY, long long n) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dY[i] *= 1.f - Y[i] * Y[i];
}

// dX[r][k] = sum_n dZ[r][n] W[k][n]: one warp per (r, k)
__global__ void k_dense_bwd_x(const float *__restrict__ dZ, const __nv_bfloat16 *__restrict__ W,
                              float *__restrict__ dX, int B, int K, int N) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= B * K) return;
    const int r = warp / K, k = warp % K;
    float s = 0.f;
    for (int n = lane; n < N; n += 32) s += dZ[(long long)r * N + n] * __bfloat162float(W[(long long)k * N + n]);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) dX[(long long)r * K + k] = s;
}

// dW[k][n] = sum_r Xin[r][k] dZ[r][n] ; db[n] = sum_r dZ[r][n]
__global__ void k_dense_bwd_w(const float *__restrict__ X, const float *__restrict__ dZ, float *__restrict__ dW,
                              float *__restrict__ db, int B, int K, int N, const float *__restrict__ mean,
                              const float *__restrict__ istd) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    const int k = blockIdx.y;
    if (n >= N) return;
    float s = 0.f, sb = 0.f;
    for (int r = 0; r < B; ++r) {
        float x = X[(long long)r * K + k];
        if (mean) x = (x - mean[k]) * istd[k];
        const float d = dZ[(long long)r * N + n];
        s += x * d;
        sb += d;
    }
    dW[(long long)k * N + n] = s;
    if (k == 0) db[n] = sb;
}

// nodes[r][q] = sum_{c<4} w[q][c] grid[r][idx[q][c]]
__global__ void k_resample(const float *__restrict__ G, const int *__restrict__ idx, const float *__restrict__ w,
                           float *__restrict__ out, int B, int ng, int nq) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x, r = blockIdx.y;
    if (q >= nq || r >= B) return;
    const float *g = G + (long long)r * ng;
    float s = 0.f;
    for (int c = 0; c < 4; ++c) s += w[q * 4 + c] * g[idx[q * 4 + c]];
    out[(long long)r * nq + q] = s;
}

// transpose: dG[r][i] = sum over (q, c) with idx[q][c] = i of w[q][c] dN[r][q]  (CSR by grid point)
__global__ void k_resample_t(const float *__restrict__ dN, const int *__restrict__ rowptr,
                             const int *__restrict__ col, const float *__restrict__ val, float *__restrict__ dG,
                             int B, int ng, int nq) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x, r = blockIdx.y;
    if (i >= ng || r >= B) return;
    float s = 0.f;
    for (int e = rowptr[i]; e < rowptr[i + 1]; ++e) s += val[e] * dN[(long long)r * nq + col[e]];
    dG[(long long)r * ng + i] = s;
}

// d = 2 (p - t) / (B nq); per-block partial sums of (p - t)^2 into part
__global__ void k_loss(const float *__restrict__ p, const float *__restrict__ t, float *__restrict__ d,
                       long long n, float scale, double *__restrict__ part) {
    __shared__ double sm[256];
    double acc = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float e = p[i] - t[i];
        d[i] = 2.f * e * scale;
        acc += (double)e * (double)e;
    }
    sm[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sm[threadIdx.x] += sm[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sm[0];
}

__global__ void k_adam(float *__restrict__ w, __nv_bfloat16 *__restrict__ wb, const float *__restrict__ g,
                       float *__restrict__ m, float *__restrict__ v, long long n, float lr, float b1, float b2,
                       float c1, float c2, float eps) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    w[i] = wi;
    if (wb) wb[i] = __float2bfloat16_rn(wi);
}

__global__ void k_gather_rows(const float *__restrict__ src, const int *__restrict__ rows, float *__restrict__ dst,
                              int B, int width) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x, r = blockIdx.y;
    if (c >= width || r >= B) return;
    dst[(long long)r * width + c] = src[(long long)rows[r] * width + c];
}

__global__ void k_to_bf16(const float *__restrict__ a, __nv_bfloat16 *__restrict__ b, long long n) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = __float2bfloat16_rn(a[i]);
}

}  // namespace

// Mass projection of predicted node fields (one block per sample): phi += (target - sum w phi) /
// sum w with the tensor-product quadrature weights w_ij = wx[j] wy[i]; FP64 sums.  A constant shift
// is the L2-closest field with the prescribed phase mass int phi.
__global__ void k_mass_shift(float *__restrict__ pn, int nqx, int nqy, const double *__restrict__ wx,
                             const double *__restrict__ wy, const double *__restrict__ target) {
    const int b = blockIdx.x, nq = nqx * nqy;
    float *p = pn + (size_t)b * nq;
    __shared__ double ss[256], sw[256];
    double s = 0.0, w = 0.0;
    for (int i = threadIdx.x; i < nq; i += blockDim.x) {
        const double wi = wx[i % nqx] * wy[i / nqx];
        s += wi * (double)p[i];
        w += wi;
    }
    ss[threadIdx.x] = s;
    sw[threadIdx.x] = w;
    __syncthreads();
    for (int k = blockDim.x / 2; k > 0; k >>= 1) {
        if (threadIdx.x < k) {
            ss[threadIdx.x] += ss[threadIdx.x + k];
            sw[threadIdx.x] += sw[threadIdx.x + k];
        }
        __syncthreads();
    }
    const double c = (target[b] - ss[0]) / sw[0];
    for (int i = threadIdx.x; i < nq; i += blockDim.x) p[i] = (float)((double)p[i] + c);
}

struct pf_no {
    std::vector<int> dims;                 // layer widths, dims[0] = 3
    int ng = 0, nq = 0, maxB = 0;
    int nqx = 0, nqy = 0;                  // node grid of the predictions ([y][x], x fastest)
    double *mw = nullptr;                  // mass projection: wx[nqx], wy[nqy], target[B]
    int mw_B = 0;
    cudaStream_t st = nullptr;
    // parameters: per layer W (dims[l] x dims[l+1]) then b (dims[l+1]), one flat FP32 master array
    std::vector<long long> woff, boff;
    long long nparam = 0;
    float *w = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;
    __nv_bfloat16 *wb = nullptr;
    std::vector<__nv_bfloat16 *> wt;       // per layer: BF16 weights transposed for the tensor cores (or null)
    int *err = nullptr;                    // device error word of the tensor-core layers (bounded waits)
    float *mean = nullptr, *istd = nullptr;
    int *ridx = nullptr, *rp = nullptr, *rc = nullptr;
    float *rw = nullptr, *rv = nullptr;
    std::vector<float *> act, dact;        // activations per layer (B x dims[l])
    float *pn = nullptr, *dn = nullptr;    // predictions and their gradient at the nodes
    float *feat = nullptr, *targ = nullptr, *bf = nullptr, *bt = nullptr;
    int *rows = nullptr;
    long long nsample_dev = 0;
    double *part = nullptr;
    long long adam_t = 0;
    std::vector<void *> allocs;
    ~pf_no() {
        for (void *p : allocs) cudaFree(p);
    }
    template <typename T>
    T *mk(size_t n) {
        T *p = nullptr;
        NO_CU(cudaMalloc(&p, std::max<size_t>(n, 1) * sizeof(T)));
        NO_CU(cudaMemset(p, 0, std::max<size_t>(n, 1) * sizeof(T)));
        allocs.push_back(p);
        return p;
    }
};

namespace {

void ensure_batch(pf_no *h, int B) {
    if (B <= h->maxB) return;
    h->act.clear();
    h->dact.clear();
    for (size_t l = 0; l < h->dims.size(); ++l) {
        h->act.push_back(h->mk<float>((size_t)B * h->dims[l]));
        h->dact.push_back(h->mk<float>((size_t)B * h->dims[l]));
    }
    h->pn = h->mk<float>((size_t)B * h->nq);
    h->dn = h->mk<float>((size_t)B * h->nq);
    h->bt = h->mk<float>((size_t)B * h->nq);
    h->rows = h->mk<int>(B);
    h->maxB = B;
}

// layers on the tensor cores: hidden and output layers with K a multiple of 64 up to 384 and N a
// multiple of 128 (the first layer standardises its 3 inputs on the CUDA cores)
bool tc_layer(const pf_no *h, int l) {
    const int K = h->dims[l], N = h->dims[l + 1];
    return l > 0 && K % 64 == 0 && K <= 384 && N % 128 == 0;
}
size_t tc_smem(int K) { return 1024 + (size_t)128 * K * 2 + (size_t)2 * NO_TC_BN * K * 2 + 64; }

// the transposed BF16 copies of the tensor-core layers' weights, after every change of wb
void refresh_wt(pf_no *h) {
    for (int l = 0; l + 1 < (int)h->dims.size(); ++l)
        if (h->wt[l]) {
            const int K = h->dims[l], N = h->dims[l + 1];
            k_transpose_bf16<<<dim3((N + 31) / 32, (K + 31) / 32), dim3(32, 8), 0, h->st>>>(h->wb + h->woff[l], h->wt[l],
                                                                                           K, N);
            NO_CU(cudaGetLastError());
        }
}

// forward from h->act[0] (B x 3 raw features) to h->pn (B x nq)
void forward(pf_no *h, int B) {
    const int L = (int)h->dims.size() - 1;
    for (int l = 0; l < L; ++l) {
        const int K = h->dims[l], N = h->dims[l + 1];
        if (h->wt[l]) {
            k_dense_fwd_tc<<<dim3(N / 128, (B + NO_TC_BN - 1) / NO_TC_BN), 128, tc_smem(K), h->st>>>(
                h->act[l], h->wt[l], h->w + h->boff[l], h->act[l + 1], B, K, N, h->err);
            NO_CU(cudaGetLastError());
            continue;
        }
        dim3 grid((N + 127) / 128, B);
        k_dense_fwd<<<grid, 128, 0, h->st>>>(h->act[l], h->wb + h->woff[l], h->w + h->boff[l], h->act[l + 1], B, K, N,
                                             l == 0 ? h->mean : nullptr, l == 0 ? h->istd : nullptr);
        NO_CU(cudaGetLastError());
    }
    k_resample<<<dim3((h->nq + 127) / 128, B), 128, 0, h->st>>>(h->act[L], h->ridx, h->rw, h->pn, B, h->ng, h->nq);
    NO_CU(cudaGetLastError());
}

// loss against targets tgt (device, B x nq) and the gradient of every parameter into h->g
double backward(pf_no *h, int B, const float *tgt) {
    const int L = (int)h->dims.size() - 1;
    const long long n = (long long)B * h->nq;
    k_loss<<<256, 256, 0, h->st>>>(h->pn, tgt, h->dn, n, 1.f / (float)n, h->part);
    NO_CU(cudaGetLastError());
    k_resample_t<<<dim3((h->ng + 127) / 128, B), 128, 0, h->st>>>(h->dn, h->rp, h->rc, h->rv, h->dact[L], B, h->ng,
                                                                  h->nq);
    NO_CU(cudaGetLastError());
    for (int l = L - 1; l >= 0; --l) {
        const int K = h->dims[l], N = h->dims[l + 1];
        const long long nz = (long long)B * N;
        k_tanh_back<<<(unsigned)((nz + 255) / 256), 256, 0, h->st>>>(h->act[l + 1], h->dact[l + 1], nz);
        NO_CU(cudaGetLastError());
        k_dense_bwd_w<<<dim3((N + 127) / 128, K), 128, 0, h->st>>>(h->act[l], h->dact[l + 1], h->g + h->woff[l],
                                                                    h->g + h->boff[l], B, K, N,
                                                                    l == 0 ? h->mean : nullptr,
                                                                    l == 0 ? h->istd : nullptr);
        NO_CU(cudaGetLastError());
        if (l > 0) {
            const long long warps = (long long)B * K;
            k_dense_bwd_x<<<(unsigned)((warps * 32 + 255) / 256), 256, 0, h->st>>>(h->dact[l + 1], h->wb + h->woff[l],
                                                                                   h->dact[l], B, K, N);
            NO_CU(cudaGetLastError());
        }
    }
    std::vector<double> part(256);
    NO_CU(cudaMemcpyAsync(part.data(), h->part, 256 * sizeof(double), cudaMemcpyDeviceToHost, h->st));
    NO_CU(cudaStreamSynchronize(h->st));
    double s = 0.0;
    for (double v : part) s += v;
    return s / (double)n;
}

void adam(pf_no *h, double lr) {
    h->adam_t += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - std::pow(b1, (float)h->adam_t), c2 = 1.f - std::pow(b2, (float)h->adam_t);
    k_adam<<<(unsigned)((h->nparam + 255) / 256), 256, 0, h->st>>>(h->w, h->wb, h->g, h->m, h->v, h->nparam, (float)lr,
                                                                   b1, b2, c1, c2, 1e-8f);
    NO_CU(cudaGetLastError());
    refresh_wt(h);
}

int no_fail(int code, const std::string &m) {
    pf_internal_set_error(m);
    return code;
}

// the tensor-core layers' error word after a synchronised call: PF_ETIMEOUT (and cleared) when a
// bounded wait gave up
int tc_status(pf_no *h) {
    int e = 0;
    if (cudaMemcpy(&e, h->err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) {
        cudaGetLastError();
        return no_fail(PF_ECUDA, "pf_no: reading the error word");
    }
    if (e == 0) return PF_OK;
    cudaMemset(h->err, 0, sizeof(int));
    return no_fail(PF_ETIMEOUT, "pf_no: a tensor-core layer's bounded wait gave up");
}

void upload_features(pf_no *h, int B, const double *feat) {
    std::vector<float> f((size_t)B * h->dims[0]);
    for (size_t i = 0; i < f.size(); ++i) f[i] = (float)feat[i];
    NO_CU(cudaMemcpyAsync(h->act[0], f.data(), f.size() * 4, cudaMemcpyHostToDevice, h->st));
    NO_CU(cudaStreamSynchronize(h->st));
}

}  // namespace

extern "C" int pf_no_create(int nlayer, const int *dims, const double *feat_mean, const double *feat_std, int gnx,
                            int gny, double x0, double x1, double y0, double y1, int nqx, int nqy,
                            const double *node_x, const double *node_y, uint64_t seed, void *cuda_stream,
                            pf_no **out) {
    if (out) *out = nullptr;
    if (nlayer < 2 || !dims || !feat_mean || !feat_std || gnx < 2 || gny < 2 || nqx < 1 || nqy < 1 || !node_x ||
        !node_y || !out || !(x1 > x0) || !(y1 > y0))
        return no_fail(PF_EINVAL, "pf_no_create: bad arguments");
    for (int l = 0; l < nlayer; ++l)
        if (dims[l] < 1) return no_fail(PF_EINVAL, "pf_no_create: layer widths must be positive");
    if (dims[nlayer - 1] != gnx * gny) return no_fail(PF_EINVAL, "pf_no_create: output width must be gnx*gny");
    std::unique_ptr<pf_no> h(new pf_no());
    try {
        h->dims.assign(dims, dims + nlayer);
        h->st = (cudaStream_t)cuda_stream;
        h->ng = gnx * gny;
        h->nq = nqx * nqy;
        h->nqx = nqx;
        h->nqy = nqy;
        long long off = 0;
        for (int l = 0; l + 1 < nlayer; ++l) {
            h->woff.push_back(off);
            off += (long long)dims[l] * dims[l + 1];
            h->boff.push_back(off);
            off += dims[l + 1];
        }
        h->nparam = off;
        // Glorot-uniform initial weights, zero biases (seeded)
        std::vector<float> w(off, 0.f);
        std::mt19937_64 rng(seed);
        for (int l = 0; l + 1 < nlayer; ++l) {
            const double a = std::sqrt(6.0 / (dims[l] + dims[l + 1]));
            std::uniform_real_distribution<double> U(-a, a);
            for (long long i = 0; i < (long long)dims[l] * dims[l + 1]; ++i) w[h->woff[l] + i] = (float)U(rng);
        }
        h->w = h->mk<float>(off);
        h->g = h->mk<float>(off);
        h->m = h->mk<float>(off);
        h->v = h->mk<float>(off);
        h->wb = h->mk<__nv_bfloat16>(off);
        NO_CU(cudaMemcpy(h->w, w.data(), off * 4, cudaMemcpyHostToDevice));
        k_to_bf16<<<(unsigned)((off + 255) / 256), 256>>>(h->w, h->wb, off);
        NO_CU(cudaGetLastError());
        NO_CU(cudaDeviceSynchronize());
        h->err = h->mk<int>(1);
        h->wt.assign(nlayer - 1, nullptr);
        int kmax = 0;
        for (int l = 0; l + 1 < nlayer; ++l)
            if (tc_layer(h.get(), l)) {
                h->wt[l] = h->mk<__nv_bfloat16>((size_t)dims[l] * dims[l + 1]);
                kmax = std::max(kmax, dims[l]);
            }
        if (kmax > 0)
            NO_CU(cudaFuncSetAttribute(k_dense_fwd_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc_smem(kmax)));
        refresh_wt(h.get());
        NO_CU(cudaStreamSynchronize(h->st));
        std::vector<float> mu(dims[0]), is(dims[0]);
        for (int k = 0; k < dims[0]; ++k) {
            mu[k] = (float)feat_mean[k];
            is[k] = (float)(1.0 / (feat_std[k] > 0 ? feat_std[k] : 1.0));
        }
        h->mean = h->mk<float>(dims[0]);
        h->istd = h->mk<float>(dims[0]);
        NO_CU(cudaMemcpy(h->mean, mu.data(), dims[0] * 4, cudaMemcpyHostToDevice));
        NO_CU(cudaMemcpy(h->istd, is.data(), dims[0] * 4, cudaMemcpyHostToDevice));
        // bilinear map from the grid (x periodic, cell starts x0 + i Lx/gnx; y from y0 to y1) to the nodes
        std::vector<int> idx((size_t)h->nq * 4);
        std::vector<float> wt((size_t)h->nq * 4);
        const double Lx = x1 - x0, Ly = y1 - y0;
        for (int qy = 0; qy < nqy; ++qy)
            for (int qx = 0; qx < nqx; ++qx) {
                const int q = qy * nqx + qx;
                double fx = (node_x[qx] - x0) / Lx * gnx;
                double fl = std::floor(fx);
                const double wx = fx - fl;
                int i0 = ((int)fl % gnx + gnx) % gnx, i1 = (i0 + 1) % gnx;
                double fy = (node_y[qy] - y0) / Ly * (gny - 1);
                int j0 = (int)std::floor(fy);
                if (j0 < 0) j0 = 0;
                if (j0 > gny - 2) j0 = gny - 2;
                const double wy = fy - j0;
                const int id[4] = {j0 * gnx + i0, j0 * gnx + i1, (j0 + 1) * gnx + i0, (j0 + 1) * gnx + i1};
                const double ww[4] = {(1 - wx) * (1 - wy), wx * (1 - wy), (1 - wx) * wy, wx * wy};
                for (int c = 0; c < 4; ++c) {
                    idx[q * 4 + c] = id[c];
                    wt[q * 4 + c] = (float)ww[c];
                }
            }
        // transpose in CSR by grid point (fixed order: node, then corner)
        std::vector<int> rp(h->ng + 1, 0), col((size_t)h->nq * 4);
        std::vector<float> val((size_t)h->nq * 4);
        for (int q = 0; q < h->nq; ++q)
            for (int c = 0; c < 4; ++c) rp[idx[q * 4 + c] + 1] += 1;
        for (int i = 0; i < h->ng; ++i) rp[i + 1] += rp[i];
        std::vector<int> fill(rp.begin(), rp.end() - 1);
        for (int q = 0; q < h->nq; ++q)
            for (int c = 0; c < 4; ++c) {
                const int i = idx[q * 4 + c];
                col[fill[i]] = q;
                val[fill[i]] = wt[q * 4 + c];
                fill[i] += 1;
            }
        h->ridx = h->mk<int>(idx.size());
        h->rw = h->mk<float>(wt.size());
        h->rp = h->mk<int>(rp.size());
        h->rc = h->mk<int>(col.size());
        h->rv = h->mk<float>(val.size());
        NO_CU(cudaMemcpy(h->ridx, idx.data(), idx.size() * 4, cudaMemcpyHostToDevice));
        NO_CU(cudaMemcpy(h->rw, wt.data(), wt.size() * 4, cudaMemcpyHostToDevice));
        NO_CU(cudaMemcpy(h->rp, rp.data(), rp.size() * 4, cudaMemcpyHostToDevice));
        NO_CU(cudaMemcpy(h->rc, col.data(), col.size() * 4, cudaMemcpyHostToDevice));
        NO_CU(cudaMemcpy(h->rv, val.data(), val.size() * 4, cudaMemcpyHostToDevice));
        h->part = h->mk<double>(256);
        ensure_batch(h.get(), 64);
        NO_CU(cudaDeviceSynchronize());
    } catch (const NoErr &e) {
        return no_fail(e.code == cudaErrorMemoryAllocation ? PF_ENOMEM : PF_ECUDA,
                       e.where + ": " + cudaGetErrorString(e.code));
    }
    *out = h.release();
    return PF_OK;
}

extern "C" long long pf_no_param_count(const pf_no *h) { return h ? h->nparam : (long long)PF_EINVAL; }

extern "C" int pf_no_get_params(pf_no *h, double *host, size_t n) {
    if (!h || !host || n < (size_t)h->nparam) return no_fail(PF_EINVAL, "pf_no_get_params: bad arguments");
    std::vector<float> w(h->nparam);
    try {
        NO_CU(cudaStreamSynchronize(h->st));
        NO_CU(cudaMemcpy(w.data(), h->w, h->nparam * 4, cudaMemcpyDeviceToHost));
    } catch (const NoErr &e) {
        return no_fail(PF_ECUDA, e.where + ": " + cudaGetErrorString(e.code));
    }
    for (long long i = 0; i < h->nparam; ++i) host[i] = w[i];
    return PF_OK;
}

extern "C" int pf_no_set_params(pf_no *h, const double *host, size_t n) {
    if (!h || !host || n < (size_t)h->nparam) return no_fail(PF_EINVAL, "pf_no_set_params: bad arguments");
    std::vector<float> w(h->nparam);
    for (long long i = 0; i < h->nparam; ++i) w[i] = (float)host[i];
    try {
        NO_CU(cudaMemcpyAsync(h->w, w.data(), h->nparam * 4, cudaMemcpyHostToDevice, h->st));
        k_to_bf16<<<(unsigned)((h->nparam + 255) / 256), 256, 0, h->st>>>(h->w, h->wb, h->nparam);
        NO_CU(cudaGetLastError());
        refresh_wt(h);
        NO_CU(cudaGetLastError());
        NO_CU(cudaStreamSynchronize(h->st));
    } catch (const NoErr &e) {
        return no_fail(PF_ECUDA, e.where + ": " + cudaGetErrorString(e.code));
    }
    return PF_OK;
}

extern "C" int pf_no_predict(pf_no *h, int B, const double *feat, double *phi_nodes) {
    if (!h || B < 1 || !feat || !phi_nodes) return no_fail(PF_EINVAL, "pf_no_predict: bad arguments");
    try {
        ensure_batch(h, B);
        upload_features(h, B, feat);
        forward(h, B);
        std::vector<float> p((size_t)B * h->nq);
        NO_CU(cudaMemcpyAsync(p.data(), h->pn, p.size() * 4, cudaMemcpyDeviceToHost, h->st));
        NO_CU(cudaStreamSynchronize(h->st));
        for (size_t i = 0; i < p.size(); ++i) phi_nodes[i] = p[i];
    } catch (const NoErr &e) {
        return no_fail(PF_ECUDA, e.where + ": " + cudaGetErrorString(e.code));
    }
    return tc_status(h);
}

extern "C" int pf_no_predict_mass(pf_no *h, int B, const double *feat, const double *mass, const double *wx,
                                  const double *wy, double *phi_nodes) {
    if (!h || B < 1 || !feat || !mass || !wx || !wy || !phi_nodes)
        return no_fail(PF_EINVAL, "pf_no_predict_mass: bad arguments");
    try {
        ensure_batch(h, B);
        upload_features(h, B, feat);
        forward(h, B);
        if (B > h->mw_B) {
            h->mw = h->mk<double>((size_t)h->nqx + h->nqy + B);
            h->mw_B = B;
        }
        NO_CU(cudaMemcpyAsync(h->mw, wx, h->nqx * sizeof(double), cudaMemcpyHostToDevice, h->st));
        NO_CU(cudaMemcpyAsync(h->mw + h->nqx, wy, h->nqy * sizeof(double), cudaMemcpyHostToDevice, h->st));
        NO_CU(cudaMemcpyAsync(h->mw + h->nqx + h->nqy, mass, B * sizeof(double), cudaMemcpyHostToDevice, h->st));
        k_mass_shift<<<B, 256, 0, h->st>>>(h->pn, h->nqx, h->nqy, h->mw, h->mw + h->nqx, h->mw + h->nqx + h->nqy);
        NO_CU(cudaGetLastError());
        std::vector<float> p((size_t)B * h->nq);
        NO_CU(cudaMemcpyAsync(p.data(), h->pn, p.size() * 4, cudaMemcpyDeviceToHost, h->st));
        NO_CU(cudaStreamSynchronize(h->st));
        for (size_t i = 0; i < p.size(); ++i) phi_nodes[i] = p[i];
    } catch (const NoErr &e) {
        return no_fail(PF_ECUDA, e.where + ": " + cudaGetErrorString(e.code));
    }
    return tc_status(h);
}

extern "C" int pf_no_loss_grad(pf_no *h, int B, const double *feat, const double *target, double *loss,
                               double *grad) {
    if (!h || B < 1 || !feat || !target || !loss) return no_fail(PF_EINVAL, "pf_no_loss_grad: bad arguments");
    try {
        ensure_batch(h, B);
        upload_features(h, B, feat);
        std::vector<float> t((size_t)B * h->nq);
        for (size_t i = 0; i < t.size(); ++i) t[i] = (float)target[i];
        NO_CU(cudaMemcpyAsync(h->bt, t.data(), t.size() * 4, cudaMemcpyHostToDevice, h->st));
        forward(h, B);
        *loss = backward(h, B, h->bt);
        if (grad) {
            std::vector<float> g(h->nparam);
            NO_CU(cudaMemcpyAsync(g.data(), h->g, h->nparam * 4, cudaMemcpyDeviceToHost, h->st));
            NO_CU(cudaStreamSynchronize(h->st));
            for (long long i = 0; i < h->nparam; ++i) grad[i] = g[i];
        }
    } catch (const NoErr &e) {
        return no_fail(PF_ECUDA, e.where + ": " + cudaGetErrorString(e.code));
    }
    return tc_status(h);
}

extern "C" int pf_no_train(pf_no *h, int nsample, const double *feat, const double *target, int batch, int epochs,
                           double lr, uint64_t seed, double *loss_per_epoch) {
    if (!h || nsample < 1 || !feat || !target || batch < 1 || epochs < 0)
        return no_fail(PF_EINVAL, "pf_no_train: bad arguments");
    try {
        const int F = h->dims[0];
        ensure_batch(h, batch);
        if (nsample > h->nsample_dev) {
            h->feat = h->mk<float>((size_t)nsample * F);
            h->targ = h->mk<float>((size_t)nsample * h->nq);
            h->bf = h->mk<float>((size_t)batch * F);
            h->nsample_dev = nsample;
        }
        std::vector<float> f((size_t)nsample * F), t((size_t)nsample * h->nq);
        for (size_t i = 0; i < f.size(); ++i) f[i] = (float)feat[i];
        for (size_t i = 0; i < t.size(); ++i) t[i] = (float)target[i];
        NO_CU(cudaMemcpyAsync(h->feat, f.data(), f.size() * 4, cudaMemcpyHostToDevice, h->st));
        NO_CU(cudaMemcpyAsync(h->targ, t.data(), t.size() * 4, cudaMemcpyHostToDevice, h->st));
        std::mt19937_64 rng(seed);
        std::vector<int> order(nsample);
        for (int i = 0; i < nsample; ++i) order[i] = i;
        for (int ep = 0; ep < epochs; ++ep) {
            std::shuffle(order.begin(), order.end(), rng);
            double lsum = 0.0;
            int nb = 0;
            for (int s0 = 0; s0 + batch <= nsample; s0 += batch) {
                NO_CU(cudaMemcpyAsync(h->rows, order.data() + s0, batch * sizeof(int), cudaMemcpyHostToDevice, h->st));
                k_gather_rows<<<dim3((F + 127) / 128, batch), 128, 0, h->st>>>(h->feat, h->rows, h->act[0], batch, F);
                k_gather_rows<<<dim3((h->nq + 127) / 128, batch), 128, 0, h->st>>>(h->targ, h->rows, h->bt, batch, h->nq);
                NO_CU(cudaGetLastError());
                forward(h, batch);
                lsum += backward(h, batch, h->bt);
                adam(h, lr);
                ++nb;
            }
            if (loss_per_epoch) loss_per_epoch[ep] = nb ? lsum / nb : 0.0;
        }
        NO_CU(cudaStreamSynchronize(h->st));
    } catch (const NoErr &e) {
        return no_fail(PF_ECUDA, e.where + ": " + cudaGetErrorString(e.code));
    }
    return tc_status(h);
}

extern "C" void pf_no_destroy(pf_no *h) {
    if (!h) return;
    if (h->st) cudaStreamSynchronize(h->st);
    delete h;
}
