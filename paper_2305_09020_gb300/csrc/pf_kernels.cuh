// CUDA kernels of the per-step path (sm_103a), templated on the working precision T.
//
// Data layout in HBM
//   nodal fields  [z][y][x]            n2 = n_y * n_x values per plane, x fastest
//   element-local [z][ey][ex][b][a]    (K+1)^2 slots per element (discontinuous data,
//                                      weak-form contributions before direct
//                                      stiffness summation)
//   mode planes   [p][y][x]            real FFT along z packed into Nz real planes:
//                                      p = 0: Re(k = 0), p = 1: Re(k = Nz/2),
//                                      p = 2k: Re(k), p = 2k+1: Im(k), 0 < k < Nz/2
//
// Kernels
//   k_potential  RHS of eq. 54a/74a (weak form of the variable-permittivity correction)
//   k_efield     E = M^{-1} (assembled weighted derivative of V), eq. 55/78
//   k_chem       Q1, Q2 and the psi right-hand side, eq. 56/75
//   k_momentum   T, G (eq. 49), the pressure RHS (eq. 58/77) and the velocity RHS
//                except its new-pressure term (eq. 59/78)
//   k_ugradp     the -(1/(nu_m rho0)) grad P^{n+1} term of eq. 59/78
//   k_fwd        direct stiffness summation + z real FFT + (A + m_k B) combination,
//                scaling and Dirichlet lifting  -> mode-plane right-hand sides
//   k_inv        inverse z FFT of a mode-plane solution (value and d/dz), Dirichlet
//                values; variant for phi that also forms psi - alpha phi combinations
//   k_gemm       C = A B with a small shared B (fast-diagonalisation transforms) and
//                an epilogue that divides by the eigenvalue sum, stores transposed, or also
//                writes -M C (the phi right-hand side of eq. 57 / 76 from psi)
//   reductions   FP64 phase mass, max |u|, max |difference|
#pragma once

#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace pf {

template <typename T>
struct cplx {
    T x, y;
};

template <typename T>
__device__ __forceinline__ cplx<T> cmul(cplx<T> a, cplx<T> b) {
    return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}

template <typename T>
struct Geo {
    int ex, ey, K, p, nx, ny, n2, nz;
    int epb;            // elements per block of the element kernels
    const T *hx, *hy;   // element sizes
    const T *D;         // D[a*p+m] = l_m'(xi_a)
    const T *Dw;        // Dw[a*p+c] = w_a D[a*p+c]
    const T *w;         // GLL weights
    const T *Mx, *My;   // assembled 1D masses
    const int *active;  // ensembles: per-plane (run) flag, 0 = frozen (its step is skipped); else null
};

// a frozen ensemble run (blockIdx.y = plane): its element and transform work is skipped
template <typename T>
__device__ __forceinline__ bool plane_frozen(const Geo<T> &G) {
    return G.active && !G.active[blockIdx.y];
}

template <typename T>
struct Phys {
    T rho1, rho2, mu1, mu2, eps1, eps2;
    T lam, inv_eta2, gamma1, S_eta2, eps0, rho0, nu_m, dt, sigma, cos_theta;
    T alpha, gamma0;
    int J;
    int wetting;   // theta_s != 90 degrees
    const T *eps1_p, *eps2_p, *eps0_p;   // per-plane permittivities of an ensemble (nullable)
};

// an ensemble plane (blockIdx.y) may carry its own permittivities
template <typename T>
__device__ __forceinline__ Phys<T> plane_phys(const Phys<T> &q) {
    Phys<T> r = q;
    if (q.eps1_p) {
        r.eps1 = q.eps1_p[blockIdx.y];
        r.eps2 = q.eps2_p[blockIdx.y];
        r.eps0 = q.eps0_p[blockIdx.y];
    }
    return r;
}

// ---- mixture laws (eq. interpolation) and free-energy pieces (Sec. 2.1) -------------------
template <typename T> __device__ __forceinline__ T rho_of(const Phys<T> &q, T phi) {
    return T(0.5) * (q.rho1 + q.rho2) + T(0.5) * (q.rho1 - q.rho2) * phi;
}
template <typename T> __device__ __forceinline__ T mu_of(const Phys<T> &q, T phi) {
    return T(0.5) * (q.mu1 + q.mu2) + T(0.5) * (q.mu1 - q.mu2) * phi;
}
template <typename T> __device__ __forceinline__ T eps_of(const Phys<T> &q, T phi) {
    return T(0.5) * (q.eps1 + q.eps2) + T(0.5) * (q.eps1 - q.eps2) * phi * (T(3) - phi * phi) * T(0.5);
}
template <typename T> __device__ __forceinline__ T deps_of(const Phys<T> &q, T phi) {
    return T(0.5) * (q.eps2 - q.eps1) * T(3) * (phi * phi - T(1)) * T(0.5);
}
template <typename T> __device__ __forceinline__ T h_of(const Phys<T> &q, T phi) {
    return phi * (phi * phi - T(1)) * q.inv_eta2;
}
template <typename T> __device__ __forceinline__ T dtheta_of(const Phys<T> &q, T phi) {
    return q.sigma * q.cos_theta * T(3) * (phi * phi - T(1)) * T(0.25);
}
// BDF-J extrapolation xi* and the history term xi_hat (Sec. 3.1)
template <typename T> __device__ __forceinline__ T star(int J, T a, T b) { return J == 1 ? a : T(2) * a - b; }
template <typename T> __device__ __forceinline__ T hatv(int J, T a, T b) { return J == 1 ? a : T(2) * a - T(0.5) * b; }

// ---- element helpers ----------------------------------------------------------------------
struct ElemIdx {
    int ex, ey, a, b, t, z, le;
    bool act;       // this thread owns a node of an existing element
    long long g;    // global nodal index (with plane offset)
    long long l;    // element-local slot (with plane offset)
};

// Element-local arrays (weak-form contributions before direct stiffness summation) are stored
// row-interleaved, [z][e_y][b][e_x][a]: the slots of one global node row lie next to each other
// (with the duplicated element-boundary slots adjacent), so the summation's gathers coalesce.
template <typename T>
__device__ __forceinline__ long long eloc(const Geo<T> &G, long long z, int ey, int ex, int b, int a) {
    return z * ((long long)G.ex * G.ey * G.p * G.p) + ((long long)(ey * G.p + b) * G.ex + ex) * G.p + a;
}

// blockIdx.x: group of G.epb elements of plane blockIdx.y; thread = (local element, node)
template <typename T>
__device__ __forceinline__ ElemIdx elem_index(const Geo<T> &G) {
    ElemIdx e;
    const int pp = G.p * G.p;
    e.le = threadIdx.x / pp;
    e.t = threadIdx.x - e.le * pp;
    const int el = blockIdx.x * G.epb + e.le;
    e.act = e.le < G.epb && el < G.ex * G.ey;
    const int elc = e.act ? el : 0;
    e.z = blockIdx.y;
    e.ex = elc % G.ex;
    e.ey = elc / G.ex;
    e.a = e.t % G.p;
    e.b = e.t / G.p;
    int xi = e.ex * G.K + e.a;
    if (xi >= G.nx) xi -= G.nx;
    e.g = (long long)e.z * G.n2 + (long long)(e.ey * G.K + e.b) * G.nx + xi;
    e.l = eloc(G, e.z, e.ey, e.ex, e.b, e.a);
    return e;
}

// shared tables: D, Dw, w (loaded by every element kernel)
template <typename T>
__device__ __forceinline__ void load_tables(const Geo<T> &G, T *sD, T *sDw, T *sw) {
    const int pp = G.p * G.p;
    for (int i = threadIdx.x; i < pp; i += blockDim.x) {
        sD[i] = G.D[i];
        sDw[i] = G.Dw[i];
    }
    for (int i = threadIdx.x; i < G.p; i += blockDim.x) sw[i] = G.w[i];
}

// d/dx and d/dy of an element array f[b*p+a] at (a, b); scale = 2/h
template <typename T>
__device__ __forceinline__ T ddx(const T *f, const T *sD, int p, int a, int b, T sc) {
    T s = 0;
#pragma unroll
    for (int m = 0; m < p; ++m) s += sD[a * p + m] * f[b * p + m];
    return s * sc;
}
template <typename T>
__device__ __forceinline__ T ddy(const T *f, const T *sD, int p, int a, int b, T sc) {
    T s = 0;
#pragma unroll
    for (int m = 0; m < p; ++m) s += sD[b * p + m] * f[m * p + a];
    return s * sc;
}
// weak forms: int F d(l_{a'b'})/dx and int F d(l_{a'b'})/dy over the element
template <typename T>
__device__ __forceinline__ T wdx(const T *F, const T *sDw, const T *sw, int p, int a, int b, T hy2) {
    T s = 0;
#pragma unroll
    for (int m = 0; m < p; ++m) s += sDw[m * p + a] * F[b * p + m];
    return s * hy2 * sw[b];
}
template <typename T>
__device__ __forceinline__ T wdy(const T *F, const T *sDw, const T *sw, int p, int a, int b, T hx2) {
    T s = 0;
    for (int m = 0; m < p; ++m) s += sDw[m * p + b] * F[m * p + a];
    return s * hx2 * sw[a];
}

// The same derivatives of NF element arrays at once: each coefficient is loaded from shared
// memory once for all NF fields (the sums per field are those of ddx/ddy/wdx/wdy, term by term)
template <int NF, typename T>
__device__ __forceinline__ void ddx_n(const T *const (&f)[NF], const T *sD, int p, int a, int b, T sc, T (&out)[NF]) {
    T s[NF];
#pragma unroll
    for (int i = 0; i < NF; ++i) s[i] = 0;
#pragma unroll
    for (int m = 0; m < p; ++m) {
        const T d = sD[a * p + m];
#pragma unroll
        for (int i = 0; i < NF; ++i) s[i] += d * f[i][b * p + m];
    }
#pragma unroll
    for (int i = 0; i < NF; ++i) out[i] = s[i] * sc;
}
template <int NF, typename T>
__device__ __forceinline__ void ddy_n(const T *const (&f)[NF], const T *sD, int p, int a, int b, T sc, T (&out)[NF]) {
    T s[NF];
#pragma unroll
    for (int i = 0; i < NF; ++i) s[i] = 0;
#pragma unroll
    for (int m = 0; m < p; ++m) {
        const T d = sD[b * p + m];
#pragma unroll
        for (int i = 0; i < NF; ++i) s[i] += d * f[i][m * p + a];
    }
#pragma unroll
    for (int i = 0; i < NF; ++i) out[i] = s[i] * sc;
}
template <int NF, typename T>
__device__ __forceinline__ void wdx_n(const T *const (&F)[NF], const T *sDw, const T *sw, int p, int a, int b, T hy2,
                                      T (&out)[NF]) {
    T s[NF];
#pragma unroll
    for (int i = 0; i < NF; ++i) s[i] = 0;
#pragma unroll
    for (int m = 0; m < p; ++m) {
        const T d = sDw[m * p + a];
#pragma unroll
        for (int i = 0; i < NF; ++i) s[i] += d * F[i][b * p + m];
    }
#pragma unroll
    for (int i = 0; i < NF; ++i) out[i] = s[i] * hy2 * sw[b];
}
template <int NF, typename T>
__device__ __forceinline__ void wdy_n(const T *const (&F)[NF], const T *sDw, const T *sw, int p, int a, int b, T hx2,
                                      T (&out)[NF]) {
    T s[NF];
#pragma unroll
    for (int i = 0; i < NF; ++i) s[i] = 0;
#pragma unroll
    for (int m = 0; m < p; ++m) {
        const T d = sDw[m * p + b];
#pragma unroll
        for (int i = 0; i < NF; ++i) s[i] += d * F[i][m * p + a];
    }
#pragma unroll
    for (int i = 0; i < NF; ++i) out[i] = s[i] * hx2 * sw[a];
}

// shared memory: D, Dw, w tables, then nfields element arrays per local element
// The element order fixed at compile time (KC > 0; KC = 0 keeps the run's order): loops over the
// K + 1 nodes of an element unroll and slot arithmetic folds.  epb follows the host's choice.
template <int KC, typename T>
__device__ __forceinline__ Geo<T> fixed_order(Geo<T> g) {
    if constexpr (KC > 0) {
        g.K = KC;
        g.p = KC + 1;
        g.epb = 256 / ((KC + 1) * (KC + 1)) > 1 ? 256 / ((KC + 1) * (KC + 1)) : 1;
    }
    return g;
}

#define PF_ELEM_SMEM(T, G, nfields)                                                   \
    extern __shared__ unsigned char pf_smem_raw[];                                    \
    T *sD = reinterpret_cast<T *>(pf_smem_raw);                                       \
    T *sDw = sD + (G).p * (G).p;                                                      \
    T *sw = sDw + (G).p * (G).p;                                                      \
    const int pp_ = (G).p * (G).p;                                                    \
    const int le_ = min((int)(threadIdx.x / pp_), (G).epb - 1);                      \
    T *sF = sw + 32 + le_ * (nfields) * pp_;

// ---- eq. 54a / 74a: RHS of the potential --------------------------------------------------
// A = -int R_2D . grad_2D w  (element-local contributions),  B = int R_z w  (iB multiplier)
// with R = (eps(phi*) - eps0) grad V*.
template <typename T, int KC = 0>
__global__ void k_potential(Geo<T> G_, Phys<T> q_, const T *__restrict__ phin, const T *__restrict__ phio,
                            const T *__restrict__ Vn, const T *__restrict__ Vo, const T *__restrict__ Ezn,
                            const T *__restrict__ Ezo, T *__restrict__ A, T *__restrict__ B) {
    if (plane_frozen(G_)) return;
    const Geo<T> G = fixed_order<KC>(G_);
    PF_ELEM_SMEM(T, G, 3)
    const Phys<T> q = plane_phys(q_);
    T *sV = sF, *sRx = sF + pp_, *sRy = sF + 2 * pp_;
    load_tables(G, sD, sDw, sw);
    const ElemIdx e = elem_index(G);
    const bool act = e.act;
    const T hx = G.hx[e.ex], hy = G.hy[e.ey];
    T phis = 0, Vs = 0;
    if (act) {
        phis = star(q.J, phin[e.g], phio[e.g]);
        Vs = star(q.J, Vn[e.g], Vo[e.g]);
        sV[e.t] = Vs;
    }
    __syncthreads();
    T c = 0;
    if (act) {
        c = eps_of(q, phis) - q.eps0;
        sRx[e.t] = c * ddx(sV, sD, G.p, e.a, e.b, T(2) / hx);
        sRy[e.t] = c * ddy(sV, sD, G.p, e.a, e.b, T(2) / hy);
    }
    __syncthreads();
    if (!act) return;
    const T hx2 = T(0.5) * hx, hy2 = T(0.5) * hy;
    A[e.l] = -(wdx(sRx, sDw, sw, G.p, e.a, e.b, hy2) + wdy(sRy, sDw, sw, G.p, e.a, e.b, hx2));
    if (B) {
        const T Ez = star(q.J, Ezn[e.g], Ezo[e.g]);
        B[e.l] = hx2 * hy2 * sw[e.a] * sw[e.b] * c * Ez;
    }
}

// ---- eq. 55 / 78: E_x, E_y = M^{-1} * sum over elements of M_e * (element derivative of V)
// On a tensor mesh the y (resp. x) factors of M_e cancel, leaving a 1D weighted average.
template <typename T, int KC = 0>
__global__ void k_efield(Geo<T> G_, const T *__restrict__ V, T *__restrict__ Ex, T *__restrict__ Ey) {
    const Geo<T> G = fixed_order<KC>(G_);
    const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long tot = (long long)G.n2 * G.nz;
    if (gid >= tot) return;
    const int z = (int)(gid / G.n2);
    const int q = (int)(gid % G.n2);
    const int i = q / G.nx, j = q % G.nx;
    const T *Vp = V + (long long)z * G.n2;
    const int p = G.p, K = G.K;
    // x: elements containing column j
    T sx = 0;
    {
        int exs[2], as[2], ne = 0;
        if (j % K == 0) {
            exs[ne] = j / K; as[ne++] = 0;
            exs[ne] = (j / K - 1 + G.ex) % G.ex; as[ne++] = K;
        } else {
            exs[ne] = j / K; as[ne++] = j % K;
        }
        for (int c = 0; c < ne; ++c) {
            T s = 0;
            for (int m = 0; m < p; ++m) {
                int xm = exs[c] * K + m;
                if (xm >= G.nx) xm -= G.nx;
                s += G.D[as[c] * p + m] * Vp[i * G.nx + xm];
            }
            sx += G.w[as[c]] * s;
        }
    }
    T sy = 0;
    {
        int eys[2], bs[2], ne = 0;
        if (i % K == 0) {
            if (i > 0) { eys[ne] = i / K - 1; bs[ne++] = K; }
            if (i < G.ny - 1) { eys[ne] = i / K; bs[ne++] = 0; }
        } else {
            eys[ne] = i / K; bs[ne++] = i % K;
        }
        for (int c = 0; c < ne; ++c) {
            T s = 0;
            for (int m = 0; m < p; ++m) s += G.D[bs[c] * p + m] * Vp[(eys[c] * K + m) * G.nx + j];
            sy += G.w[bs[c]] * s;
        }
    }
    Ex[gid] = sx / G.Mx[j];
    Ey[gid] = sy / G.My[i];
}

// The same E_x, E_y (eq. 55 / 78) for FP32 runs of a compiled order: one block per element row
// e_y and plane.  A thread takes a whole element segment of a node row (x) or a whole element
// column (y), so that the derivative weights are the same in every thread and come from the
// kernel's parameters: K + 1 (2K + 2 at element boundaries) values per K nodes instead of up to
// 4(K + 1) loads per node.  The node rows of the block are staged in shared memory; E_x goes
// through shared memory so that its global stores coalesce.  A block has one thread per node
// column (n_x rounded up to a warp, at most 1024), so both passes take about one round.  Same
// sums in the same order as k_efield.
template <int KC>
struct DTab {
    float d[(KC + 1) * (KC + 1)];   // D[a (K+1) + m]
    float w[KC + 1];                // GLL weights
};

template <int KC>
__global__ void __launch_bounds__(1024) k_efield_rows(Geo<float> G_, DTab<KC> t, const float *__restrict__ V,
                                                     float *__restrict__ Ex, float *__restrict__ Ey) {
    constexpr int K = KC, P = KC + 1;
    const Geo<float> G = fixed_order<KC>(G_);
    extern __shared__ __align__(16) unsigned char pf_smem_raw[];
    float *sV = reinterpret_cast<float *>(pf_smem_raw);
    const int nx = G.nx, ey = blockIdx.x, r0 = ey * K;
    const int nr = (ey == G.ey - 1) ? K + 1 : K;   // node rows r0 .. r0 + nr - 1 (the top one once)
    float *sE = sV + P * nx;
    const float *Vp = V + (long long)blockIdx.y * G.n2;
    for (int i = threadIdx.x; i < nr * nx; i += blockDim.x) sV[i] = Vp[(long long)r0 * nx + i];
    // y: one element column per thread (element e_y, and e_y - 1 for the shared bottom row)
    for (int j = threadIdx.x; j < nx; j += blockDim.x) {
        float c[P], cl[P];
#pragma unroll
        for (int m = 0; m < P; ++m) c[m] = Vp[(long long)(r0 + m) * nx + j];
        if (ey > 0) {
#pragma unroll
            for (int m = 0; m < P; ++m) cl[m] = Vp[(long long)(r0 - K + m) * nx + j];
        }
        float *Eyp = Ey + (long long)blockIdx.y * G.n2 + j;
#pragma unroll
        for (int b = 0; b < P; ++b) {
            if (b == K && ey != G.ey - 1) break;
            float sy = 0.f;
            if (b == 0 && ey > 0) {
                float s = 0.f;
#pragma unroll
                for (int m = 0; m < P; ++m) s += t.d[K * P + m] * cl[m];
                sy += t.w[K] * s;
            }
            float s = 0.f;
#pragma unroll
            for (int m = 0; m < P; ++m) s += t.d[b * P + m] * c[m];
            sy += t.w[b] * s;
            Eyp[(long long)(r0 + b) * nx] = sy / G.My[r0 + b];
        }
    }
    __syncthreads();
    // x: one element segment of a node row per thread (the element, and its left neighbour for
    // the shared node a = 0; x is periodic)
    for (int it = threadIdx.x; it < nr * G.ex; it += blockDim.x) {
        const int r = it / G.ex, e = it - r * G.ex;
        const float *row = sV + r * nx;
        const int el = e == 0 ? G.ex - 1 : e - 1;
        float v[P], vl[P];
#pragma unroll
        for (int m = 0; m < P; ++m) {
            int cc = e * K + m;
            if (cc >= nx) cc -= nx;
            v[m] = row[cc];
            vl[m] = row[el * K + m < nx ? el * K + m : el * K + m - nx];
        }
#pragma unroll
        for (int a = 0; a < K; ++a) {
            float s = 0.f;
#pragma unroll
            for (int m = 0; m < P; ++m) s += t.d[a * P + m] * v[m];
            float sx = t.w[a] * s;
            if (a == 0) {
                float sl = 0.f;
#pragma unroll
                for (int m = 0; m < P; ++m) sl += t.d[K * P + m] * vl[m];
                sx += t.w[K] * sl;
            }
            sE[r * nx + e * K + a] = sx / G.Mx[e * K + a];
        }
    }
    __syncthreads();
    float *Exp = Ex + (long long)blockIdx.y * G.n2 + (long long)r0 * nx;
    for (int i = threadIdx.x; i < nr * nx; i += blockDim.x) Exp[i] = sE[i];
}

// ---- eq. 56 / 75: psi right-hand side ----------------------------------------------------
// Q1 = (-u* . grad phi* + phi_hat/dt)/(lambda gamma1) (element-local),
// Q2 = h(phi*) - (S/eta^2) phi* - eps'(phi*)/(2 lambda) |E|^2 (nodal, written to Q2n),
// A = -int Q1 w + int grad_2D Q2 . grad_2D w + (alpha + S/eta^2) int_wall U w,
// U = -Theta'(phi*)/lambda; faceU (optional) = int_wall U w (element-local face slots).
template <typename T, int KC = 0>
__global__ void k_chem(Geo<T> G_, Phys<T> q_, const T *__restrict__ phin, const T *__restrict__ phio,
                       const T *__restrict__ dzphin, const T *__restrict__ dzphio,
                       const T *__restrict__ uxn, const T *__restrict__ uxo, const T *__restrict__ uyn,
                       const T *__restrict__ uyo, const T *__restrict__ uzn, const T *__restrict__ uzo,
                       const T *__restrict__ Ex, const T *__restrict__ Ey, const T *__restrict__ Ez,
                       T *__restrict__ A, T *__restrict__ Q2n, T *__restrict__ faceU) {
    if (plane_frozen(G_)) return;
    const Geo<T> G = fixed_order<KC>(G_);
    PF_ELEM_SMEM(T, G, 4)
    const Phys<T> q = plane_phys(q_);
    T *sP = sF, *sQ = sF + pp_, *sQx = sF + 2 * pp_, *sQy = sF + 3 * pp_;
    load_tables(G, sD, sDw, sw);
    const ElemIdx e = elem_index(G);
    const bool act = e.act;
    const T hx = G.hx[e.ex], hy = G.hy[e.ey];
    T phis = 0, Q1 = 0;
    if (act) {
        phis = star(q.J, phin[e.g], phio[e.g]);
        sP[e.t] = phis;
        const T ex = Ex[e.g], ey = Ey[e.g], ez = Ez ? Ez[e.g] : T(0);
        const T E2 = ex * ex + ey * ey + ez * ez;
        const T Q2 = h_of(q, phis) - q.S_eta2 * phis - deps_of(q, phis) / (T(2) * q.lam) * E2;
        sQ[e.t] = Q2;
        Q2n[e.g] = Q2;   // identical value from every element sharing the node
    }
    __syncthreads();
    if (act) {
        const T sx = T(2) / hx, sy = T(2) / hy;
        const T *fs[2] = {sP, sQ};   // phi* and Q2, each coefficient loaded once for both
        T dx[2], dy[2];
        ddx_n(fs, sD, G.p, e.a, e.b, sx, dx);
        ddy_n(fs, sD, G.p, e.a, e.b, sy, dy);
        const T gpx = dx[0];
        const T gpy = dy[0];
        T adv = star(q.J, uxn[e.g], uxo[e.g]) * gpx + star(q.J, uyn[e.g], uyo[e.g]) * gpy;
        if (uzn) adv += star(q.J, uzn[e.g], uzo[e.g]) * star(q.J, dzphin[e.g], dzphio[e.g]);
        const T phh = hatv(q.J, phin[e.g], phio[e.g]);
        Q1 = (-adv + phh / q.dt) / (q.lam * q.gamma1);
        sQx[e.t] = dx[1];
        sQy[e.t] = dy[1];
    }
    __syncthreads();
    if (!act) return;
    const T hx2 = T(0.5) * hx, hy2 = T(0.5) * hy;
    T r = -hx2 * hy2 * sw[e.a] * sw[e.b] * Q1 + wdx(sQx, sDw, sw, G.p, e.a, e.b, hy2) +
          wdy(sQy, sDw, sw, G.p, e.a, e.b, hx2);
    if (q.wetting && e.ey == 0 && e.b == 0) {
        const T U = -dtheta_of(q, phis) / q.lam;
        const T fu = hx2 * sw[e.a] * U;
        r += (q.alpha + q.S_eta2) * fu;
        if (faceU) faceU[((long long)e.z * G.ex + e.ex) * G.p + e.a] = fu;
    }
    A[e.l] = r;
}

// ---- eq. 49, 58a / 77a, 59a / 78a: momentum right-hand sides -------------------------------
// T = (1/rho)[-lambda L grad phi - eps'(phi)/2 |E|^2 grad phi + grad mu . D(u*) - Jt . grad u*]
//     + u_hat/dt - u* . grad u* + (1/rho0 - 1/rho) grad P*,     L = psi - alpha phi,
// Jt = (rho1 - rho2)/2 lambda gamma1 grad W,  G = T + grad(mu/rho) x omega*.
// Outputs (element-local): AP = rho0 int G_2D . grad_2D q + wall term,  BP = -rho0 int G_z q + wall,
// AU[c], BU[c]: the velocity right-hand side without the new pressure gradient.
template <typename T>
struct MomIn {
    const T *phi, *dzphi, *W, *dzW, *L, *Ex, *Ey, *Ez;
    const T *un[3], *uo[3], *dzun[3], *dzuo[3];
    const T *Pn, *Po, *dzPn, *dzPo;
};
template <typename T>
struct MomOut {
    T *AP, *BP, *AU[3], *BU[3];
};

template <typename T, int KC = 0>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 4 : 2) k_momentum(Geo<T> G_, Phys<T> q_, MomIn<T> in, MomOut<T> out) {
    if (plane_frozen(G_)) return;
    const Geo<T> G = fixed_order<KC>(G_);
    PF_ELEM_SMEM(T, G, 12)
    const Phys<T> q = plane_phys(q_);
    // inputs with in-plane derivatives: phi, W, u*_x, u*_y, u*_z, P*
    T *sphi = sF, *sW = sF + pp_, *sux = sF + 2 * pp_, *suy = sF + 3 * pp_, *suz = sF + 4 * pp_,
      *sPs = sF + 5 * pp_;
    // fluxes for weak derivatives (reuse after the derivative pass)
    T *sGx = sF + 6 * pp_, *sGy = sF + 7 * pp_, *sKx = sF + 8 * pp_, *sKy = sF + 9 * pp_,
      *sKz = sF + 10 * pp_, *sJx = sF + 11 * pp_;
    load_tables(G, sD, sDw, sw);
    const ElemIdx e = elem_index(G);
    const bool act = e.act;
    const bool d3 = in.un[2] != nullptr;
    const int J = q.J;
    const T hx = G.hx[e.ex], hy = G.hy[e.ey];
    T us[3] = {0, 0, 0};
    if (act) {
        sphi[e.t] = in.phi[e.g];
        sW[e.t] = in.W[e.g];
        us[0] = star(J, in.un[0][e.g], in.uo[0][e.g]);
        us[1] = star(J, in.un[1][e.g], in.uo[1][e.g]);
        if (d3) us[2] = star(J, in.un[2][e.g], in.uo[2][e.g]);
        sux[e.t] = us[0];
        suy[e.t] = us[1];
        suz[e.t] = us[2];
        sPs[e.t] = star(J, in.Pn[e.g], in.Po[e.g]);
    }
    __syncthreads();
    T mr = 0, om[3] = {0, 0, 0}, Gv[3] = {0, 0, 0};
    if (act) {
        const T sx = T(2) / hx, sy = T(2) / hy;
        const T phi = sphi[e.t];
        // x and y derivatives of phi, W, u*_x, u*_y, u*_z (0 in 2D), P*, each coefficient loaded once
        const T *fs[6] = {sphi, sW, sux, suy, suz, sPs};
        T dx[6], dy[6];
        ddx_n(fs, sD, G.p, e.a, e.b, sx, dx);
        ddy_n(fs, sD, G.p, e.a, e.b, sy, dy);
        T gphi[3] = {dx[0], dy[0], d3 ? in.dzphi[e.g] : T(0)};
        T gW[3] = {dx[1], dy[1], d3 ? in.dzW[e.g] : T(0)};
        T gu[3][3];   // gu[c][d] = d u*_c / d x_d
        gu[0][0] = dx[2];
        gu[0][1] = dy[2];
        gu[1][0] = dx[3];
        gu[1][1] = dy[3];
        gu[2][0] = d3 ? dx[4] : T(0);
        gu[2][1] = d3 ? dy[4] : T(0);
        if (d3) {
            for (int c = 0; c < 3; ++c) gu[c][2] = star(J, in.dzun[c][e.g], in.dzuo[c][e.g]);
        } else {
            gu[0][2] = gu[1][2] = gu[2][2] = 0;
        }
        T gP[3] = {dx[5], dy[5], d3 ? star(J, in.dzPn[e.g], in.dzPo[e.g]) : T(0)};
        const T rho = rho_of(q, phi), mu = mu_of(q, phi);
        const T irho = T(1) / rho;
        mr = mu * irho;
        const T ex = in.Ex[e.g], ey = in.Ey[e.g], ez = d3 ? in.Ez[e.g] : T(0);
        const T E2 = ex * ex + ey * ey + ez * ez;
        const T Lv = in.L[e.g];
        const T dmu = T(0.5) * (q.mu1 - q.mu2);
        const T drho = T(0.5) * (q.rho1 - q.rho2);
        const T cJ = drho * q.lam * q.gamma1;
        const T kf = -q.lam * Lv - T(0.5) * deps_of(q, phi) * E2;
        T uh[3];
        for (int c = 0; c < 3; ++c) uh[c] = (c < 2 || d3) ? hatv(J, in.un[c][e.g], in.uo[c][e.g]) : T(0);
        T Tv[3];
        for (int c = 0; c < 3; ++c) {
            T visc = 0, jgu = 0, conv = 0;
            for (int d = 0; d < 3; ++d) {
                visc += dmu * gphi[d] * (gu[c][d] + gu[d][c]);
                jgu += cJ * gW[d] * gu[c][d];
                conv += us[d] * gu[c][d];
            }
            Tv[c] = (kf * gphi[c] + visc - jgu) * irho + uh[c] / q.dt - conv + (T(1) / q.rho0 - irho) * gP[c];
        }
        om[0] = gu[2][1] - gu[1][2];
        om[1] = gu[0][2] - gu[2][0];
        om[2] = gu[1][0] - gu[0][1];
        const T dmr = (dmu * rho - mu * drho) * irho * irho;
        const T gm[3] = {dmr * gphi[0], dmr * gphi[1], dmr * gphi[2]};
        Gv[0] = Tv[0] + gm[1] * om[2] - gm[2] * om[1];
        Gv[1] = Tv[1] + gm[2] * om[0] - gm[0] * om[2];
        Gv[2] = Tv[2] + gm[0] * om[1] - gm[1] * om[0];
    }
    __syncthreads();   // derivative inputs consumed; flux arrays written next
    const T Kf = mr - q.nu_m;
    if (act) {
        sGx[e.t] = Gv[0];
        sGy[e.t] = Gv[1];
        sKx[e.t] = Kf * om[0];
        sKy[e.t] = Kf * om[1];
        sKz[e.t] = Kf * om[2];
        sJx[e.t] = mr * om[2];   // wall: -J_x = (mu/rho) omega_z for n = (0,-1,0)
    }
    __syncthreads();
    if (!act) return;
    const T hx2 = T(0.5) * hx, hy2 = T(0.5) * hy;
    const T Me = hx2 * hy2 * sw[e.a] * sw[e.b];
    const T inu = T(1) / q.nu_m;
    const int p = G.p;
    // pressure: rho0 int G_2D . grad q - rho0 int_wall J_x dq/dx  ;  iB part: -rho0 int G_z q + rho0 int_wall J_z q
    // weak x derivatives of G_x, K_z, K_y and weak y derivatives of G_y, K_z, K_x, each coefficient
    // loaded once
    const T *fwx[3] = {sGx, sKz, sKy}, *fwy[3] = {sGy, sKz, sKx};
    T wx[3], wy[3];
    wdx_n(fwx, sDw, sw, p, e.a, e.b, hy2, wx);
    wdy_n(fwy, sDw, sw, p, e.a, e.b, hx2, wy);
    T ap = q.rho0 * (wx[0] + wy[0]);
    T bp = -q.rho0 * Me * Gv[2];
    if (e.ey == 0 && e.b == 0) {
        // -rho0 int_wall J_x dq/dx with J_x = -(mu/rho) omega_z: 1D weak x-derivative of the face row
        T s = 0;
        for (int m = 0; m < p; ++m) s += sDw[m * p + e.a] * sJx[m];   // row b = 0
        ap += q.rho0 * s;
        bp += q.rho0 * hx2 * sw[e.a] * mr * om[0];                     // J_z = (mu/rho) omega_x
    }
    out.AP[e.l] = ap;
    if (out.BP) out.BP[e.l] = bp;
    // velocity (without the new pressure): (1/nu_m) int G v - (1/nu_m) int K x grad v - (1/nu_m) int_top L v
    T ax = inu * (Me * Gv[0] + wy[1]);
    T ay = inu * (Me * Gv[1] - wx[1]);
    T az = inu * (Me * Gv[2] - wy[2] + wx[2]);
    if (e.ey == G.ey - 1 && e.b == G.K) {
        ax -= inu * hx2 * sw[e.a] * Kf * om[2];      // L_x = (mu/rho - nu_m) omega_z
        az += inu * hx2 * sw[e.a] * Kf * om[0];      // L_z = -(mu/rho - nu_m) omega_x
    }
    out.AU[0][e.l] = ax;
    out.AU[1][e.l] = ay;
    if (d3) {
        out.AU[2][e.l] = az;
        out.BU[0][e.l] = inu * Me * Kf * om[1];       //  i beta (1/nu_m) int K_y v
        out.BU[1][e.l] = -inu * Me * Kf * om[0];      // -i beta (1/nu_m) int K_x v
    }
}

// -(1/(nu_m rho0)) int grad P^{n+1} v: added to AU[0], AU[1]; the z part is -(1/(nu_m rho0)) i beta int P v.
template <typename T, int KC = 0>
__global__ void k_ugradp(Geo<T> G_, Phys<T> q, const T *__restrict__ P, T *__restrict__ AUx,
                         T *__restrict__ AUy, T *__restrict__ BUz) {
    if (plane_frozen(G_)) return;
    const Geo<T> G = fixed_order<KC>(G_);
    PF_ELEM_SMEM(T, G, 1)
    T *sPv = sF;
    load_tables(G, sD, sDw, sw);
    const ElemIdx e = elem_index(G);
    const bool act = e.act;
    if (act) sPv[e.t] = P[e.g];
    __syncthreads();
    if (!act) return;
    const T hx = G.hx[e.ex], hy = G.hy[e.ey];
    const T Me = T(0.25) * hx * hy * sw[e.a] * sw[e.b];
    const T c = -T(1) / (q.nu_m * q.rho0);
    AUx[e.l] += c * Me * ddx(sPv, sD, G.p, e.a, e.b, T(2) / hx);
    AUy[e.l] += c * Me * ddy(sPv, sD, G.p, e.a, e.b, T(2) / hy);
    if (BUz) BUz[e.l] = c * Me * sPv[e.t];
}

// ---- direct stiffness summation of element-local contributions at nodal index (z, i, j) ----
template <typename T>
__device__ __forceinline__ T dssum(const Geo<T> &G, const T *__restrict__ Lv, int z, int i, int j) {
    const int K = G.K, p = G.p;
    int eys[2], bs[2], ny_ = 0;
    if (i % K == 0) {
        if (i > 0) { eys[ny_] = i / K - 1; bs[ny_++] = K; }
        if (i < G.ny - 1) { eys[ny_] = i / K; bs[ny_++] = 0; }
    } else {
        eys[ny_] = i / K; bs[ny_++] = i % K;
    }
    int exs[2], as[2], nx_ = 0;
    if (j % K == 0) {
        exs[nx_] = j / K; as[nx_++] = 0;
        exs[nx_] = (j / K - 1 + G.ex) % G.ex; as[nx_++] = K;
    } else {
        exs[nx_] = j / K; as[nx_++] = j % K;
    }
    T s = 0;
    for (int cy = 0; cy < ny_; ++cy)
        for (int cx = 0; cx < nx_; ++cx) s += Lv[eloc(G, z, eys[cy], exs[cx], bs[cy], as[cx])];
    return s;
}

// ---- in-shared-memory radix-2 FFT along z -------------------------------------------------
__device__ __forceinline__ int bitrev(int v, int bits) { return bits ? (int)(__brev((unsigned)v) >> (32 - bits)) : 0; }

// in-place DIT FFT of npen pencils of length n = 2^lg (bit-reversed input), forward or inverse;
// all index arithmetic is shifts and masks (n, the spans and the pencil count are powers of two
// or plain multiples)
template <typename T>
__device__ __forceinline__ void fft_pencils(cplx<T> *buf, int ld, int npen, int n, const cplx<T> *tw, bool inverse) {
    const int lg = 31 - __clz(n);
    const int hb = lg - 1;                       // log2(n / 2)
    const int nb = npen << hb;
#pragma unroll
    for (int s = 1; s <= lg; ++s) {
        const int hs = s - 1;                    // log2(half span)
        const int hmask = (1 << hs) - 1;
        for (int t = threadIdx.x; t < nb; t += blockDim.x) {
            const int pen = t >> hb, bf = t & ((1 << hb) - 1);
            const int grp = bf >> hs, jj = bf & hmask;
            const int i0 = (grp << s) + jj, i1 = i0 + (1 << hs);
            cplx<T> w = tw[jj << (lg - s)];
            if (inverse) w.y = -w.y;
            cplx<T> *x = buf + pen * ld;
            const cplx<T> u = x[i0];
            const cplx<T> v = cmul(x[i1], w);
            x[i0] = {u.x + v.x, u.y + v.y};
            x[i1] = {u.x - v.x, u.y - v.y};
        }
        __syncthreads();
    }
}

// The radix-2 DIT of fft_pencils for n = 2^LGZ = 32 .. 256, one warp per pencil in registers:
// lane l holds the E = n/32 elements l + 32 e (bit-reversed order as loaded).  A stage of half
// span h < 32 pairs lanes l and l ^ h (__shfl_xor; the twiddle depends on l mod h only), a stage of
// span h >= 32 pairs the lane's own elements e and e ^ (h/32) (twiddle of (l + 32 e) mod h); the
// butterfly arithmetic is that of fft_pencils.  Called after the block barrier that completes the
// buffer's loads; ends with a block barrier (the buffer is read by other threads next).
template <typename T, int LGZ>
__device__ __forceinline__ void fft_pencils_warp(cplx<T> *buf, int ld, int npen, const cplx<T> *tw, bool inverse) {
    static_assert(LGZ >= 5 && LGZ <= 8, "one warp per pencil of 32 to 256 points");
    constexpr int E = (1 << LGZ) / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    for (int pen = warp; pen < npen; pen += nwarp) {
        cplx<T> *x = buf + pen * ld;
        cplx<T> v[E];
#pragma unroll
        for (int e = 0; e < E; ++e) v[e] = x[lane + 32 * e];
#pragma unroll
        for (int s = 1; s <= LGZ; ++s) {
            const int h = 1 << (s - 1);
            if (h < 32) {
                cplx<T> w = tw[(lane & (h - 1)) << (LGZ - s)];
                if (inverse) w.y = -w.y;
                const bool top = (lane & h) == 0;
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    cplx<T> pr;
                    pr.x = __shfl_xor_sync(0xffffffffu, v[e].x, h);
                    pr.y = __shfl_xor_sync(0xffffffffu, v[e].y, h);
                    if (top) {
                        const cplx<T> m = cmul(pr, w);
                        v[e] = {v[e].x + m.x, v[e].y + m.y};
                    } else {
                        const cplx<T> m = cmul(v[e], w);
                        v[e] = {pr.x - m.x, pr.y - m.y};
                    }
                }
            } else {   // span h >= 32: elements e and e + h/32 of this lane
                const int hh = h >> 5;
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    if ((e & hh) == 0) {
                        cplx<T> w = tw[(lane + 32 * (e & (hh - 1))) << (LGZ - s)];
                        if (inverse) w.y = -w.y;
                        const cplx<T> m = cmul(v[e + hh], w);
                        const cplx<T> u = v[e];
                        v[e] = {u.x + m.x, u.y + m.y};
                        v[e + hh] = {u.x - m.x, u.y - m.y};
                    }
                }
            }
        }
#pragma unroll
        for (int e = 0; e < E; ++e) x[lane + 32 * e] = v[e];
    }
    __syncthreads();
}

// 8-point DFT of v in registers, natural order in and out (radix-2 decimation in frequency,
// the bit-reversed result renamed at compile time); w8 = exp(-+ i pi / 4)
template <typename T>
__device__ __forceinline__ void dft8(cplx<T> *v, bool inverse) {
    const T r = T(0.70710678118654752440);
    const T sg = inverse ? T(1) : T(-1);   // sign of the imaginary part of w8
    cplx<T> a[8];
#pragma unroll
    for (int j = 0; j < 4; ++j) {          // span 4, twiddles w8^j
        const cplx<T> p = v[j], q = v[j + 4];
        a[j] = {p.x + q.x, p.y + q.y};
        const cplx<T> d = {p.x - q.x, p.y - q.y};
        if (j == 0) a[4] = d;
        else if (j == 1) a[5] = {r * (d.x - sg * d.y), r * (d.y + sg * d.x)};
        else if (j == 2) a[6] = {-sg * d.y, sg * d.x};
        else a[7] = {r * (-d.x - sg * d.y), r * (-d.y + sg * d.x)};
    }
#pragma unroll
    for (int h = 0; h < 8; h += 4) {       // span 2, twiddles w8^(2j) = 1, -+i
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const cplx<T> p = a[h + j], q = a[h + j + 2];
            a[h + j] = {p.x + q.x, p.y + q.y};
            const cplx<T> d = {p.x - q.x, p.y - q.y};
            a[h + j + 2] = j == 0 ? d : cplx<T>{-sg * d.y, sg * d.x};
        }
    }
#pragma unroll
    for (int h = 0; h < 8; h += 2) {       // span 1
        const cplx<T> p = a[h], q = a[h + 1];
        a[h] = {p.x + q.x, p.y + q.y};
        a[h + 1] = {p.x - q.x, p.y - q.y};
    }
    // a[i] holds output bitrev3(i)
    v[0] = a[0]; v[4] = a[1]; v[2] = a[2]; v[6] = a[3]; v[1] = a[4]; v[5] = a[5]; v[3] = a[6]; v[7] = a[7];
}

// w^m, w = exp(-+ 2 pi i / 256), 0 <= m < 256, from the half table tw (w^(m + 128) = -w^m)
template <typename T>
__device__ __forceinline__ cplx<T> tw256(const cplx<T> *tw, int m, bool inverse) {
    cplx<T> w = tw[m & 127];
    if (m & 128) w = {-w.x, -w.y};
    if (inverse) w.y = -w.y;
    return w;
}

// 256-point FFT of npen pencils, one warp per pencil, natural order in and out, in four steps
// (256 = 8 x 32 = 8 x 8 x 4): lane l takes x[l + 32 e] (e < 8) and runs an 8-point DFT over e,
// twiddled by w^(l k1); a transpose through the pencil's own buffer (rows of 36 so that the reads
// below hit every bank pair twice) gives lane (k1, l1) = 4 k1 + l1 the eight values of lanes
// l1 + 4 l2, an 8-point DFT over l2 twiddled by w32^(l1 k2); a 4-point DFT over l1 across the four
// lanes of a quad (two shuffle stages) completes X[k1 + 8 k2 + 64 k3].  The pencil buffer must
// hold 8 x 36 = 288 values (ld >= 288).  Called after the block barrier that completes the
// loads; ends with a block barrier.
template <typename T>
__device__ __forceinline__ void fft256_warp(cplx<T> *buf, int ld, int npen, const cplx<T> *tw, bool inverse) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    const int k1q = lane >> 2, l1 = lane & 3;
    for (int pen = warp; pen < npen; pen += nwarp) {
        cplx<T> *x = buf + pen * ld;
        cplx<T> v[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) v[e] = x[lane + 32 * e];
        dft8(v, inverse);
#pragma unroll
        for (int k = 1; k < 8; ++k) v[k] = cmul(v[k], tw256(tw, lane * k, inverse));
        __syncwarp();
#pragma unroll
        for (int k = 0; k < 8; ++k) x[k * 36 + lane] = v[k];
        __syncwarp();
#pragma unroll
        for (int j = 0; j < 8; ++j) v[j] = x[k1q * 36 + 4 * j + l1];
        dft8(v, inverse);
#pragma unroll
        for (int k = 1; k < 8; ++k) v[k] = cmul(v[k], tw256(tw, 8 * l1 * k, inverse));
        // 4-point DFT over l1 (the quad's lanes): pairs l1, l1 ^ 2, then l1, l1 ^ 1; lane l1 ends
        // with output k3 = {0, 2, 1, 3}[l1]
        const T sg = inverse ? T(1) : T(-1);
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            cplx<T> p;
            p.x = __shfl_xor_sync(0xffffffffu, v[k].x, 2);
            p.y = __shfl_xor_sync(0xffffffffu, v[k].y, 2);
            v[k] = l1 < 2 ? cplx<T>{v[k].x + p.x, v[k].y + p.y} : cplx<T>{p.x - v[k].x, p.y - v[k].y};
            p.x = __shfl_xor_sync(0xffffffffu, v[k].x, 1);
            p.y = __shfl_xor_sync(0xffffffffu, v[k].y, 1);
            if (l1 == 0) v[k] = {v[k].x + p.x, v[k].y + p.y};
            else if (l1 == 1) v[k] = {p.x - v[k].x, p.y - v[k].y};
            else if (l1 == 2) v[k] = {v[k].x - sg * p.y, v[k].y + sg * p.x};   // + w4 p, w4 = -+i
            else v[k] = {p.x + sg * v[k].y, p.y - sg * v[k].x};                 // p - w4 v
        }
        const int k3 = (l1 == 1) ? 2 : (l1 == 2) ? 1 : l1;
        __syncwarp();
#pragma unroll
        for (int k = 0; k < 8; ++k) x[k1q + 8 * k + 64 * k3] = v[k];
        __syncwarp();
    }
    __syncthreads();
}

// Stockham autosort FFT of npen pencils of any even length n = 2^a 3^b 5^c 7^d (natural order in
// and out; the result ends in buf, tmp is scratch of the same shape).  Each stage of radix R
// (4, 2, 3, 5 or 7, taken in that order while it divides what is left) combines R inputs
// x[j + r n/R] of the pencil, twiddled by w^(r (j mod Ns) n/(Ns R)), through an R-point DFT into
// the outputs (j / Ns) Ns R + (j mod Ns) + s Ns, Ns = product of the earlier radices.  Twiddles
// w^m = exp(-+2 pi i m / n) come from the half table tw (w^(m + n/2) = -w^m).
template <typename T>
__device__ void fft_pencils_mixed(cplx<T> *buf, cplx<T> *tmp, int ld, int npen, int n, const cplx<T> *tw,
                                  bool inverse) {
    const int h = n / 2;
    auto W = [&](int m) {
        cplx<T> w = m < h ? tw[m] : cplx<T>{-tw[m - h].x, -tw[m - h].y};
        if (inverse) w.y = -w.y;
        return w;
    };
    cplx<T> *in = buf, *out = tmp;
    int Ns = 1, rem = n;
    while (rem > 1) {
        const int R = (rem % 4 == 0) ? 4 : (rem % 2 == 0) ? 2 : (rem % 3 == 0) ? 3 : (rem % 5 == 0) ? 5 : 7;
        const int nb = n / R, tstep = n / (Ns * R), sstep = n / R;
        for (int t = threadIdx.x; t < npen * nb; t += blockDim.x) {
            const int pen = t / nb, j = t - pen * nb, k = j % Ns;
            const cplx<T> *x = in + pen * ld;
            cplx<T> *y = out + pen * ld;
            cplx<T> v[7];
#pragma unroll
            for (int r = 0; r < 7; ++r) {
                if (r >= R) break;
                v[r] = x[j + r * nb];
                if (r) v[r] = cmul(v[r], W(r * k * tstep));
            }
            const int o = (j / Ns) * Ns * R + k;
#pragma unroll
            for (int s = 0; s < 7; ++s) {
                if (s >= R) break;
                cplx<T> acc = v[0];
#pragma unroll
                for (int r = 1; r < 7; ++r) {
                    if (r >= R) break;
                    const cplx<T> p = cmul(v[r], W(((r * s) % R) * sstep));
                    acc.x += p.x;
                    acc.y += p.y;
                }
                y[o + s * Ns] = acc;
            }
        }
        __syncthreads();
        cplx<T> *sw = in;
        in = out;
        out = sw;
        Ns *= R;
        rem /= R;
    }
    if (in != buf) {
        for (int t = threadIdx.x; t < npen * n; t += blockDim.x) {
            const int pen = t / n, i = t - pen * n;
            buf[pen * ld + i] = in[pen * ld + i];
        }
        __syncthreads();
    }
}

// FP32 256-plane transforms run fft256_warp: natural order and 289-value pencil rows (it
// transposes through the pencil's own buffer); every other transform: bit-reversed DIT, nz + 1
template <typename T, int LGZ>
__host__ __device__ constexpr bool fft_four_step() { return LGZ == 8 && sizeof(T) == 4; }
template <typename T, int LGZ>
__host__ __device__ constexpr int fft_ld(int nz) { return fft_four_step<T, LGZ>() ? 289 : nz + 1; }

// position of sample (or mode) i in the transform buffer: bit-reversed for the radix-2 DIT
__device__ __forceinline__ int fft_slot(int i, int bits, bool pow2) { return pow2 ? bitrev(i, bits) : i; }

// mode index k and real/imaginary part of packed plane p
__device__ __forceinline__ void plane_mode(int p, int nz, int &k, int &im) {
    if (nz == 1 || p == 0) { k = 0; im = 0; return; }
    if (p == 1) { k = nz / 2; im = 0; return; }
    k = p >> 1; im = p & 1;
}

template <typename T>
struct FwdArgs {
    long long cs_x0, cs_x1, cs_out; // strides between components (blockIdx.y), 0 for one
    const T *X0; int x0_local;      // input 0: element-local (1) or nodal (0)
    const T *X1; int x1_local;      // input 1 (nullable)
    int mult;                       // 0: X0 + i beta X1 ; 1: X0 + beta^2 M X1
    T scale;                        // applied to the combined result
    const T *lift;                  // nullable: n_y vector; plane 0 gets -lift[i] * Mx[j]
    const T *lift2y, *lift2x;       // nullable: plane p also gets -lift2y[i] * Mx[j] * lift2x[p][j] (n_x per plane)
    T *out;                         // packed mode planes [nz][n2]
    T *out1;                        // nullable: packed FFT of X1 alone
    T two_pi_over_lz;
    const cplx<T> *tw;              // nz/2 twiddles exp(-2 pi i k / nz)
    int tp;                         // nodes per block
};

// element-local slots (within plane 0) that sum into nodal index q; unused slots are -1
template <typename T>
__device__ __forceinline__ void dss_sources(const Geo<T> &G, int q, int src[4]) {
    const int K = G.K, p = G.p, i = q / G.nx, j = q % G.nx;
    int eys[2], bs[2], ny_ = 0;
    if (i % K == 0) {
        if (i > 0) { eys[ny_] = i / K - 1; bs[ny_++] = K; }
        if (i < G.ny - 1) { eys[ny_] = i / K; bs[ny_++] = 0; }
    } else {
        eys[ny_] = i / K; bs[ny_++] = i % K;
    }
    int exs[2], as[2], nx_ = 0;
    if (j % K == 0) {
        exs[nx_] = j / K; as[nx_++] = 0;
        exs[nx_] = (j / K - 1 + G.ex) % G.ex; as[nx_++] = K;
    } else {
        exs[nx_] = j / K; as[nx_++] = j % K;
    }
    int c = 0;
    for (int cy = 0; cy < ny_; ++cy)
        for (int cx = 0; cx < nx_; ++cx) src[c++] = (int)eloc(G, 0, eys[cy], exs[cx], bs[cy], as[cx]);
    for (; c < 4; ++c) src[c] = -1;
}

template <typename T>
__device__ __forceinline__ T gather4(const T *__restrict__ L, long long zoff, const int *s) {
    T v = L[zoff + s[0]];
    if (s[1] >= 0) v += L[zoff + s[1]];
    if (s[2] >= 0) v += L[zoff + s[2]];
    if (s[3] >= 0) v += L[zoff + s[3]];
    return v;
}

// LGZ > 0: Nz = 2^LGZ fixed at compile time (the FFT stages unroll, index arithmetic on Nz folds);
// LGZ = 0: Nz from G (any supported value)
template <typename T, int LGZ = 0>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 5 : 2) k_fwd(Geo<T> G, FwdArgs<T> a) {
    if (blockIdx.y) {   // component blockIdx.y of a batched launch
        a.X0 += blockIdx.y * a.cs_x0;
        if (a.X1) a.X1 += blockIdx.y * a.cs_x1;
        a.out += blockIdx.y * a.cs_out;
    }
    extern __shared__ unsigned char pf_smem_raw[];
    cplx<T> *stw = reinterpret_cast<cplx<T> *>(pf_smem_raw);
    const int nz = LGZ ? (1 << LGZ) : G.nz, ld = fft_ld<T, LGZ>(nz), tp = a.tp;
    cplx<T> *buf = stw + (nz > 1 ? nz / 2 : 1);
    int *ssrc = reinterpret_cast<int *>(buf + tp * ld);   // tp x 4 DSSUM sources
    const bool pow2 = (nz & (nz - 1)) == 0 && !fft_four_step<T, LGZ>();   // bit-reversed slots
    cplx<T> *tmp = reinterpret_cast<cplx<T> *>(ssrc + tp * 4);   // mixed-radix scratch (nz not 2^k)
    const int bits = 31 - __clz(nz);
    for (int i = threadIdx.x; i < nz / 2; i += blockDim.x) stw[i] = a.tw[i];
    const int q0 = blockIdx.x * tp;
    for (int ql = threadIdx.x; ql < tp; ql += blockDim.x) {
        int s[4] = {-1, -1, -1, -1};
        if (q0 + ql < G.n2) dss_sources(G, q0 + ql, s);
        for (int c = 0; c < 4; ++c) ssrc[ql * 4 + c] = s[c];
    }
    __syncthreads();
    const long long lplane = (long long)G.ex * G.ey * G.p * G.p;
    const int lgtp = 31 - __clz(tp);          // tp is a power of two dividing blockDim.x
    {
        // this thread's pencil column is fixed (blockDim.x is a multiple of tp): its DSSUM sources
        // live in registers, and it walks the planes z0, z0 + zs, ... eight gathers at a time
        const int ql = threadIdx.x & (tp - 1), qg = q0 + ql, z0 = threadIdx.x >> lgtp, zs = blockDim.x >> lgtp;
        int sr[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) sr[c] = ssrc[ql * 4 + c];
        const bool live = qg < G.n2;
        for (int zb = z0; zb < nz; zb += 8 * zs) {
            T v0[8], v1[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {   // eight independent gathers in flight
                const int z = zb + u * zs;
                v0[u] = 0;
                v1[u] = 0;
                if (live && z < nz) {
                    const long long gi = (long long)z * G.n2 + qg;
                    v0[u] = a.x0_local ? gather4(a.X0, z * lplane, sr) : a.X0[gi];
                    if (a.X1) v1[u] = a.x1_local ? gather4(a.X1, z * lplane, sr) : a.X1[gi];
                }
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int z = zb + u * zs;
                if (z < nz) buf[ql * ld + fft_slot(z, bits, pow2)] = {v0[u], v1[u]};
            }
        }
    }
    __syncthreads();
    if constexpr (fft_four_step<T, LGZ>()) {
        fft256_warp(buf, ld, tp, stw, false);
    } else if constexpr (LGZ >= 5 && sizeof(T) == 4) {   // FP64 keeps the shared-memory stages
        fft_pencils_warp<T, LGZ>(buf, ld, tp, stw, false);
    } else if (nz > 1) {
        if (pow2) fft_pencils(buf, ld, tp, nz, stw, false);
        else fft_pencils_mixed(buf, tmp, ld, tp, nz, stw, false);
    }
    const T inv_n = T(1) / T(nz);
    for (int idx = threadIdx.x; idx < tp * nz; idx += blockDim.x) {
        const int p = idx >> lgtp, ql = idx & (tp - 1), qg = q0 + ql;
        if (qg >= G.n2) continue;
        int k, im;
        plane_mode(p, nz, k, im);
        const cplx<T> zk = buf[ql * ld + k];
        const cplx<T> zn = buf[ql * ld + ((nz - k) % nz)];
        // spectra of the two real inputs
        const cplx<T> X0 = {T(0.5) * (zk.x + zn.x) * inv_n, T(0.5) * (zk.y - zn.y) * inv_n};
        const cplx<T> X1 = {T(0.5) * (zk.y + zn.y) * inv_n, -T(0.5) * (zk.x - zn.x) * inv_n};
        cplx<T> R = X0;
        if (a.X1) {
            const T beta = a.two_pi_over_lz * T(k);
            if (a.mult == 0) {
                const T b = (nz > 1 && k == nz / 2) ? T(0) : beta;   // Nyquist: no first derivative
                R.x -= b * X1.y;
                R.y += b * X1.x;
            } else {
                const int i = qg / G.nx, j = qg % G.nx;
                const T m = beta * beta * G.Mx[j] * G.My[i];
                R.x += m * X1.x;
                R.y += m * X1.y;
            }
        }
        T v = a.scale * (im ? R.y : R.x);
        if (p == 0 && a.lift) {
            const int i = qg / G.nx, j = qg % G.nx;
            v -= a.lift[i] * G.Mx[j];
        }
        if (a.lift2y) {
            const int i = qg / G.nx, j = qg % G.nx;
            v -= a.lift2y[i] * G.Mx[j] * a.lift2x[(long long)p * G.nx + j];
        }
        a.out[(long long)p * G.n2 + qg] = v;
        if (a.out1) a.out1[(long long)p * G.n2 + qg] = im ? X1.y : X1.x;
    }
}

template <typename T>
struct InvArgs {
    long long cs_y, cs_out; // strides between components (blockIdx.y), 0 for one
    const T *Y;          // packed mode planes of the solution (the plain variant's input)
    const T *psi;        // phi variant: packed psi modes
    const T *Q2h;        // phi variant: packed Q2 modes
    const T *Q2n;        // phi variant: nodal Q2 (for L = W + (S/eta^2) phi + Q2)
    T alpha, S_eta2;
    int phi_variant;
    int drow0, drow1;    // Dirichlet rows that receive the values v0 / v1 in mode 0 (-1: none)
    T v0, v1;
    T *out, *dzout;      // value and d/dz (dzout nullable)
    T *out2, *dzout2;    // phi variant: W and d/dz W
    T *out3;             // phi variant: L = psi - alpha phi
    T two_pi_over_lz;
    const cplx<T> *tw;
    int tp;
};

// Build the full complex spectrum Z = X + i Y of two real signals, Y = i beta X (d/dz),
// from the packed half spectrum X of pencil column ql; buffer is bit-reversed for the DIT.
template <typename T>
__device__ __forceinline__ void put_pair(cplx<T> *x, int nz, int bits, bool pow2, int k, cplx<T> Xk, T beta) {
    // Z_k = (1 - beta) X_k ; Z_{N-k} = (1 + beta) conj(X_k)
    const bool nyq = (nz > 1 && k == nz / 2);
    const T b = nyq ? T(0) : beta;
    x[fft_slot(k, bits, pow2)] = {(T(1) - b) * Xk.x, (T(1) - b) * Xk.y};
    if (k != 0 && !nyq) x[fft_slot(nz - k, bits, pow2)] = {(T(1) + b) * Xk.x, -(T(1) + b) * Xk.y};
}

template <typename T, int LGZ = 0>   // LGZ as for k_fwd
__global__ void k_inv(Geo<T> G, InvArgs<T> a) {
    if (blockIdx.y) {
        a.Y += blockIdx.y * a.cs_y;
        a.out += blockIdx.y * a.cs_out;
        if (a.dzout) a.dzout += blockIdx.y * a.cs_out;
    }
    extern __shared__ unsigned char pf_smem_raw[];
    cplx<T> *stw = reinterpret_cast<cplx<T> *>(pf_smem_raw);
    const int nz = LGZ ? (1 << LGZ) : G.nz, ld = fft_ld<T, LGZ>(nz), tp = a.tp;
    const int npair = a.phi_variant ? 2 : 1;
    cplx<T> *buf = stw + (nz > 1 ? nz / 2 : 1);
    const bool pow2 = (nz & (nz - 1)) == 0 && !fft_four_step<T, LGZ>();   // bit-reversed slots
    cplx<T> *tmp = buf + tp * npair * ld;   // mixed-radix scratch (nz not 2^k)
    const int bits = 31 - __clz(nz);
    for (int i = threadIdx.x; i < nz / 2; i += blockDim.x) stw[i] = a.tw[i];
    const int q0 = blockIdx.x * tp;
    // load the half spectra: one (k) per thread-iteration, both Re and Im planes
    const int nk = nz / 2 + 1;
    const int lgtp = 31 - __clz(tp);          // tp is a power of two dividing blockDim.x
    {
        // fixed pencil column per thread; modes k0, k0 + ks, ... four at a time, loads first
        const int ql = threadIdx.x & (tp - 1), qg = q0 + ql, k0 = threadIdx.x >> lgtp, ks = blockDim.x >> lgtp;
        const int nkk = nz > 1 ? nk : 1;
        const bool live = qg < G.n2;
        const int row = live ? qg / G.nx : -1;
        for (int kb = k0; kb < nkk; kb += 4 * ks) {
            cplx<T> X[4], PS[4], Q[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int k = kb + u * ks;
                X[u] = PS[u] = Q[u] = cplx<T>{0, 0};
                if (live && k < nkk) {
                    int pre, pim;
                    if (nz == 1 || k == 0) { pre = 0; pim = -1; }
                    else if (k == nz / 2) { pre = 1; pim = -1; }
                    else { pre = 2 * k; pim = 2 * k + 1; }
                    const long long ore = (long long)pre * G.n2 + qg, oim = (long long)pim * G.n2 + qg;
                    X[u] = {a.Y[ore], pim >= 0 ? a.Y[oim] : T(0)};
                    if (a.phi_variant) {
                        PS[u] = {a.psi[ore], pim >= 0 ? a.psi[oim] : T(0)};
                        Q[u] = {a.Q2h[ore], pim >= 0 ? a.Q2h[oim] : T(0)};
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int k = kb + u * ks;
                if (k >= nkk) continue;
                cplx<T> Xk = X[u], Wk = {0, 0};
                if (k == 0 && a.drow0 >= 0 && row == a.drow0) Xk.x += a.v0;
                if (k == 0 && a.drow1 >= 0 && row == a.drow1) Xk.x += a.v1;
                if (a.phi_variant) {
                    const T c = a.alpha + a.S_eta2;
                    Wk = {PS[u].x - c * Xk.x - Q[u].x, PS[u].y - c * Xk.y - Q[u].y};
                }
                const T beta = a.two_pi_over_lz * T(k);
                if (nz == 1) {
                    buf[ql * ld] = Xk;
                    if (a.phi_variant) buf[(tp + ql) * ld] = Wk;
                } else {
                    put_pair(buf + ql * ld, nz, bits, pow2, k, Xk, beta);
                    if (a.phi_variant) put_pair(buf + (tp + ql) * ld, nz, bits, pow2, k, Wk, beta);
                }
            }
        }
    }
    __syncthreads();
    if constexpr (fft_four_step<T, LGZ>()) {
        fft256_warp(buf, ld, tp * npair, stw, true);
    } else if constexpr (LGZ >= 5 && sizeof(T) == 4) {   // FP64 keeps the shared-memory stages
        fft_pencils_warp<T, LGZ>(buf, ld, tp * npair, stw, true);
    } else if (nz > 1) {
        if (pow2) fft_pencils(buf, ld, tp * npair, nz, stw, true);
        else fft_pencils_mixed(buf, tmp, ld, tp * npair, nz, stw, true);
    }
    for (int idx = threadIdx.x; idx < tp * nz; idx += blockDim.x) {
        const int z = idx >> lgtp, ql = idx & (tp - 1), qg = q0 + ql;
        if (qg >= G.n2) continue;
        const long long gi = (long long)z * G.n2 + qg;
        const cplx<T> r = buf[ql * ld + z];
        a.out[gi] = r.x;
        if (a.dzout) a.dzout[gi] = r.y;
        if (a.phi_variant) {
            const cplx<T> rw = buf[(tp + ql) * ld + z];
            a.out2[gi] = rw.x;
            if (a.dzout2) a.dzout2[gi] = rw.y;
            a.out3[gi] = rw.x + a.S_eta2 * r.x + a.Q2n[gi];
        }
    }
}

// ---- ensembles of independent 2D runs (blockIdx.y = run): no z transform ---------------------
// forward: out = scale_p * (DSSUM X0) - (liftb[i] vb_p + liftt[i] vt_p) Mx[j]   (X1, when given,
// is DSSUM'd nodal Q2 copied to out1 for the phi step)
template <typename T>
struct IndepFwd {
    long long cs_x0, cs_out;   // strides between components (blockIdx.z)
    const T *X0;          // element-local
    const T *X1;          // nodal (copied to out1) or nullptr
    const T *scale_p;     // per-run scale or nullptr (then 1)
    const T *liftb, *liftt, *vb_p, *vt_p;   // lifting (nullable)
    T *out, *out1;
};

template <typename T>
__global__ void k_fwd_indep(Geo<T> G, IndepFwd<T> a) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= G.n2 || plane_frozen(G)) return;
    const int p = blockIdx.y;
    int s[4];
    dss_sources(G, q, s);
    const long long lplane = (long long)G.ex * G.ey * G.p * G.p;
    const long long gi = (long long)p * G.n2 + q;
    T v = gather4(a.X0 + blockIdx.z * a.cs_x0, p * lplane, s);
    if (a.scale_p) v *= a.scale_p[p];
    if (a.liftb) {
        const int i = q / G.nx, j = q % G.nx;
        v -= (a.liftb[i] * a.vb_p[p] + a.liftt[i] * a.vt_p[p]) * G.Mx[j];
    }
    a.out[blockIdx.z * a.cs_out + gi] = v;
    if (a.out1) a.out1[gi] = a.X1[gi];
}

template <typename T>
struct IndepInv {
    long long cs_y, cs_out;   // strides between components (blockIdx.z)
    const T *Y;               // solution planes
    int drow0, drow1;         // Dirichlet rows (-1: none) receiving v0_p / v1_p
    const T *v0_p, *v1_p;
    T *out;
    T *cur;                   // level n of the same field (frozen runs swap it with out)
    // phi variant
    const T *psi, *Q2n;
    T alpha, S_eta2;
    T *outW, *outL;
};

template <typename T>
__global__ void k_inv_indep(Geo<T> G, IndepInv<T> a) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= G.n2) return;
    const int p = blockIdx.y;
    const long long gi = (long long)p * G.n2 + q;
    if (plane_frozen(G)) {
        // the run has stopped: exchange its two history levels, so that after the slots change
        // roles it holds the same level n and n - 1 as before this step
        const long long o = blockIdx.z * a.cs_out + gi;
        const T t = a.out[o];
        a.out[o] = a.cur[o];
        a.cur[o] = t;
        return;
    }
    T x = a.Y[blockIdx.z * a.cs_y + gi];
    const int i = q / G.nx;
    if (a.drow0 >= 0 && i == a.drow0) x += a.v0_p[p];
    if (a.drow1 >= 0 && i == a.drow1) x += a.v1_p[p];
    a.out[blockIdx.z * a.cs_out + gi] = x;
    if (a.outW) {
        const T ps = a.psi[gi];
        const T W = ps - (a.alpha + a.S_eta2) * x - a.Q2n[gi];
        a.outW[gi] = W;
        a.outL[gi] = ps - a.alpha * x;
    }
}

// wall face slots of every run summed along x (no z transform)
template <typename T>
__global__ void k_face_indep(Geo<T> G, const T *__restrict__ face, T *__restrict__ out) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= G.nx || plane_frozen(G)) return;
    const int p = blockIdx.y, K = G.K, pp = G.p;
    const long long base = (long long)p * G.ex;
    T v;
    if (j % K == 0) v = face[(base + j / K) * pp] + face[(base + (j / K - 1 + G.ex) % G.ex) * pp + K];
    else v = face[(base + j / K) * pp + j % K];
    out[(long long)p * G.nx + j] = v;
}

// per-plane FP64 max |x| (or sum M x with kind 0), one block per plane
template <typename T>
__global__ void k_reduce_planes(const T *__restrict__ x, const T *__restrict__ y, const T *__restrict__ Mx,
                                const T *__restrict__ My, int nx, int n2, int kind, double *__restrict__ out) {
    __shared__ double sm[256];
    const int p = blockIdx.x;
    const T *xp = x + (long long)p * n2;
    const T *yp = y ? y + (long long)p * n2 : nullptr;
    double acc = 0.0;
    for (int i = threadIdx.x; i < n2; i += blockDim.x) {
        if (kind == 0) {
            acc += (double)Mx[i % nx] * (double)My[i / nx] * (double)xp[i];
        } else {
            const double v = yp ? fabs((double)xp[i] - (double)yp[i]) : fabs((double)xp[i]);
            if (acc == acc) {
                if (v != v) acc = v;
                else if (v > acc) acc = v;
            }
        }
    }
    sm[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            const double a = sm[threadIdx.x], b = sm[threadIdx.x + s];
            sm[threadIdx.x] = kind == 0 ? a + b : ((a != a || b != b) ? (a != a ? a : b) : fmax(a, b));
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) out[p] = sm[0];
}

// Per-run exit of an ensemble (one block per run, after the run's step): the run's FP64 max |u|
// (equilibrium system: max |phi^{n+1} - phi^n| / dt) against *tol; a run that falls below it, or
// whose value is not finite, is frozen (active = 0) and its step count recorded in steps_at
// (-2 when not finite).  count[p] counts the steps the run has taken.
template <typename T>
__global__ void k_batch_check(const T *__restrict__ a0, const T *__restrict__ a1, const T *__restrict__ phin,
                              double inv_dt, int n2, const double *__restrict__ tol, int *__restrict__ active,
                              int *__restrict__ count, int *__restrict__ steps_at) {
    const int p = blockIdx.x;
    if (!active[p]) return;
    __shared__ double sm[256];
    const long long off = (long long)p * n2;
    double m = 0.0;
    for (int i = threadIdx.x; i < n2; i += blockDim.x) {
        double v;
        if (phin) v = fabs((double)a0[off + i] - (double)phin[off + i]) * inv_dt;
        else v = fmax(fabs((double)a0[off + i]), fabs((double)a1[off + i]));
        if (!(v == v) || isinf(v)) v = INFINITY;   // not finite: stops the run
        m = fmax(m, v);
    }
    sm[threadIdx.x] = m;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sm[threadIdx.x] = fmax(sm[threadIdx.x], sm[threadIdx.x + s]);
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const int c = ++count[p];
        if (isinf(sm[0])) {
            active[p] = 0;
            steps_at[p] = -2;
        } else if (sm[0] < *tol) {
            active[p] = 0;
            steps_at[p] = c;
        }
    }
}

// z-FFT of the wall face slots (direct stiffness summation along x first)
template <typename T>
__global__ void k_face_fft(Geo<T> G, const T *__restrict__ face, T *__restrict__ out, const cplx<T> *tw,
                           int tp) {
    extern __shared__ unsigned char pf_smem_raw[];
    cplx<T> *stw = reinterpret_cast<cplx<T> *>(pf_smem_raw);
    const int nz = G.nz, ld = nz + 1;
    cplx<T> *buf = stw + (nz > 1 ? nz / 2 : 1);
    const bool pow2 = (nz & (nz - 1)) == 0;
    cplx<T> *tmp = buf + tp * ld;   // mixed-radix scratch (nz not 2^k)
    const int bits = 31 - __clz(nz);
    for (int i = threadIdx.x; i < nz / 2; i += blockDim.x) stw[i] = tw[i];
    const int j0 = blockIdx.x * tp;
    const int lgtp = 31 - __clz(tp);          // tp is a power of two
    for (int idx = threadIdx.x; idx < tp * nz; idx += blockDim.x) {
        const int z = idx >> lgtp, jl = idx & (tp - 1), j = j0 + jl;
        T v = 0;
        if (j < G.nx) {
            const int K = G.K, p = G.p;
            const long long base = (long long)z * G.ex;
            if (j % K == 0) {
                v = face[(base + j / K) * p] + face[(base + (j / K - 1 + G.ex) % G.ex) * p + K];
            } else {
                v = face[(base + j / K) * p + j % K];
            }
        }
        buf[jl * ld + fft_slot(z, bits, pow2)] = {v, T(0)};
    }
    __syncthreads();
    if (nz > 1) {
        if (pow2) fft_pencils(buf, ld, tp, nz, stw, false);
        else fft_pencils_mixed(buf, tmp, ld, tp, nz, stw, false);
    }
    const T inv_n = T(1) / T(nz);
    for (int idx = threadIdx.x; idx < tp * nz; idx += blockDim.x) {
        const int p = idx >> lgtp, jl = idx & (tp - 1), j = j0 + jl;
        if (j >= G.nx) continue;
        int k, im;
        plane_mode(p, nz, k, im);
        const cplx<T> zk = buf[jl * ld + k];
        out[(long long)p * G.nx + j] = (im ? zk.y : zk.x) * inv_n;
    }
}

// ---- C = A B, B small (N x N) shared by all rows; A is Mrows x N row-major -----------------
// store: 0 plain C[m][n]; 1 transposed within planes of R rows: C[p][n][r], m = p R + r.
// div: if lamN != nullptr, C[m][n] /= lamN[n] + lamR[r] + cpl[p]  (0 when the sum is 0).
template <typename T>
struct GemmArgs {
    const T *A, *B;
    T *C;
    long long Mrows;
    int N, R, store;
    const T *lamN, *lamR, *cpl;
    int cpl_mod;   // plane index for cpl: p % cpl_mod
    // optional second plain-store output C2 = -m2x[n] m2y[r] C (+ face2[p N + n] where r == 0):
    // the phi right-hand side -M psi (+ wall term) written by the psi solve's last transform
    T *C2;
    const T *m2x, *m2y, *face2;
    const int *active;   // ensembles: per-run flags (0 = frozen), run = plane % amod; null otherwise
    int amod;
};

// ensembles: true when every row of the tile [m0, m0 + BM) belongs to a frozen run (plane = m / R)
template <typename T>
__device__ __forceinline__ bool tile_frozen(const GemmArgs<T> &g, long long m0, int BM) {
    if (!g.active) return false;
    const long long p1 = (min(m0 + BM, g.Mrows) - 1) / g.R;
    for (long long p = m0 / g.R; p <= p1; ++p)
        if (g.active[p % g.amod]) return false;
    return true;
}

template <typename T, int BM, int BN, int BK, int TM, int TN>
__global__ void __launch_bounds__((BM / TM) * (BN / TN)) k_gemm(GemmArgs<T> g) {
    if (tile_frozen(g, (long long)blockIdx.y * BM, BM)) return;
    constexpr int NTH = (BM / TM) * (BN / TN);
    constexpr int LA = BM * BK / NTH;   // A elements staged per thread per k tile
    constexpr int LB = BK * BN / NTH;
    __shared__ T sA[2][BK][BM + 1];
    __shared__ T sB[2][BK][BN];
    const int tid = threadIdx.x;
    const int tx = tid % (BN / TN), ty = tid / (BN / TN);
    const long long m0 = (long long)blockIdx.y * BM;
    const int n0 = blockIdx.x * BN;
    // blocked summation: in FP32 each k tile is summed into `part` and then added to `acc` (the
    // rounding error of a length-n dot product grows with the block length plus the number of
    // blocks instead of n); in FP64 the whole k range is one block, i.e. plain sequential order
    T acc[TM][TN], part[TM][TN];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = part[i][j] = 0;
    T ra_[LA], rb_[LB];
    auto fetch = [&](int k0) {   // all loads of one k tile issued back to back
#pragma unroll
        for (int i = 0; i < LA; ++i) {
            const int idx = tid + NTH * i, r = idx / BK, c = idx % BK;
            const long long m = m0 + r;
            const int k = k0 + c;
            ra_[i] = (m < g.Mrows && k < g.N) ? g.A[m * g.N + k] : T(0);
        }
#pragma unroll
        for (int i = 0; i < LB; ++i) {
            const int idx = tid + NTH * i, r = idx / BN, c = idx % BN;
            const int k = k0 + r, n = n0 + c;
            rb_[i] = (k < g.N && n < g.N) ? g.B[(long long)k * g.N + n] : T(0);
        }
    };
    auto put = [&](int buf) {
#pragma unroll
        for (int i = 0; i < LA; ++i) {
            const int idx = tid + NTH * i;
            sA[buf][idx % BK][idx / BK] = ra_[i];
        }
#pragma unroll
        for (int i = 0; i < LB; ++i) {
            const int idx = tid + NTH * i;
            sB[buf][idx / BN][idx % BN] = rb_[i];
        }
    };
    fetch(0);
    put(0);
    __syncthreads();
    int buf = 0;
    for (int k0 = 0; k0 < g.N; k0 += BK) {
        const bool more = k0 + BK < g.N;
        if (more) fetch(k0 + BK);          // next tile in flight during this tile's FMAs
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            T ra[TM], rb[TN];
#pragma unroll
            for (int i = 0; i < TM; ++i) ra[i] = sA[buf][kk][ty * TM + i];
#pragma unroll
            for (int j = 0; j < TN; ++j) rb[j] = sB[buf][kk][tx * TN + j];
#pragma unroll
            for (int i = 0; i < TM; ++i)
#pragma unroll
                for (int j = 0; j < TN; ++j) part[i][j] += ra[i] * rb[j];
        }
        if (sizeof(T) == 4 || !more) {
#pragma unroll
            for (int i = 0; i < TM; ++i)
#pragma unroll
                for (int j = 0; j < TN; ++j) {
                    acc[i][j] += part[i][j];
                    part[i][j] = 0;
                }
        }
        if (more) put(buf ^ 1);
        __syncthreads();
        buf ^= 1;
    }
#pragma unroll
    for (int i = 0; i < TM; ++i) {
        const long long m = m0 + ty * TM + i;
        if (m >= g.Mrows) continue;
        const long long p = m / g.R;
        const int r = (int)(m - p * g.R);
        const T lr = g.lamN ? g.lamR[r] : T(0), cp = g.lamN ? g.cpl[p % g.cpl_mod] : T(0);   // once per row
#pragma unroll
        for (int j = 0; j < TN; ++j) {
            const int n = n0 + tx * TN + j;
            if (n >= g.N) continue;
            T v = acc[i][j];
            if (g.lamN) {
                const T d = g.lamN[n] + lr + cp;
                v = (d != T(0)) ? v / d : T(0);
            }
            if (g.store == 0) g.C[m * g.N + n] = v;
            else g.C[(p * g.N + n) * g.R + r] = v;
            if (g.C2) {
                T w = -g.m2x[n] * g.m2y[r] * v;
                if (g.face2 && r == 0) w += g.face2[p * g.N + n];
                g.C2[m * g.N + n] = w;
            }
        }
    }
}

// ---- the same transform GEMM with a cp.async multi-stage pipeline -----------------------------
// C = A B with the epilogues of k_gemm.  STAGES - 1 k tiles are in flight (global -> shared memory
// copies issued asynchronously), so the loop does not wait on the L2 latency of each tile.  A is
// kept row-major in shared memory ([m][k], rows padded to BK + PAD), B as [k][n]; VEC selects
// 16-byte copies (N a multiple of 16 / sizeof(T) and 16-byte aligned pointers), else one copy per
// element.  Out-of-range elements are zero-filled by the copy (source size 0).
__device__ __forceinline__ void cp_async_elem(void *sdst, const void *gsrc, int bytes, bool in) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(sdst);
    const int n = in ? bytes : 0;
    if (bytes == 16)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(gsrc), "r"(n) : "memory");
    else if (bytes == 8)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(d), "l"(gsrc), "r"(n) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(gsrc), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

template <typename T, int BM, int BN, int BK, int TM, int TN, int STAGES, bool VEC>
__global__ void __launch_bounds__((BM / TM) * (BN / TN)) k_gemm_cp(GemmArgs<T> g) {
    if (tile_frozen(g, (long long)blockIdx.y * BM, BM)) return;
    constexpr int NTH = (BM / TM) * (BN / TN);
    constexpr int VW = VEC ? 16 / (int)sizeof(T) : 1;   // elements per copy
    constexpr int PA = 16 / (int)sizeof(T);             // A row padding (keeps rows 16-byte aligned)
    constexpr int LDA = BK + PA;
    constexpr int CA = BM * BK / VW, CB = BK * BN / VW;  // copies per tile
    static_assert(TN * sizeof(T) % 16 == 0, "B fragment is read as 16-byte vectors");
    __shared__ __align__(16) T sA[STAGES][BM][LDA];
    __shared__ __align__(16) T sB[STAGES][BK][BN];
    const int tid = threadIdx.x;
    const int tx = tid % (BN / TN), ty = tid / (BN / TN);
    const long long m0 = (long long)blockIdx.y * BM;
    const int n0 = blockIdx.x * BN;
    const int KT = (g.N + BK - 1) / BK;
    auto load = [&](int slot, int kt) {
        const int k0 = kt * BK;
#pragma unroll
        for (int i = 0; i < (CA + NTH - 1) / NTH; ++i) {
            const int c = tid + NTH * i, r = c / (BK / VW), kc = (c % (BK / VW)) * VW;
            if (CA % NTH != 0 && c >= CA) break;
            const long long m = m0 + r;
            const bool in = m < g.Mrows && k0 + kc < g.N;
            cp_async_elem(&sA[slot][r][kc], in ? (const void *)(g.A + m * g.N + k0 + kc) : (const void *)g.A,
                          VW * (int)sizeof(T), in);
        }
#pragma unroll
        for (int i = 0; i < (CB + NTH - 1) / NTH; ++i) {
            const int c = tid + NTH * i, r = c / (BN / VW), nc = (c % (BN / VW)) * VW;
            if (CB % NTH != 0 && c >= CB) break;
            const bool in = k0 + r < g.N && n0 + nc < g.N;
            cp_async_elem(&sB[slot][r][nc], in ? (const void *)(g.B + (long long)(k0 + r) * g.N + n0 + nc)
                                               : (const void *)g.B,
                          VW * (int)sizeof(T), in);
        }
    };
    // blocked summation as in k_gemm: FP32 sums each k tile separately, FP64 in one block
    T acc[TM][TN], part[TM][TN];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = part[i][j] = 0;
#pragma unroll
    for (int s = 0; s < STAGES - 1; ++s) {
        if (s < KT) load(s, s);
        cp_async_commit();
    }
    for (int kt = 0; kt < KT; ++kt) {
        cp_async_wait<STAGES - 2>();
        __syncthreads();                       // tile kt landed for every thread; slot kt-1 is free
        const int nk = kt + STAGES - 1;
        if (nk < KT) load(nk % STAGES, nk);
        cp_async_commit();
        const int slot = kt % STAGES;
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            T ra[TM], rb[TN];
#pragma unroll
            for (int i = 0; i < TM; ++i) ra[i] = sA[slot][ty * TM + i][kk];
#pragma unroll
            for (int j = 0; j < TN; j += 16 / (int)sizeof(T)) {
                const float4 v = *reinterpret_cast<const float4 *>(&sB[slot][kk][tx * TN + j]);
                const T *pv = reinterpret_cast<const T *>(&v);
#pragma unroll
                for (int q = 0; q < 16 / (int)sizeof(T); ++q) rb[j + q] = pv[q];
            }
#pragma unroll
            for (int i = 0; i < TM; ++i)
#pragma unroll
                for (int j = 0; j < TN; ++j) part[i][j] += ra[i] * rb[j];
        }
        if (sizeof(T) == 4 || kt == KT - 1) {
#pragma unroll
            for (int i = 0; i < TM; ++i)
#pragma unroll
                for (int j = 0; j < TN; ++j) {
                    acc[i][j] += part[i][j];
                    part[i][j] = 0;
                }
        }
    }
    cp_async_wait<0>();
#pragma unroll
    for (int i = 0; i < TM; ++i) {
        const long long m = m0 + ty * TM + i;
        if (m >= g.Mrows) continue;
        const long long p = m / g.R;
        const int r = (int)(m - p * g.R);
        const T lr = g.lamN ? g.lamR[r] : T(0), cp = g.lamN ? g.cpl[p % g.cpl_mod] : T(0);   // once per row
#pragma unroll
        for (int j = 0; j < TN; ++j) {
            const int n = n0 + tx * TN + j;
            if (n >= g.N) continue;
            T v = acc[i][j];
            if (g.lamN) {
                const T d = g.lamN[n] + lr + cp;
                v = (d != T(0)) ? v / d : T(0);
            }
            if (g.store == 0) g.C[m * g.N + n] = v;
            else g.C[(p * g.N + n) * g.R + r] = v;
            if (g.C2) {
                T w = -g.m2x[n] * g.m2y[r] * v;
                if (g.face2 && r == 0) w += g.face2[p * g.N + n];
                g.C2[m * g.N + n] = w;
            }
        }
    }
}

// dst(t, src(t)) for t < n by the whole block, U independent global loads in flight per thread
// before their shared-memory stores (a plain strided loop waits on each load in turn)
template <int U, typename T, typename Src, typename Dst>
__device__ __forceinline__ void block_stage(int n, Src src, Dst dst) {
    for (int t0 = threadIdx.x; t0 < n; t0 += U * blockDim.x) {
        T v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int t = t0 + u * (int)blockDim.x;
            v[u] = t < n ? src(t) : T(0);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int t = t0 + u * (int)blockDim.x;
            if (t < n) dst(t, v[u]);
        }
    }
}

// ---- fused y-direction pair of a fast-diagonalisation solve ------------------------------------
// For BM rows of A (rows m = p R + r, length ny): t = A_m Sy, t /= (lamN[n] + lamR[r] + cpl[p]),
// out = t SyT stored transposed within planes: C[p][n][r].  Sy, SyT, the row block and t stay in
// shared memory; thread (row, column group of CG columns).  Used when 2 ny^2 + 2 BM ny values fit.
template <typename T, int BM, int CG>
__global__ void k_fdm_y(const T *__restrict__ A, const T *__restrict__ Sy, const T *__restrict__ SyT,
                        T *__restrict__ C, long long Mrows, int ny, int R, const T *__restrict__ lamN,
                        const T *__restrict__ lamR, const T *__restrict__ cpl, int cpl_mod,
                        const int *__restrict__ active) {
    if (active) {   // ensembles: skip a block whose rows all belong to frozen runs
        const long long b0 = (long long)blockIdx.x * BM, b1 = (min(b0 + BM, Mrows) - 1) / R;
        bool any = false;
        for (long long p = b0 / R; p <= b1 && !any; ++p) any = active[p % cpl_mod] != 0;
        if (!any) return;
    }
    extern __shared__ unsigned char pf_smem_raw[];
    T *sS = reinterpret_cast<T *>(pf_smem_raw);    // ny x ny
    T *sST = sS + ny * ny;                         // ny x ny
    T *sA = sST + ny * ny;                         // BM x ny
    T *sT = sA + BM * ny;                          // BM x ny
    const int tid = threadIdx.x;
    const long long m0 = (long long)blockIdx.x * BM;
    block_stage<8, T>(ny * ny, [&](int i) { return Sy[i]; }, [&](int i, T v) { sS[i] = v; });
    block_stage<8, T>(ny * ny, [&](int i) { return SyT[i]; }, [&](int i, T v) { sST[i] = v; });
    block_stage<8, T>(BM * ny, [&](int i) { return m0 + i / ny < Mrows ? A[m0 * ny + i] : T(0); },
                      [&](int i, T v) { sA[i] = v; });
    __syncthreads();
    const int ngrp = (ny + CG - 1) / CG;
    const int row = tid / ngrp, grp = tid - row * ngrp;
    const bool act = row < BM;
    const int c0 = grp * CG;
    const long long m = m0 + row;
    long long p = 0;
    int r = 0;
    if (act && m < Mrows) {
        p = m / R;
        r = (int)(m - p * R);
    }
    // blocked summation as in k_gemm: blocks of 16 terms in FP32, one block in FP64
    constexpr int KB = sizeof(T) == 4 ? 16 : (1 << 30);
    T acc[CG], part[CG];
    if (act) {
#pragma unroll
        for (int j = 0; j < CG; ++j) acc[j] = 0;
        for (int i0 = 0; i0 < ny; i0 += KB) {
#pragma unroll
            for (int j = 0; j < CG; ++j) part[j] = 0;
            const int i1 = min(ny, i0 + KB);
            for (int i = i0; i < i1; ++i) {
                const T a = sA[row * ny + i];
#pragma unroll
                for (int j = 0; j < CG; ++j)
                    if (c0 + j < ny) part[j] += a * sS[i * ny + c0 + j];
            }
#pragma unroll
            for (int j = 0; j < CG; ++j) acc[j] += part[j];
        }
        const T base = lamR[r] + cpl[p % cpl_mod];
#pragma unroll
        for (int j = 0; j < CG; ++j) {
            const int n = c0 + j;
            if (n < ny) {
                const T d = lamN[n] + base;
                sT[row * ny + n] = (d != T(0)) ? acc[j] / d : T(0);
            }
        }
    }
    __syncthreads();
    if (!act || m >= Mrows) return;
#pragma unroll
    for (int j = 0; j < CG; ++j) acc[j] = 0;
    for (int i0 = 0; i0 < ny; i0 += KB) {
#pragma unroll
        for (int j = 0; j < CG; ++j) part[j] = 0;
        const int i1 = min(ny, i0 + KB);
        for (int i = i0; i < i1; ++i) {
            const T t = sT[row * ny + i];
#pragma unroll
            for (int j = 0; j < CG; ++j)
                if (c0 + j < ny) part[j] += t * sST[i * ny + c0 + j];
        }
#pragma unroll
        for (int j = 0; j < CG; ++j) acc[j] += part[j];
    }
#pragma unroll
    for (int j = 0; j < CG; ++j) {
        const int n = c0 + j;
        if (n < ny) C[(p * ny + n) * R + r] = acc[j];
    }
}

// ---- a whole fast-diagonalisation solve per mode plane, in shared memory ----------------------
// out[p] = Sy [ (Sy^T rhs[p] Sx) / (Ly + Lx + c_p) ] Sx^T for plane p = blockIdx.x (FP32), with the
// optional second output C2 = -Mx My out (+ face2 on row 0) of the psi solve.  The plane stays in
// shared memory through the four transforms.  Warp w owns rows 8w..8w+7 of each stage's output, lane
// l the columns l + 32q (q < CQ), so the per-lane operand is read without bank conflicts and the
// per-warp operand is a broadcast (four k at a time where it is a row).  Sx is stored with its
// columns XOR-swizzled by the row (c ^ (r & 31)) so that its rows (x stage) and its columns (x^T
// stage) are both conflict-free.  Shared layout (floats): Sx nxp^2, Sy nyp^2, plane nyp x nxp, with
// nxp = 32 CQ and nyp = ny rounded up to 8; the padding is zero.
__host__ __device__ constexpr int fdm_plane_nyp(int ny) { return (ny + 7) & ~7; }

template <int CQ>
__global__ void __launch_bounds__(512) k_fdm_plane(const float *__restrict__ rhs, float *__restrict__ out, int nx,
                                                     int ny, const float *__restrict__ Sx,
                                                     const float *__restrict__ Sy, const float *__restrict__ Lx,
                                                     const float *__restrict__ Ly, const float *__restrict__ cpl,
                                                     int cpl_mod, float *__restrict__ C2,
                                                     const float *__restrict__ Mx, const float *__restrict__ My,
                                                     const float *__restrict__ face2,
                                                     const int *__restrict__ run_active) {
    if (run_active && !run_active[blockIdx.x % cpl_mod]) return;   // ensembles: a frozen run
    constexpr int NXP = 32 * CQ, RW = 8;
    extern __shared__ __align__(16) unsigned char pf_smem_raw[];
    const int nyp = fdm_plane_nyp(ny);
    float *sSx = reinterpret_cast<float *>(pf_smem_raw);
    float *sSy = sSx + NXP * NXP;
    float *pl = sSy + nyp * nyp;
    const int p = blockIdx.x, lane = threadIdx.x & 31, w = threadIdx.x >> 5, i0 = RW * w;
    const long long n2 = (long long)nx * ny;
    block_stage<8, float>(
        NXP * NXP, [&](int t) { const int r = t / NXP, c = t % NXP; return (r < nx && c < nx) ? Sx[r * nx + c] : 0.f; },
        [&](int t, float v) { const int r = t / NXP, c = t % NXP; sSx[r * NXP + (c ^ (r & 31))] = v; });
    block_stage<8, float>(
        nyp * nyp, [&](int t) { const int r = t / nyp, c = t - r * nyp; return (r < ny && c < ny) ? Sy[r * ny + c] : 0.f; },
        [&](int t, float v) { sSy[t] = v; });
    block_stage<8, float>(
        nyp * NXP,
        [&](int t) {
            const int r = t / NXP, c = t % NXP;
            return (r < ny && c < nx) ? rhs[p * n2 + (long long)r * nx + c] : 0.f;
        },
        [&](int t, float v) { pl[t] = v; });
    __syncthreads();
    // blocked summation: each block of 16 k is summed into `part`, then added to `acc`
    constexpr int KB = 16;
    float acc[RW][CQ], part[RW][CQ];
    auto zero = [&](float (&x)[RW][CQ]) {
#pragma unroll
        for (int r = 0; r < RW; ++r)
#pragma unroll
            for (int q = 0; q < CQ; ++q) x[r][q] = 0.f;
    };
    auto flush = [&]() {
#pragma unroll
        for (int r = 0; r < RW; ++r)
#pragma unroll
            for (int q = 0; q < CQ; ++q) {
                acc[r][q] += part[r][q];
                part[r][q] = 0.f;
            }
    };
    // acc = (rows i0.. of) L R, L row-major in shared memory with leading dimension ldl (a multiple
    // of 4) read four k at a time; R(k, j) given by rk
    auto rows_times = [&](const float *L, int ldl, int kdim, auto rk) {
        zero(acc);
        zero(part);
        for (int k0 = 0; k0 < kdim; k0 += 4) {
            if (k0 > 0 && k0 % KB == 0) flush();
            float4 a[RW];
#pragma unroll
            for (int r = 0; r < RW; ++r) a[r] = *reinterpret_cast<const float4 *>(L + (i0 + r) * ldl + k0);
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
                float b[CQ];
#pragma unroll
                for (int q = 0; q < CQ; ++q) b[q] = rk(k0 + kk, lane + 32 * q);
#pragma unroll
                for (int r = 0; r < RW; ++r) {
                    const float av = kk == 0 ? a[r].x : kk == 1 ? a[r].y : kk == 2 ? a[r].z : a[r].w;
#pragma unroll
                    for (int q = 0; q < CQ; ++q) part[r][q] += av * b[q];
                }
            }
        }
        flush();
    };
    auto put = [&]() {   // acc -> plane rows i0.., after every warp has read the old plane
        __syncthreads();
#pragma unroll
        for (int r = 0; r < RW; ++r)
#pragma unroll
            for (int q = 0; q < CQ; ++q)
                if (i0 + r < ny && lane + 32 * q < nx) pl[(i0 + r) * NXP + lane + 32 * q] = acc[r][q];
        __syncthreads();
    };
    const bool active = i0 < nyp;
    // x: t1[i][j'] = sum_j rhs[i][j] Sx[j][j']
    if (active) rows_times(pl, NXP, nx, [&](int k, int j) { return sSx[k * NXP + (j ^ (k & 31))]; });
    put();
    // y and the eigenvalue division: t2[i'][j'] = sum_i Sy[i][i'] t1[i][j'] / (Ly[i'] + Lx[j'] + c)
    if (active) {
        zero(acc);
        zero(part);
        for (int k = 0; k < ny; ++k) {
            if (k > 0 && k % KB == 0) flush();
            const float4 s0 = *reinterpret_cast<const float4 *>(sSy + k * nyp + i0);
            const float4 s1 = *reinterpret_cast<const float4 *>(sSy + k * nyp + i0 + 4);
            const float sv[RW] = {s0.x, s0.y, s0.z, s0.w, s1.x, s1.y, s1.z, s1.w};
            float b[CQ];
#pragma unroll
            for (int q = 0; q < CQ; ++q) b[q] = pl[k * NXP + lane + 32 * q];
#pragma unroll
            for (int r = 0; r < RW; ++r)
#pragma unroll
                for (int q = 0; q < CQ; ++q) part[r][q] += sv[r] * b[q];
        }
        flush();
        const float c = cpl[p % cpl_mod];
#pragma unroll
        for (int r = 0; r < RW; ++r)
#pragma unroll
            for (int q = 0; q < CQ; ++q) {
                const int i = i0 + r, j = lane + 32 * q;
                if (i < ny && j < nx) {
                    const float d = Ly[i] + Lx[j] + c;
                    acc[r][q] = (d != 0.f) ? acc[r][q] / d : 0.f;
                }
            }
    }
    put();
    // y^T: t3[i][j'] = sum_i' Sy[i][i'] t2[i'][j']
    if (active) rows_times(sSy, nyp, ny, [&](int k, int j) { return pl[k * NXP + j]; });
    put();
    // x^T: out[i][j] = sum_j' t3[i][j'] Sx[j][j']
    if (active) {
        rows_times(pl, NXP, nx, [&](int k, int j) { return sSx[j * NXP + (k ^ (j & 31))]; });
#pragma unroll
        for (int r = 0; r < RW; ++r)
#pragma unroll
            for (int q = 0; q < CQ; ++q) {
                const int i = i0 + r, j = lane + 32 * q;
                if (i >= ny || j >= nx) continue;
                const long long o = p * n2 + (long long)i * nx + j;
                out[o] = acc[r][q];
                if (C2) {
                    float v = -Mx[j] * My[i] * acc[r][q];
                    if (face2 && i == 0) v += face2[(long long)p * nx + j];
                    C2[o] = v;
                }
            }
    }
}

// ---- a fast-diagonalisation solve per mode plane on a cluster of CL thread blocks ----------------
// out[p] = Sy [ (Sy^T rhs[p] Sx) / (Ly + Lx + c_p) ] Sx^T (FP32) with the optional second output of
// k_gemm.  The cluster of plane p = blockIdx.x / CL splits the plane: block r owns the rows
// [r RC, (r+1) RC) for the two x transforms and the columns [r XC, (r+1) XC) for the two y
// transforms (RC = ceil(ny / CL), XC = ceil(nx / CL)).  After the x transform every block writes
// its rows' pieces into the owners' column buffers (distributed shared memory), after the y^T
// transform the pieces go back into the owners' row buffers; two cluster barriers order these
// exchanges.  Shared memory (floats): Sx NXP^2 (columns XOR-swizzled by the row, as in
// k_fdm_plane), Sy ny^2, row buffer RC x NXP, column buffer ny x XC.  Each k sum is blocked by 16.
// Every thread passes the same three cluster barriers and two block barriers (no early exit).
template <int CL, int CQ>
__global__ void __launch_bounds__(256) k_fdm_cluster(const float *__restrict__ rhs, float *__restrict__ out, int nx,
                                                      int ny, const float *__restrict__ Sx,
                                                      const float *__restrict__ Sy, const float *__restrict__ Lx,
                                                      const float *__restrict__ Ly, const float *__restrict__ cpl,
                                                      int cpl_mod, float *__restrict__ C2,
                                                      const float *__restrict__ Mx, const float *__restrict__ My,
                                                      const float *__restrict__ face2,
                                                      const int *__restrict__ run_active) {
    if (run_active && !run_active[(blockIdx.x / CL) % cpl_mod]) return;   // ensembles: a frozen run (whole cluster)
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    constexpr int NXP = 32 * CQ, NW = 8, KB = 16;
    constexpr int RTX = 64 / NW;                 // x stages: up to 64 rows per block
    constexpr int RTY = 128 / NW;                // y stages: up to 128 rows (ny)
    constexpr int CQY = CL >= 4 ? 1 : 2;         // y stages: up to 32 CQY columns per block
    extern __shared__ __align__(16) unsigned char pf_smem_raw[];
    const int rank = (int)cl.block_rank();
    const int p = blockIdx.x / CL;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int RC = (ny + CL - 1) / CL, XC = (nx + CL - 1) / CL;
    const int row0 = rank * RC, nrow = max(0, min(RC, ny - row0));
    const int col0 = rank * XC, ncol = max(0, min(XC, nx - col0));
    const long long n2 = (long long)nx * ny;
    float *sSx = reinterpret_cast<float *>(pf_smem_raw);
    float *sSy = sSx + NXP * NXP;
    float *rowb = sSy + ny * ny;
    float *colb = rowb + RC * NXP;
    block_stage<8, float>(
        NXP * NXP, [&](int t) { const int r = t / NXP, c = t % NXP; return (r < nx && c < nx) ? Sx[r * nx + c] : 0.f; },
        [&](int t, float v) { const int r = t / NXP, c = t % NXP; sSx[r * NXP + (c ^ (r & 31))] = v; });
    block_stage<8, float>(ny * ny, [&](int t) { return Sy[t]; }, [&](int t, float v) { sSy[t] = v; });
    block_stage<8, float>(
        RC * NXP,
        [&](int t) {
            const int r = t / NXP, c = t % NXP;
            return (r < nrow && c < nx) ? rhs[p * n2 + (long long)(row0 + r) * nx + c] : 0.f;
        },
        [&](int t, float v) { rowb[t] = v; });
    cl.sync();   // every block of the cluster is running and has its operands

    // x: T1[i][j'] = sum_j rhs[i][j] Sx[j][j'] for my rows; pieces to the column owners
    {
        float acc[RTX][CQ], part[RTX][CQ];
#pragma unroll
        for (int t = 0; t < RTX; ++t)
#pragma unroll
            for (int q = 0; q < CQ; ++q) acc[t][q] = part[t][q] = 0.f;
        for (int k = 0; k < nx; ++k) {
            if (k > 0 && k % KB == 0) {
#pragma unroll
                for (int t = 0; t < RTX; ++t)
#pragma unroll
                    for (int q = 0; q < CQ; ++q) { acc[t][q] += part[t][q]; part[t][q] = 0.f; }
            }
            float b[CQ];
#pragma unroll
            for (int q = 0; q < CQ; ++q) {
                const int j = lane + 32 * q;
                b[q] = sSx[k * NXP + (j ^ (k & 31))];
            }
#pragma unroll
            for (int t = 0; t < RTX; ++t) {
                const int i = w + NW * t;
                if (i < nrow) {
                    const float a = rowb[i * NXP + k];
#pragma unroll
                    for (int q = 0; q < CQ; ++q) part[t][q] += a * b[q];
                }
            }
        }
#pragma unroll
        for (int t = 0; t < RTX; ++t)
#pragma unroll
            for (int q = 0; q < CQ; ++q) {
                const int i = w + NW * t, j = lane + 32 * q;
                if (i < nrow && j < nx) {
                    const int s = j / XC;
                    cl.map_shared_rank(colb, s)[(row0 + i) * XC + (j - s * XC)] = acc[t][q] + part[t][q];
                }
            }
    }
    cl.sync();   // column buffers complete

    // y and the eigenvalue division: T2[i'][j'] = sum_i Sy[i][i'] T1[i][j'] / (Ly[i'] + Lx[j'] + c),
    // then y^T: T3[i][j'] = sum_i' Sy[i][i'] T2[i'][j'], for my columns
    const float c = cpl[p % cpl_mod];
    for (int pass = 0; pass < 2; ++pass) {
        float acc[RTY][CQY], part[RTY][CQY];
#pragma unroll
        for (int t = 0; t < RTY; ++t)
#pragma unroll
            for (int q = 0; q < CQY; ++q) acc[t][q] = part[t][q] = 0.f;
        for (int k = 0; k < ny; ++k) {
            if (k > 0 && k % KB == 0) {
#pragma unroll
                for (int t = 0; t < RTY; ++t)
#pragma unroll
                    for (int q = 0; q < CQY; ++q) { acc[t][q] += part[t][q]; part[t][q] = 0.f; }
            }
            float b[CQY];
#pragma unroll
            for (int q = 0; q < CQY; ++q) {
                const int j = lane + 32 * q;
                b[q] = j < XC ? colb[k * XC + j] : 0.f;
            }
#pragma unroll
            for (int t = 0; t < RTY; ++t) {
                const int i = w + NW * t;
                if (i < ny) {
                    const float a = pass == 0 ? sSy[k * ny + i] : sSy[i * ny + k];
#pragma unroll
                    for (int q = 0; q < CQY; ++q) part[t][q] += a * b[q];
                }
            }
        }
        if (pass == 0) {
            __syncthreads();   // every thread has read the column buffer
#pragma unroll
            for (int t = 0; t < RTY; ++t)
#pragma unroll
                for (int q = 0; q < CQY; ++q) {
                    const int i = w + NW * t, j = lane + 32 * q;
                    if (i < ny && j < ncol) {
                        const float d = Ly[i] + Lx[col0 + j] + c;
                        const float v = acc[t][q] + part[t][q];
                        colb[i * XC + j] = (d != 0.f) ? v / d : 0.f;
                    }
                }
            __syncthreads();
        } else {
#pragma unroll
            for (int t = 0; t < RTY; ++t)
#pragma unroll
                for (int q = 0; q < CQY; ++q) {
                    const int i = w + NW * t, j = lane + 32 * q;
                    if (i < ny && j < ncol) {
                        const int r = i / RC;
                        cl.map_shared_rank(rowb, r)[(i - r * RC) * NXP + col0 + j] = acc[t][q] + part[t][q];
                    }
                }
        }
    }
    cl.sync();   // row buffers complete; no shared memory of another block is touched after this

    // x^T: out[i][j] = sum_j' T3[i][j'] Sx[j][j'] for my rows
    {
        float acc[RTX][CQ], part[RTX][CQ];
#pragma unroll
        for (int t = 0; t < RTX; ++t)
#pragma unroll
            for (int q = 0; q < CQ; ++q) acc[t][q] = part[t][q] = 0.f;
        for (int k = 0; k < nx; ++k) {
            if (k > 0 && k % KB == 0) {
#pragma unroll
                for (int t = 0; t < RTX; ++t)
#pragma unroll
                    for (int q = 0; q < CQ; ++q) { acc[t][q] += part[t][q]; part[t][q] = 0.f; }
            }
            float b[CQ];
#pragma unroll
            for (int q = 0; q < CQ; ++q) {
                const int j = lane + 32 * q;
                b[q] = sSx[j * NXP + (k ^ (j & 31))];
            }
#pragma unroll
            for (int t = 0; t < RTX; ++t) {
                const int i = w + NW * t;
                if (i < nrow) {
                    const float a = rowb[i * NXP + k];
#pragma unroll
                    for (int q = 0; q < CQ; ++q) part[t][q] += a * b[q];
                }
            }
        }
#pragma unroll
        for (int t = 0; t < RTX; ++t)
#pragma unroll
            for (int q = 0; q < CQ; ++q) {
                const int i = w + NW * t, j = lane + 32 * q;
                if (i >= nrow || j >= nx) continue;
                const int y = row0 + i;
                const long long o = p * n2 + (long long)y * nx + j;
                const float v = acc[t][q] + part[t][q];
                out[o] = v;
                if (C2) {
                    float u = -Mx[j] * My[y] * v;
                    if (face2 && y == 0) u += face2[(long long)p * nx + j];
                    C2[o] = u;
                }
            }
    }
}

// ---- electrode patches: capacitance correction of the potential (eq. 21) ----------------------
// Plane p = blockIdx.x.  y: base solution with the whole wall Dirichlet at the values w[p][:]
// (electrode voltages in plane 0, the previous gap values); rhs: its right-hand side, whose wall
// row is b_G - Ky[0][0] Mx[j] w[j] (the forward transform's lifting).  For gap node j:
//   s_j = b_G,j - (A_G,wall w)_j - (A_GI y)_j,
//   (A_G,wall w)_j = My[0] sum_l Kx[j][l] w[l] + Mx[j] (Ky[0][0] + c_p My[0]) w[j],
//   (A_GI y)_j = Mx[j] sum_{i >= 1} Ky[0][i] y[i][j];
// the Ky[0][0] part is already in rhs.
// d = Cinv_p s (m x m), and the right-hand side of the correction solve
// rhs2[i][j] = Ky[i][0] Mx[j] d_j on gap columns (i >= 1), 0 elsewhere.
template <typename T>
__global__ void k_cap_solve(Geo<T> G, const T *__restrict__ rhs, const T *__restrict__ y, const int *__restrict__ gapj,
                            const int *__restrict__ gapidx, int m, const T *__restrict__ w,
                            const T *__restrict__ Kx, const T *__restrict__ Ky0, T my0,
                            const T *__restrict__ sh, const T *__restrict__ Cinv, T *__restrict__ d,
                            T *__restrict__ rhs2) {
    extern __shared__ unsigned char pf_smem_raw[];
    T *s = reinterpret_cast<T *>(pf_smem_raw);
    T *ds = s + m;
    const int p = blockIdx.x, nx = G.nx, ny = G.ny;
    const long long base = (long long)p * G.n2;
    const T *wp = w + (long long)p * nx;
    const T c = sh[p];
    const int imax = min(G.K, ny - 1);   // K_y[0][i] vanishes beyond the first element
    for (int jj = threadIdx.x; jj < m; jj += blockDim.x) {
        const int j = gapj[jj];
        T acc = 0;
        for (int i = 1; i <= imax; ++i) acc += Ky0[i] * y[base + (long long)i * nx + j];
        T kw = 0;
        if (nx > 2 * G.K) {   // K_x couples j only with the nodes of its element(s): j - K .. j + K
            for (int d = -G.K; d <= G.K; ++d) {
                const int l = (j + d + nx) % nx;
                kw += Kx[(long long)j * nx + l] * wp[l];
            }
        } else {
            for (int l = 0; l < nx; ++l) kw += Kx[(long long)j * nx + l] * wp[l];
        }
        s[jj] = rhs[base + j] - G.Mx[j] * acc - my0 * kw - G.Mx[j] * c * my0 * wp[j];
    }
    __syncthreads();
    const T *Ci = Cinv + (long long)p * m * m;
    for (int jj = threadIdx.x; jj < m; jj += blockDim.x) {
        T acc = 0;
        for (int ll = 0; ll < m; ++ll) acc += Ci[(long long)jj * m + ll] * s[ll];
        ds[jj] = acc;
        d[(long long)p * m + jj] = acc;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int i = threadIdx.x >> 5; i < ny; i += nw) {
        for (int j = lane; j < nx; j += 32) {
            const int jj = gapidx[j];
            rhs2[base + (long long)i * nx + j] = (i >= 1 && jj >= 0) ? Ky0[i] * G.Mx[j] * ds[jj] : T(0);
        }
    }
}

// V = y - z off the wall (z nullable: no gap nodes); on the wall w + d (d on gaps only), and w
// takes the new gap values
template <typename T>
__global__ void k_cap_combine(Geo<T> G, const T *y, const T *z, const T *__restrict__ d, const int *__restrict__ gapidx,
                              int m, T *__restrict__ w, T *out, long long total) {
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const long long p = t / G.n2;
        const int q = (int)(t - p * G.n2), i = q / G.nx, j = q - (q / G.nx) * G.nx;
        if (i > 0) {
            out[t] = z ? y[t] - z[t] : y[t];
        } else {
            const int jj = gapidx[j];
            T v = w[p * G.nx + j];
            if (jj >= 0) {
                v += d[p * m + jj];
                w[p * G.nx + j] = v;
            }
            out[t] = v;
        }
    }
}

// ---- FP64 reductions (two passes, deterministic) --------------------------------------------
// kind 0: sum of w[q % n2w] * x[q] (phase mass, w = nodal mass); kind 1: max |x|; kind 2: max |x - y|
// A non-finite entry propagates as NaN through every kind.
template <typename T>
__global__ void k_reduce(const T *__restrict__ x, const T *__restrict__ y, const T *__restrict__ w1,
                         const T *__restrict__ w2, int nx, int n2w, long long n, int kind,
                         double *__restrict__ part) {
    __shared__ double sm[256];
    double acc = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        double v;
        if (kind == 0) {
            const int q = (int)(i % n2w);
            v = (double)w1[q % nx] * (double)w2[q / nx] * (double)x[i];
            acc += v;
        } else {
            v = (kind == 1) ? fabs((double)x[i]) : fabs((double)x[i] - (double)y[i]);
            if (acc == acc) {   // once NaN, stays NaN
                if (v != v) acc = v;
                else if (v > acc) acc = v;
            }
        }
    }
    sm[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            double a = sm[threadIdx.x], b = sm[threadIdx.x + s];
            if (kind == 0) sm[threadIdx.x] = a + b;
            else sm[threadIdx.x] = (a != a || b != b) ? (a != a ? a : b) : fmax(a, b);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sm[0];
}

// ---- eq. 14: the discrete energy E(t) (diagnostic; FP64 arithmetic and accumulation) -------
// Per element, with GLL quadrature and element-local derivatives:
//   sum_{a,b} w_a w_b (h_x/2)(h_y/2) [ rho(phi)|u|^2/2 + lambda|grad phi|^2/2
//                                       + lambda (phi^2 - 1)^2 / (4 eta^2) + eps(phi)|E|^2/2 ]
// plus, on the wall row of the wall elements, sum_a w_a (h_x/2) Theta(phi) with
// Theta = sigma cos(theta_s) phi (phi^2 - 3)/4 (eq. theta_def, constant dropped).  3D: d/dz phi is
// the spectral derivative at the node; the caller multiplies by the plane weight Lz/Nz.
// One partial sum per block (blockIdx.y = plane), summed in order on the host.
struct EnergyConst {
    double rho1, rho2, eps1, eps2, lam, inv_eta2, sigma_cos;
};

template <typename T>
__global__ void k_energy(Geo<T> G, EnergyConst c, const T *__restrict__ phi, const T *__restrict__ dzphi,
                         const T *__restrict__ ux, const T *__restrict__ uy, const T *__restrict__ uz,
                         const T *__restrict__ Ex, const T *__restrict__ Ey, const T *__restrict__ Ez,
                         double *__restrict__ part) {
    PF_ELEM_SMEM(T, G, 1)
    T *sP = sF;
    load_tables(G, sD, sDw, sw);
    const ElemIdx e = elem_index(G);
    if (e.act) sP[e.t] = phi[e.g];
    __syncthreads();
    double v = 0.0;
    if (e.act) {
        const double hx = (double)G.hx[e.ex], hy = (double)G.hy[e.ey];
        double gx = 0.0, gy = 0.0;
        for (int m = 0; m < G.p; ++m) {
            gx += (double)sD[e.a * G.p + m] * (double)sP[e.b * G.p + m];
            gy += (double)sD[e.b * G.p + m] * (double)sP[m * G.p + e.a];
        }
        gx *= 2.0 / hx;
        gy *= 2.0 / hy;
        const double gz = dzphi ? (double)dzphi[e.g] : 0.0;
        const double f = (double)phi[e.g];
        const double u0 = (double)ux[e.g], u1 = (double)uy[e.g], u2 = uz ? (double)uz[e.g] : 0.0;
        const double e0 = (double)Ex[e.g], e1 = (double)Ey[e.g], e2 = Ez ? (double)Ez[e.g] : 0.0;
        const double rho = 0.5 * (c.rho1 + c.rho2) + 0.5 * (c.rho1 - c.rho2) * f;
        const double eps = 0.5 * (c.eps1 + c.eps2) + 0.5 * (c.eps1 - c.eps2) * f * (3.0 - f * f) / 2.0;
        const double w2 = f * f - 1.0;
        const double dens = 0.5 * rho * (u0 * u0 + u1 * u1 + u2 * u2) + 0.5 * c.lam * (gx * gx + gy * gy + gz * gz) +
                            c.lam * c.inv_eta2 / 4.0 * w2 * w2 + 0.5 * eps * (e0 * e0 + e1 * e1 + e2 * e2);
        v = (double)sw[e.a] * (double)sw[e.b] * (0.5 * hx) * (0.5 * hy) * dens;
        if (e.ey == 0 && e.b == 0) v += (double)sw[e.a] * (0.5 * hx) * c.sigma_cos * f * (f * f - 3.0) / 4.0;
    }
    __shared__ double red[32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
        part[(size_t)blockIdx.y * gridDim.x + blockIdx.x] = t;
    }
}

template <typename T, typename S>
__global__ void k_convert(const T *__restrict__ in, S *__restrict__ out, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = (S)in[i];
}

}  // namespace pf
