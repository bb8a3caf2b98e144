// C-ABI of the decoupled phase-field step (declarations and contracts in include/pf.h).
//
// One handle owns an Engine<T> (T = double for PF_FP64, float for PF_MIXED) that
// holds every device array of the step: 1D tables, eigenbases, the two BDF history
// levels of the state, element-local right-hand sides and mode-plane work arrays.
// A step is the kernel sequence of Algorithm 1 / Algorithm 2:
//   k_potential -> k_fwd -> FDM -> k_inv (V, Ez) -> k_efield (Ex, Ey)
//   k_chem -> k_fwd (psi RHS, Q2 modes) -> FDM (psi; its last transform also writes the phi
//   right-hand side -M psi) -> FDM (phi) -> k_inv (phi, dphi/dz, W, dW/dz, L)
//   k_momentum -> k_fwd -> FDM (P) -> k_inv (P)
//   k_ugradp -> k_fwd (all components) -> FDM (u, batched) -> k_inv (all components)
// The new level is written over level n-1, then the two levels swap roles.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <string>
#include <type_traits>
#include <vector>

#include "../../include/pf.h"
#include "pf_kernels.cuh"
#include "pf_tc.cuh"

using pf::cplx;

namespace {

std::string g_create_error;

struct CudaError {
    cudaError_t code;
    std::string where;
};

#define PF_CU(call)                                                                  \
    do {                                                                             \
        cudaError_t e_ = (call);                                                     \
        if (e_ != cudaSuccess) {                                                     \
            cudaGetLastError(); /* a non-sticky error must not resurface later */    \
            throw CudaError{e_, std::string(#call)};                                 \
        }                                                                            \
    } while (0)

// Raise (never lower) a kernel's dynamic shared-memory limit.  The limit belongs to the function,
// not to an engine: lowering it for a small mesh would make a larger engine's launches invalid.
void raise_smem_limit(const void *fn, size_t bytes) {
    if (bytes <= 48 * 1024) return;
    cudaFuncAttributes fa{};
    PF_CU(cudaFuncGetAttributes(&fa, fn));
    if ((size_t)fa.maxDynamicSharedSizeBytes < bytes)
        PF_CU(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
}

// cuTensorMapEncodeTiled from the driver, through the runtime (no link against libcuda); null when
// the driver does not provide it
using EncodeTiled = PFN_cuTensorMapEncodeTiled_v12000;
EncodeTiled tc_encode() {
    static EncodeTiled fn = [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            cudaGetLastError();
            p = nullptr;
        }
        return reinterpret_cast<EncodeTiled>(p);
    }();
    return fn;
}

int num_sms() {
    int dev = 0, n = 0;
    PF_CU(cudaGetDevice(&dev));
    PF_CU(cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev));
    return n;
}

struct HostSetup {
    int ex, ey, K, p, nx, ny, nz;
    double lz;
    std::vector<double> xb, yb, xi, w, D, Dw, hx, hy;
    std::vector<double> Kx, Mx, Ky, My;          // assembled 1D operators
    std::vector<double> Sx, Lx;                  // periodic x eigenbasis
    std::vector<double> Sy[4], Ly[4];            // y eigenbases per bcset
    std::vector<double> X, Y;                    // node coordinates
    std::vector<double> liftV;                   // K_y[:, D] * V_D (potential lifting)
    int vrow0 = -1, vrow1 = -1;                  // Dirichlet rows of the potential
    double v0 = 0, v1 = 0;
    // electrode patches on the wall (eq. 21): intervals and voltages; gap nodes and the
    // capacitance (Schur-complement) inverses of the gap rows, one m x m block per mode plane
    bool patch = false;
    std::vector<double> px0, px1, pv;
    std::vector<int> gapj, gapidx;               // gap node x-indices; x-index -> gap index or -1
    std::vector<double> vbx, Ky0, Cinv;          // wall voltages (0 on gaps), K_y[0][:], C^-1 per plane
    // physics
    double rho1, rho2, mu1, mu2, eps1, eps2, sigma, eta, gamma1, theta;
    double dt, S, nu_m, rho0, eps0, lam, cos_theta;
    int bdf, precision;
    int model = PF_MODEL_FULL;
    // ensemble of independent 2D runs (batch > 0): per-run permittivities and voltages
    int batch = 0;
    std::vector<double> beps1, beps2, bvb, bvt;
};

double alpha_of(const HostSetup &s, int J) {
    // alpha of eq. 44; a discriminant below 1e-10 is taken as 0
    const double g0 = J == 1 ? 1.0 : 1.5;
    double disc = 1.0 - 4.0 * g0 * std::pow(s.eta, 4.0) / (s.lam * s.gamma1 * s.dt * std::pow(s.S, 2.0));
    if (disc < 1e-10) disc = 0.0;
    return -s.S / (2.0 * std::pow(s.eta, 2.0)) * (1.0 + std::sqrt(disc));
}

template <typename T>
T *dalloc(size_t n) {
    T *p = nullptr;
    PF_CU(cudaMalloc(&p, std::max<size_t>(n, 1) * sizeof(T)));
    return p;
}

template <typename T>
T *dupload(const std::vector<double> &v, cudaStream_t st) {
    std::vector<T> h(v.begin(), v.end());
    T *d = dalloc<T>(h.size());
    PF_CU(cudaMemcpyAsync(d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, st));
    PF_CU(cudaStreamSynchronize(st));
    return d;
}

// Per-class launch counters and optional CUDA-event timers of the kernels a handle launches.
struct Prof {
    bool on = false;
    long long launches[PF_KC_COUNT] = {};
    double ms[PF_KC_COUNT] = {};
    std::vector<cudaEvent_t> pool;
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> pending;
    cudaEvent_t ev_begin = nullptr;
    int kc_open = -1;

    cudaEvent_t take() {
        if (pool.empty()) {
            cudaEvent_t e;
            PF_CU(cudaEventCreate(&e));
            return e;
        }
        cudaEvent_t e = pool.back();
        pool.pop_back();
        return e;
    }
    void begin(int kc, cudaStream_t st) {
        launches[kc] += 1;
        if (!on) return;
        ev_begin = take();
        kc_open = kc;
        PF_CU(cudaEventRecord(ev_begin, st));
    }
    void end(cudaStream_t st) {
        if (!on || kc_open < 0) return;
        cudaEvent_t e = take();
        PF_CU(cudaEventRecord(e, st));
        pending.push_back({kc_open, {ev_begin, e}});
        kc_open = -1;
        if (pending.size() > 4096) resolve();
    }
    void resolve() {
        for (auto &p : pending) {
            PF_CU(cudaEventSynchronize(p.second.second));
            float t = 0.f;
            PF_CU(cudaEventElapsedTime(&t, p.second.first, p.second.second));
            ms[p.first] += t;
            pool.push_back(p.second.first);
            pool.push_back(p.second.second);
        }
        pending.clear();
    }
    ~Prof() {
        for (auto &p : pending) { cudaEventDestroy(p.second.first); cudaEventDestroy(p.second.second); }
        for (auto e : pool) cudaEventDestroy(e);
    }
};

template <typename T>
struct Engine {
    const HostSetup &hs;
    Prof *prof = nullptr;
    cudaStream_t st;
    int ex, ey, K, p, nx, ny, n2, nz;
    long long N, NL;
    bool d3;
    std::vector<void *> allocs;
    // tables
    T *hx, *hy, *D, *Dw, *w, *Mx, *My;
    T *Sx, *SxT, *Lx, *Sy[4], *SyT[4], *Ly[4];
    T *liftV;
    cplx<T> *tw;
    T *shV, *shP, *shPsi[2], *shPhi[2], *shU[2], *shTmp;
    // electrode patches: gap tables, wall voltages, capacitance inverses, gap values per plane
    int npatch_gap = 0;
    int *gapj = nullptr, *gapidx = nullptr;
    T *Ky0 = nullptr, *Kxd = nullptr, *Cinv = nullptr, *gbuf = nullptr;
    T *wallw = nullptr;   // wall values per mode plane [nz][nx]: electrode voltages (plane 0), last gap values
    // state: level slots [0], [1]; cur = slot of level n
    T *V[2], *Ez[2], *phi[2], *dzphi[2], *P[2], *dzP[2], *u[3][2], *dzu[3][2];
    T *Ex, *Ey, *W, *dzW, *Lf, *Q2;
    T *LA, *LB, *LAU[3], *LBU[3], *faceU;
    T *RHS, *OUT, *PSIH, *Q2H, *FACEH, *W1, *W2;
    // ensemble planes (indep): per-plane permittivities, 1/eps0, voltages, lifting columns
    bool indep = false;
    T *peps1 = nullptr, *peps2 = nullptr, *peps0 = nullptr, *pscale = nullptr, *pvb = nullptr, *pvt = nullptr;
    T *liftb = nullptr, *liftt = nullptr;
    // ensembles: per-run exit on the device (pf_batch_run_to_equilibrium): run flags (0 = frozen),
    // steps taken, exit step (-1 none, -2 not finite), and the tolerance (< 0: none)
    int *active = nullptr, *run_count = nullptr, *steps_at = nullptr;
    double *tol_dev = nullptr;
    double *red;
    int *dev_err;   // device error word (bounded waits)
    int cur = 0;
    // 3xTF32 tensor-core transforms: for each B matrix (an eigenbasis or its transpose), B^T split
    // into TF32 head and tail, zero padded to Npad x Kpad, with its TMA descriptors
    struct TcB {
        const T *key;
        float *hi, *lo;
        int N, BN, BNlast, ntn, Npad, Kpad, stages, tmem_cols, nr;
        size_t smem;
        CUtensorMap mh, ml;
    };
    std::vector<TcB> tcb;
    bool use_tc = false;
    // TMEM accumulation of the tensor-core transforms, per variant (index 0: PF_GEMM_TC, 1:
    // PF_GEMM_TC_HYBRID) and solve family (index 0: the psi and phi solves of the Cahn-Hilliard
    // pair, whose errors feed phi directly; 1: V, P and u): 8-wide K slices per group, and whether
    // the correction products chain in a per-tile region of their own (pf::TcArgs::sep).  The
    // hybrid runs the psi and phi solves on CUDA cores, so its index-0 entries are unused.
    int tc_gs[2][2] = {{2, 8}, {4, 4}};
    int tc_sepv[2][2] = {{1, 1}, {0, 0}};
    int tc_group = 2;                 // of the solve being launched
    int tc_sep = 1;
    int tc_stall = 0;                 // test hook: the next tensor-core launch reports a time-out
    unsigned long long tc_wait_ns = 1000000000ull;   // bound of every wait (1 s)
    unsigned long long tc_wait_ns_next = 0;          // the test hook's bound
    int nyp = 0;                      // row pitch of the y-transform intermediates (multiple of 4)
    int sms = 0;                      // multiprocessors of the device (persistent grid)
    // TMA descriptors of the A operands, by (base, rows, K, pitch)
    struct AMap {
        const void *ptr;
        long long rows;
        int K, pitch;
        CUtensorMap map;
    };
    std::vector<AMap> amaps;
    int simt_tile = 0;   // SIMT GEMM tile: 0 heuristic, 32 or 64 forced (autotuner)
    int tp_override = 0; // pencils per transform block: 0 heuristic, else forced (autotuner)
    // steady-state (BDF2) step captured once per history-slot parity; replayed by pf_step
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    long long graph_launches[2][PF_KC_COUNT] = {};

    // one BDF2 step through the captured graph of the current slot parity (captured on first use)
    void step_graph() {
        const int c = cur;
        if (!graph[c]) {
            long long before[PF_KC_COUNT];
            for (int k = 0; k < PF_KC_COUNT; ++k) before[k] = prof->launches[k];
            cudaGraph_t g = nullptr;
            PF_CU(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
            try {
                step(2);
            } catch (...) {
                cudaStreamEndCapture(st, &g);
                if (g) cudaGraphDestroy(g);
                cur = c;
                throw;
            }
            PF_CU(cudaStreamEndCapture(st, &g));
            cudaError_t e = cudaGraphInstantiate(&graph[c], g, 0);
            cudaGraphDestroy(g);
            PF_CU(e);
            for (int k = 0; k < PF_KC_COUNT; ++k) {
                graph_launches[c][k] = prof->launches[k] - before[k];
                prof->launches[k] = before[k];
            }
            cur = c;   // the capture did not run anything
        }
        PF_CU(cudaGraphLaunch(graph[c], st));
        for (int k = 0; k < PF_KC_COUNT; ++k) prof->launches[k] += graph_launches[c][k];
        cur = 1 - c;
    }

    template <typename U>
    U *mk(size_t n) {
        U *q = dalloc<U>(n);
        allocs.push_back(q);
        PF_CU(cudaMemsetAsync(q, 0, std::max<size_t>(n, 1) * sizeof(U), st));
        return q;
    }
    T *up(const std::vector<double> &v) {
        T *q = dupload<T>(v, st);
        allocs.push_back(q);
        return q;
    }

    Engine(const HostSetup &s, cudaStream_t stream, Prof *pr) : hs(s), prof(pr), st(stream) {
        ex = s.ex; ey = s.ey; K = s.K; p = s.p; nx = s.nx; ny = s.ny;
        indep = s.batch > 0;
        nz = indep ? s.batch : s.nz;   // planes: Fourier planes, or the runs of an ensemble
        n2 = nx * ny;
        N = (long long)n2 * nz;
        NL = (long long)ex * ey * p * p * nz;
        d3 = !indep && nz > 1;
        hx = up(s.hx); hy = up(s.hy); D = up(s.D); Dw = up(s.Dw); w = up(s.w);
        Mx = up(s.Mx); My = up(s.My);
        std::vector<double> tmp;
        Sx = up(s.Sx);
        tmp.assign(s.Sx.size(), 0.0);
        for (int i = 0; i < nx; ++i)
            for (int j = 0; j < nx; ++j) tmp[(size_t)i * nx + j] = s.Sx[(size_t)j * nx + i];
        SxT = up(tmp);
        Lx = up(s.Lx);
        for (int b = 0; b < 4; ++b) {
            Sy[b] = up(s.Sy[b]);
            tmp.assign(s.Sy[b].size(), 0.0);
            for (int i = 0; i < ny; ++i)
                for (int j = 0; j < ny; ++j) tmp[(size_t)i * ny + j] = s.Sy[b][(size_t)j * ny + i];
            SyT[b] = up(tmp);
            Ly[b] = up(s.Ly[b]);
        }
        liftV = up(s.liftV);
        if (s.patch) {
            npatch_gap = (int)s.gapj.size();
            gapj = mk<int>(std::max(1, npatch_gap));
            gapidx = mk<int>(nx);
            if (npatch_gap > 0)
                PF_CU(cudaMemcpyAsync(gapj, s.gapj.data(), s.gapj.size() * sizeof(int), cudaMemcpyHostToDevice, st));
            PF_CU(cudaMemcpyAsync(gapidx, s.gapidx.data(), s.gapidx.size() * sizeof(int), cudaMemcpyHostToDevice, st));
            PF_CU(cudaStreamSynchronize(st));
            Ky0 = up(s.Ky0); Kxd = up(s.Kx); Cinv = up(s.Cinv);
            gbuf = mk<T>((size_t)nz * std::max(1, npatch_gap));
            std::vector<double> w0((size_t)nz * nx, 0.0);
            std::copy(s.vbx.begin(), s.vbx.end(), w0.begin());
            wallw = up(w0);
        }
        if (indep) {
            std::vector<double> e0(nz), sc(nz), lb(ny, 0.0), lt(ny, 0.0);
            for (int q = 0; q < nz; ++q) {
                e0[q] = std::max(s.beps1[q], s.beps2[q]);
                sc[q] = 1.0 / e0[q];
            }
            peps1 = up(s.beps1); peps2 = up(s.beps2); peps0 = up(e0); pscale = up(sc);
            pvb = up(s.bvb); pvt = up(s.bvt);
            for (int i = 0; i < ny; ++i) {
                if (s.vrow0 >= 0) lb[i] = s.Ky[(size_t)i * ny + 0];
                if (s.vrow1 >= 0) lt[i] = s.Ky[(size_t)i * ny + (ny - 1)];
            }
            liftb = up(lb); liftt = up(lt);
            active = mk<int>(nz); run_count = mk<int>(nz); steps_at = mk<int>(nz); tol_dev = mk<double>(1);
            reset_exit(-1.0, 0);
        }
        {
            std::vector<cplx<T>> h(std::max(1, nz / 2));
            for (int k = 0; k < nz / 2; ++k) {
                const double ang = -2.0 * M_PI * k / nz;
                h[k] = {(T)std::cos(ang), (T)std::sin(ang)};
            }
            tw = mk<cplx<T>>(h.size());
            PF_CU(cudaMemcpyAsync(tw, h.data(), h.size() * sizeof(cplx<T>), cudaMemcpyHostToDevice, st));
        }
        // per-plane shifts c + beta_k^2 of every solve (3 blocks for the batched velocity)
        auto shifts = [&](double c) {
            std::vector<double> v(3 * nz);
            for (int pl = 0; pl < 3 * nz; ++pl) {
                const int pp = pl % nz;
                int k = 0;
                if (d3) k = (pp == 0) ? 0 : (pp == 1 ? nz / 2 : pp / 2);
                const double beta = d3 ? 2.0 * M_PI * k / s.lz : 0.0;
                v[pl] = c + beta * beta;
            }
            return up(v);
        };
        shV = shifts(0.0);
        shP = shifts(0.0);
        for (int J = 1; J <= 2; ++J) {
            const double al = alpha_of(s, J);
            const double g0 = J == 1 ? 1.0 : 1.5;
            shPsi[J - 1] = shifts(al + s.S / std::pow(s.eta, 2.0));
            shPhi[J - 1] = shifts(-al);
            shU[J - 1] = shifts(g0 / (s.nu_m * s.dt));
        }
        shTmp = mk<T>(3 * nz);
        for (int l = 0; l < 2; ++l) {
            V[l] = mk<T>(N); phi[l] = mk<T>(N); P[l] = mk<T>(N);
            for (int c = 0; c < 3; ++c) u[c][l] = nullptr;
            const int dcomp = d3 ? 3 : 2;
            T *ub = mk<T>((size_t)dcomp * N);   // components contiguous: batched transforms
            for (int c = 0; c < dcomp; ++c) u[c][l] = ub + (size_t)c * N;
            if (d3) {
                Ez[l] = mk<T>(N); dzphi[l] = mk<T>(N); dzP[l] = mk<T>(N);
                T *db = mk<T>((size_t)3 * N);
                for (int c = 0; c < 3; ++c) dzu[c][l] = db + (size_t)c * N;
            } else {
                Ez[l] = dzphi[l] = dzP[l] = nullptr;
                for (int c = 0; c < 3; ++c) dzu[c][l] = nullptr;
            }
        }
        if (!d3) { u[2][0] = u[2][1] = nullptr; }
        Ex = mk<T>(N); Ey = mk<T>(N); W = mk<T>(N); Lf = mk<T>(N); Q2 = mk<T>(N);
        dzW = d3 ? mk<T>(N) : nullptr;
        LA = mk<T>(NL);
        LB = d3 ? mk<T>(NL) : nullptr;
        {
            const int dcomp = d3 ? 3 : 2;
            T *la = mk<T>((size_t)dcomp * NL);
            T *lb = d3 ? mk<T>((size_t)3 * NL) : nullptr;
            for (int c = 0; c < 3; ++c) {
                LAU[c] = c < dcomp ? la + (size_t)c * NL : nullptr;
                LBU[c] = d3 ? lb + (size_t)c * NL : nullptr;
            }
        }
        faceU = mk<T>((size_t)ex * p * nz);
        nyp = (ny + 3) / 4 * 4;
        RHS = mk<T>(3 * N); OUT = mk<T>(3 * N);
        W1 = mk<T>((size_t)3 * nz * nx * nyp); W2 = mk<T>((size_t)3 * nz * nx * nyp);
        PSIH = mk<T>(N); Q2H = mk<T>(N); FACEH = mk<T>((size_t)nx * nz);
        if (fdm_y_smem() > 48 * 1024 && fdm_y_smem() <= 200 * 1024)
            raise_smem_limit((const void *)pf::k_fdm_y<T, 32, 8>, fdm_y_smem());
        {   // z-transform kernels: opt in once, before any graph capture
            const void *fns[] = {(const void *)pf::k_fwd<T, 0>, (const void *)pf::k_fwd<T, 4>,
                                 (const void *)pf::k_fwd<T, 5>, (const void *)pf::k_fwd<T, 6>,
                                 (const void *)pf::k_fwd<T, 7>, (const void *)pf::k_fwd<T, 8>,
                                 (const void *)pf::k_inv<T, 0>, (const void *)pf::k_inv<T, 4>,
                                 (const void *)pf::k_inv<T, 5>, (const void *)pf::k_inv<T, 6>,
                                 (const void *)pf::k_inv<T, 7>, (const void *)pf::k_inv<T, 8>,
                                 (const void *)pf::k_face_fft<T>};
            for (const void *fn : fns) raise_smem_limit(fn, FFT_SMEM_LIMIT);
        }
        if constexpr (sizeof(T) == 4) {
            if (plane_fits()) {   // opt in once, before any graph capture
                const int cq = plane_cq();
                const void *fn = cq == 1 ? (const void *)pf::k_fdm_plane<1>
                                 : cq == 2 ? (const void *)pf::k_fdm_plane<2> : (const void *)pf::k_fdm_plane<4>;
                raise_smem_limit(fn, fdm_plane_smem());
            }
            const int cq = plane_cq();
            if (cluster_fits(4)) {
                const void *fn = cq == 1 ? (const void *)pf::k_fdm_cluster<4, 1>
                                 : cq == 2 ? (const void *)pf::k_fdm_cluster<4, 2> : (const void *)pf::k_fdm_cluster<4, 4>;
                raise_smem_limit(fn, fdm_cluster_smem(4));
            }
            if (cluster_fits(2)) {
                const void *fn = cq == 1 ? (const void *)pf::k_fdm_cluster<2, 1>
                                 : cq == 2 ? (const void *)pf::k_fdm_cluster<2, 2> : (const void *)pf::k_fdm_cluster<2, 4>;
                raise_smem_limit(fn, fdm_cluster_smem(2));
            }
        }

        red = mk<double>(std::max<long long>(1024, nz));
        dev_err = mk<int>(1);
        use_tc = (sizeof(T) == 4) && s.precision == PF_MIXED && tc_possible();
        if (use_tc) {
            // B = Sx (Bt = Sx^T), B = Sx^T (Bt = Sx), B = Sy (Bt = Sy^T), B = Sy^T (Bt = Sy)
            auto tr = [](const std::vector<double> &m, int n) {
                std::vector<double> t((size_t)n * n);
                for (int i = 0; i < n; ++i)
                    for (int j = 0; j < n; ++j) t[(size_t)i * n + j] = m[(size_t)j * n + i];
                return t;
            };
            add_tc(Sx, tr(s.Sx, nx), nx);
            add_tc(SxT, s.Sx, nx);
            for (int b = 0; b < 4; ++b) {
                add_tc(Sy[b], tr(s.Sy[b], ny), ny);
                add_tc(SyT[b], s.Sy[b], ny);
            }
            size_t most = 0;
            for (auto &t : tcb) most = std::max(most, t.smem);
            raise_smem_limit((const void *)pf::k_gemm_tc, most);
        }
        PF_CU(cudaStreamSynchronize(st));
    }

    // host TF32 rounding to nearest, ties away from zero (the rounding of cvt.rna.tf32.f32)
    static float tf32_rna_host(float x) {
        uint32_t u;
        std::memcpy(&u, &x, 4);
        if ((u & 0x7F800000u) != 0x7F800000u) u = (u + 0x1000u) & 0xFFFFE000u;
        float r;
        std::memcpy(&r, &u, 4);
        return r;
    }

    // the tensor-core transforms need 16-byte row pitches for TMA: n_x a multiple of 4 (the
    // right-hand sides and solutions keep pitch n_x; the y intermediates are padded to nyp)
    bool tc_possible() const { return nx % 4 == 0 && tc_encode() != nullptr; }

    // column tiles of an N-column product: full tiles of BN = min(2 TC_MAXH, N rounded up to 16)
    // columns and a last one that holds the rest (a multiple of 16)
    static int tc_bn(int n, int *ntn, int *bnlast) {
        const int npad = (n + 15) / 16 * 16;
        const int bn = std::min(2 * pf::TC_MAXH, npad);
        *ntn = (npad + bn - 1) / bn;
        *bnlast = npad - (*ntn - 1) * bn;
        return bn;
    }

    static void encode_2d(CUtensorMap *m, const void *ptr, long long rows, int K, int pitch, int box_rows) {
        cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
        cuuint64_t strides[1] = {(cuuint64_t)pitch * 4};
        cuuint32_t box[2] = {(cuuint32_t)pf::TC_KC, (cuuint32_t)box_rows};
        cuuint32_t estr[2] = {1, 1};
        const CUresult r = tc_encode()(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void *>(ptr), dims, strides,
                                       box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                                       CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) throw CudaError{cudaErrorInvalidValue, "cuTensorMapEncodeTiled"};
    }

    // Bt (n x n row-major, FP64) -> TF32 head/tail on the device, padded to ntn BN rows and to
    // whole K chunks of 32, with the TMA descriptors of both halves
    void add_tc(const T *key, const std::vector<double> &Bt, int n) {
        TcB t;
        t.key = key;
        t.N = n;
        t.BN = tc_bn(n, &t.ntn, &t.BNlast);
        t.Npad = (t.ntn - 1) * t.BN + t.BNlast;
        t.Kpad = (n + pf::TC_KC - 1) / pf::TC_KC * pf::TC_KC;
        const size_t stage = (size_t)2 * pf::TC_BM * pf::TC_KC * 4 + (size_t)2 * t.BN * pf::TC_KC * 4;
        const size_t fixed = 1024 + 512;   // alignment slack, barriers, TMEM slot, abort flag
        t.stages = (int)std::min<size_t>(4, (size_t)(227 * 1024 - fixed) / stage);
        t.smem = t.stages * stage + fixed;
        t.tmem_cols = 512;                 // the ring of accumulation regions: one CTA per SM
        t.nr = std::min(pf::TC_MAXR, 512 / t.BN);
        std::vector<float> hi((size_t)t.Npad * t.Kpad, 0.f), lo((size_t)t.Npad * t.Kpad, 0.f);
        for (int r = 0; r < n; ++r)
            for (int k = 0; k < n; ++k) {
                const double v = Bt[(size_t)r * n + k];
                const float h = tf32_rna_host((float)v);
                hi[(size_t)r * t.Kpad + k] = h;
                lo[(size_t)r * t.Kpad + k] = tf32_rna_host((float)(v - (double)h));
            }
        t.hi = mk<float>(hi.size());
        t.lo = mk<float>(lo.size());
        PF_CU(cudaMemcpyAsync(t.hi, hi.data(), hi.size() * 4, cudaMemcpyHostToDevice, st));
        PF_CU(cudaMemcpyAsync(t.lo, lo.data(), lo.size() * 4, cudaMemcpyHostToDevice, st));
        PF_CU(cudaStreamSynchronize(st));
        encode_2d(&t.mh, t.hi, t.Npad, t.Kpad, t.Kpad, t.BN);
        encode_2d(&t.ml, t.lo, t.Npad, t.Kpad, t.Kpad, t.BN);
        tcb.push_back(t);
    }

    const CUtensorMap &amap(const T *ptr, long long rows, int K, int pitch) {
        for (auto &a : amaps)
            if (a.ptr == ptr && a.rows == rows && a.K == K && a.pitch == pitch) return a.map;
        AMap a;
        a.ptr = ptr; a.rows = rows; a.K = K; a.pitch = pitch;
        encode_2d(&a.map, ptr, rows, K, pitch, pf::TC_BM);
        amaps.push_back(a);
        return amaps.back().map;
    }

    // C = A B on the tensor cores (B one of the eigenbases registered by add_tc); A has `rows` rows
    // of K values at pitch lda; epilogue as pf::TcArgs
    void gemm_tc(const T *A, int lda, const T *B, T *C, long long rows, int R, int store, int ldc, int ldr,
                 const T *lamN, const T *lamR, const T *cpl, int cpl_mod, T *C2 = nullptr, const T *face2 = nullptr) {
        const TcB *tb = nullptr;
        for (auto &t : tcb)
            if (t.key == B) tb = &t;
        if (!tb) throw CudaError{cudaErrorInvalidValue, "tensor-core transform without its eigenbasis"};
        pf::TcArgs a{};
        if (rows >= (1ll << 31)) throw CudaError{cudaErrorInvalidValue, "tensor-core transform with 2^31 rows"};
        a.M = (int)rows; a.N = tb->N; a.BN = tb->BN; a.BNlast = tb->BNlast; a.ntn = tb->ntn;
        a.nchunk = tb->Kpad / pf::TC_KC;
        a.gs = tc_group; a.stages = tb->stages; a.tmem_cols = tb->tmem_cols;
        a.sep = tc_sep;
        a.nr = tc_sep ? std::min(pf::TC_MAXR, tb->tmem_cols / tb->BN - 2) : tb->nr;
        a.ntiles = (int)((rows + pf::TC_BM - 1) / pf::TC_BM * tb->ntn);
        a.R = R; a.store = store; a.ldc = ldc; a.ldr = ldr;
        a.lamN = reinterpret_cast<const float *>(lamN);
        a.lamR = reinterpret_cast<const float *>(lamR);
        a.cpl = reinterpret_cast<const float *>(cpl);
        a.cpl_mod = cpl_mod;
        a.C = reinterpret_cast<float *>(C);
        a.C2 = reinterpret_cast<float *>(C2);
        a.m2x = reinterpret_cast<const float *>(Mx);
        a.m2y = reinterpret_cast<const float *>(My);
        a.face2 = reinterpret_cast<const float *>(face2);
        a.err = dev_err;
        a.wait_ns = tc_stall ? tc_wait_ns_next : tc_wait_ns;
        a.stall = tc_stall;
        tc_stall = 0;
        const CUtensorMap &ma = amap(A, rows, tb->N, lda);
        if (sms == 0) sms = num_sms();
        const unsigned grid = (unsigned)std::min(a.ntiles, sms);
        prof->begin(PF_KC_GEMM, st);
        pf::k_gemm_tc<<<grid, pf::TC_THREADS, tb->smem, st>>>(ma, tb->mh, tb->ml, a);
        check_launch();
        prof->end(st);
    }

    // fast-diagonalisation solve on the tensor cores: the four transforms of fdm() with the y
    // intermediates at row pitch nyp (16-byte rows for TMA)
    void fdm_tc(const T *rhs, T *out, int bcset, const T *sh, long long P, T *minus_m_out, const T *face) {
        // the psi, phi pair, and with electrode patches the potential (whose capacitance correction
        // subtracts two solves), take the accurate family
        const int fam = (bcset == PF_BCSET_NN || (bcset == PF_BCSET_V && hs.patch)) ? 0 : 1;
        tc_group = tc_gs[tc_hybrid ? 1 : 0][fam];
        tc_sep = tc_sepv[tc_hybrid ? 1 : 0][fam];
        // x: W1[p][x][y] (pitch nyp) = (rhs[p][y][:] Sx)^T
        gemm_tc(rhs, nx, Sx, W1, P * ny, ny, 1, 0, nyp, nullptr, nullptr, nullptr, 1);
        // y with the eigenvalue division: W2[p][x][:] = (W1[p][x][:] Sy) / (Ly + Lx + shift)
        gemm_tc(W1, nyp, Sy[bcset], W2, P * nx, nx, 0, nyp, 0, Ly[bcset], Lx, sh, nz);
        // y^T: W1[p][y][x] (pitch nx) = (W2[p][x][:] Sy^T)^T
        gemm_tc(W2, nyp, SyT[bcset], W1, P * nx, nx, 1, 0, nx, nullptr, nullptr, nullptr, 1);
        // x^T: out[p][y][:] = W1[p][y][:] Sx^T (and the phi right-hand side -M psi (+ wall term))
        gemm_tc(W1, nx, SxT, out, P * ny, ny, 0, nx, 0, nullptr, nullptr, nullptr, 1, minus_m_out, face);
    }

    ~Engine() {
        for (int c = 0; c < 2; ++c)
            if (graph[c]) cudaGraphExecDestroy(graph[c]);
        for (void *q : allocs) cudaFree(q);
    }

    // ensembles: every run active, no exit recorded, step counts `count`, tolerance tol (< 0: only
    // non-finite runs stop)
    void reset_exit(double tol, int count) {
        std::vector<int> one(nz, 1), cnt(nz, count), none(nz, -1);
        PF_CU(cudaMemcpyAsync(active, one.data(), nz * sizeof(int), cudaMemcpyHostToDevice, st));
        PF_CU(cudaMemcpyAsync(run_count, cnt.data(), nz * sizeof(int), cudaMemcpyHostToDevice, st));
        PF_CU(cudaMemcpyAsync(steps_at, none.data(), nz * sizeof(int), cudaMemcpyHostToDevice, st));
        PF_CU(cudaMemcpyAsync(tol_dev, &tol, sizeof(double), cudaMemcpyHostToDevice, st));
        PF_CU(cudaStreamSynchronize(st));
    }
    // ensembles: per-run exit check after a step (the new level is in slot o, the old in slot n)
    void batch_check(int n, int o) {
        const bool eq = hs.model == PF_MODEL_EQUILIBRIUM;
        prof->begin(PF_KC_OTHER, st);
        pf::k_batch_check<T><<<nz, 256, 0, st>>>(eq ? phi[o] : u[0][o], eq ? nullptr : u[1][o], eq ? phi[n] : nullptr,
                                                 1.0 / hs.dt, n2, tol_dev, active, run_count, steps_at);
        check_launch();
        prof->end(st);
    }

    pf::Geo<T> geo() const {
        pf::Geo<T> g;
        g.ex = ex; g.ey = ey; g.K = K; g.p = p; g.nx = nx; g.ny = ny; g.n2 = n2; g.nz = nz;
        g.epb = epb();
        g.hx = hx; g.hy = hy; g.D = D; g.Dw = Dw; g.w = w; g.Mx = Mx; g.My = My;
        g.active = active;
        return g;
    }
    pf::Phys<T> phys(int J) const {
        pf::Phys<T> q;
        q.rho1 = (T)hs.rho1; q.rho2 = (T)hs.rho2; q.mu1 = (T)hs.mu1; q.mu2 = (T)hs.mu2;
        q.eps1 = (T)hs.eps1; q.eps2 = (T)hs.eps2; q.lam = (T)hs.lam;
        q.inv_eta2 = (T)(1.0 / std::pow(hs.eta, 2.0)); q.gamma1 = (T)hs.gamma1;
        q.S_eta2 = (T)(hs.S / std::pow(hs.eta, 2.0)); q.eps0 = (T)hs.eps0; q.rho0 = (T)hs.rho0;
        q.nu_m = (T)hs.nu_m; q.dt = (T)hs.dt; q.sigma = (T)hs.sigma; q.cos_theta = (T)hs.cos_theta;
        q.alpha = (T)alpha_of(hs, J); q.gamma0 = (T)(J == 1 ? 1.0 : 1.5); q.J = J;
        q.wetting = std::fabs(hs.cos_theta) > 1e-15 ? 1 : 0;
        q.eps1_p = peps1; q.eps2_p = peps2; q.eps0_p = peps0;
        return q;
    }

    // ---- launch helpers -----------------------------------------------------------------
    // element kernels: as many whole elements as fit in 256 threads per block
    int epb() const { return std::max(1, 256 / (p * p)); }
    int elem_threads() const { return ((epb() * p * p + 31) / 32) * 32; }
    size_t elem_smem(int nfields) const {
        return (size_t)(2 * p * p + 32 + (size_t)epb() * nfields * p * p) * sizeof(T);
    }
    dim3 elem_grid() const { return dim3((ex * ey + epb() - 1) / epb(), nz); }
    // pencils per transform block: enough blocks for 4 per SM, shared memory <= 24 KiB
    // log2(nz) for the transform kernels compiled for a fixed plane count (16..256), else 0
    int lgz() const {
        if (!nz_pow2() || nz < 16 || nz > 256) return 0;
        int l = 0;
        while ((1 << l) < nz) ++l;
        return l;
    }
    void launch_inv(dim3 grid, size_t smem, const pf::InvArgs<T> &a) {
        switch (lgz()) {
            case 4: pf::k_inv<T, 4><<<grid, 256, smem, st>>>(geo(), a); break;
            case 5: pf::k_inv<T, 5><<<grid, 256, smem, st>>>(geo(), a); break;
            case 6: pf::k_inv<T, 6><<<grid, 256, smem, st>>>(geo(), a); break;
            case 7: pf::k_inv<T, 7><<<grid, 256, smem, st>>>(geo(), a); break;
            case 8: pf::k_inv<T, 8><<<grid, 256, smem, st>>>(geo(), a); break;
            default: pf::k_inv<T, 0><<<grid, 256, smem, st>>>(geo(), a);
        }
    }
    // transform buffers of a non-power-of-two nz need a second (scratch) copy for the mixed radices
    bool nz_pow2() const { return (nz & (nz - 1)) == 0; }
    // row pitch of a pencil in the z-transform buffers (the kernels' pf::fft_ld)
    int fld() const { return (sizeof(T) == 4 && lgz() == 8) ? 289 : nz + 1; }
    size_t fft_scratch(int pencils) const { return nz_pow2() ? 0 : (size_t)pencils * (nz + 1) * sizeof(cplx<T>); }
    // shared memory of the z-transform pencils: 72 KB for 2^k planes (the FFT itself runs in
    // registers for FP32 32..256 planes), half of it for the mixed radices (a scratch copy)
    static constexpr int FFT_SMEM_BUDGET = 73728;
    static constexpr size_t FFT_SMEM_LIMIT = 96 * 1024;   // raised once per kernel at set-up
    int fwd_tp() const {
        int tp = (int)((nz_pow2() ? FFT_SMEM_BUDGET : FFT_SMEM_BUDGET / 2) / (sizeof(cplx<T>) * fld()));
        const int by_grid = tp_override > 0 ? tp_override : n2 / (4 * 152);
        if (tp > by_grid) tp = by_grid;
        if (tp > 64) tp = 64;
        if (tp < 4) tp = 4;
        int p2 = 4;                  // a power of two: the kernels index with shifts and masks
        while (p2 * 2 <= tp) p2 *= 2;
        return p2;
    }
    // element kernels compiled for the orders of the timed workloads (8, 10, 12), else generic
    template <typename F>
    void by_order(F f) {
        if (K == 8) f(std::integral_constant<int, 8>{});
        else if (K == 10) f(std::integral_constant<int, 10>{});
        else if (K == 12) f(std::integral_constant<int, 12>{});
        else f(std::integral_constant<int, 0>{});
    }
    void check_launch() { PF_CU(cudaGetLastError()); }

    void gemm(const T *A, const T *B, T *C, long long Mrows, int Ncol, int R, int store, const T *lamN,
              const T *lamR, const T *cpl, int cpl_mod, T *C2 = nullptr, const T *face2 = nullptr) {
        pf::GemmArgs<T> g{A, B, C, Mrows, Ncol, R, store, lamN, lamR, cpl, cpl_mod, C2, Mx, My, face2, active, nz};
        constexpr int BK = sizeof(T) == 8 ? 8 : 16;
        if (simt_tile >= 3 && simt_tile <= 5) {   // cp.async pipelines: 64x64, 32x32, 32x64 tiles
            constexpr int VWE = 16 / (int)sizeof(T);
            const bool vec = Ncol % VWE == 0 && ((uintptr_t)A % 16) == 0 && ((uintptr_t)B % 16) == 0;
            prof->begin(PF_KC_GEMM, st);
            if (Ncol > 64 && Ncol <= 80 && (simt_tile == 3 || simt_tile == 4)) {
                // one 80-wide column tile (e.g. the y transforms of n_y = 65) instead of a second,
                // nearly empty 64- or 32-wide one
                if (simt_tile == 3) {
                    dim3 grid(1, (unsigned)((Mrows + 63) / 64));
                    // FP32: k tiles of ceil(N / 5) so that five tiles hold N exactly (13 for N = 65)
                    const int bky = sizeof(T) == 4 ? (Ncol + 4) / 5 : BK;
                    if (vec) pf::k_gemm_cp<T, 64, 80, BK, 4, 4, 4, true><<<grid, 320, 0, st>>>(g);
                    else if (bky == 13) pf::k_gemm_cp<T, 64, 80, 13, 4, 4, 4, false><<<grid, 320, 0, st>>>(g);
                    else if (bky == 14) pf::k_gemm_cp<T, 64, 80, 14, 4, 4, 4, false><<<grid, 320, 0, st>>>(g);
                    else if (bky == 15) pf::k_gemm_cp<T, 64, 80, 15, 4, 4, 4, false><<<grid, 320, 0, st>>>(g);
                    else pf::k_gemm_cp<T, 64, 80, BK, 4, 4, 4, false><<<grid, 320, 0, st>>>(g);
                } else {
                    dim3 grid(1, (unsigned)((Mrows + 31) / 32));
                    if (vec) pf::k_gemm_cp<T, 32, 80, BK, 2, 4, 4, true><<<grid, 320, 0, st>>>(g);
                    else pf::k_gemm_cp<T, 32, 80, BK, 2, 4, 4, false><<<grid, 320, 0, st>>>(g);
                }
            } else if (simt_tile == 3) {
                dim3 grid((Ncol + 63) / 64, (unsigned)((Mrows + 63) / 64));
                if (vec) pf::k_gemm_cp<T, 64, 64, BK, 4, 4, 4, true><<<grid, 256, 0, st>>>(g);
                else pf::k_gemm_cp<T, 64, 64, BK, 4, 4, 4, false><<<grid, 256, 0, st>>>(g);
            } else if (simt_tile == 4) {
                dim3 grid((Ncol + 31) / 32, (unsigned)((Mrows + 31) / 32));
                if (vec) pf::k_gemm_cp<T, 32, 32, BK, 2, 4, 4, true><<<grid, 128, 0, st>>>(g);
                else pf::k_gemm_cp<T, 32, 32, BK, 2, 4, 4, false><<<grid, 128, 0, st>>>(g);
            } else {
                dim3 grid((Ncol + 63) / 64, (unsigned)((Mrows + 31) / 32));
                if (vec) pf::k_gemm_cp<T, 32, 64, BK, 2, 4, 4, true><<<grid, 256, 0, st>>>(g);
                else pf::k_gemm_cp<T, 32, 64, BK, 2, 4, 4, false><<<grid, 256, 0, st>>>(g);
            }
            check_launch();
            prof->end(st);
            return;
        }
        const long long tiles64 = ((Ncol + 63) / 64) * ((Mrows + 63) / 64);
        prof->begin(PF_KC_GEMM, st);
        const bool big = simt_tile == 64 || (simt_tile == 0 && tiles64 >= 4 * 152 && Ncol % 64 > 32);
        if (simt_tile == 2) {   // 32x64 tiles
            dim3 grid((Ncol + 63) / 64, (unsigned)((Mrows + 31) / 32));
            pf::k_gemm<T, 32, 64, BK, 2, 4><<<grid, 256, 0, st>>>(g);
        } else if (big) {
            dim3 grid((Ncol + 63) / 64, (unsigned)((Mrows + 63) / 64));
            pf::k_gemm<T, 64, 64, BK, 4, 4><<<grid, 256, 0, st>>>(g);
        } else {
            // small or ragged problems: 32x32 tiles give 4x the blocks and less padding
            dim3 grid((Ncol + 31) / 32, (unsigned)((Mrows + 31) / 32));
            pf::k_gemm<T, 32, 32, BK, 2, 2><<<grid, 256, 0, st>>>(g);
        }
        check_launch();
        prof->end(st);
    }

    // fast-diagonalisation solve of nplanes mode planes: out = S_y [ (S_y^T rhs S_x) / (L_y + L_x + c_p) ] S_x^T
    // shared memory of the fused y pair (Sy, SyT, row block, intermediate)
    size_t fdm_y_smem() const { return (size_t)(2 * ny * ny + 2 * 32 * ny) * sizeof(T); }
    bool fuse_y = true;   // the autotuner may turn the fused y pair off
    // the whole-plane solve (FP32 only): columns per lane, shared memory (Sx, Sy, one plane)
    int plane_cq() const { return nx <= 32 ? 1 : nx <= 64 ? 2 : 4; }
    size_t fdm_plane_smem() const {
        const size_t nxp = 32 * plane_cq(), nyp = pf::fdm_plane_nyp(ny);
        return (nxp * nxp + nyp * nyp + nyp * nxp) * sizeof(float);
    }
    bool plane_fits() const {
        return sizeof(T) == 4 && nx <= 128 && ny <= 128 && fdm_plane_smem() <= 227 * 1024;
    }
    bool fuse_plane = false;   // chosen by the autotuner when it is faster
    // the cluster solve (FP32): CL blocks per plane; shared memory per block
    int cluster = 0;
    size_t fdm_cluster_smem(int CL) const {
        const size_t nxp = 32 * plane_cq(), rc = (ny + CL - 1) / CL, xc = (nx + CL - 1) / CL;
        return (nxp * nxp + (size_t)ny * ny + rc * nxp + (size_t)ny * xc) * sizeof(float);
    }
    bool cluster_fits(int CL) const {
        return sizeof(T) == 4 && (CL == 2 || CL == 4) && nx <= 128 && ny <= 128 && nx >= CL && ny >= CL &&
               fdm_cluster_smem(CL) <= 227 * 1024;
    }
    template <int CL, int CQ>
    void launch_cluster(const T *rhs, T *out, int bcset, const T *sh, long long P, T *c2, const T *face) {
        if constexpr (sizeof(T) == 4) {
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3((unsigned)(P * CL));
            cfg.blockDim = dim3(256);
            cfg.dynamicSmemBytes = fdm_cluster_smem(CL);
            cfg.stream = st;
            cudaLaunchAttribute at[1];
            at[0].id = cudaLaunchAttributeClusterDimension;
            at[0].val.clusterDim.x = CL;
            at[0].val.clusterDim.y = 1;
            at[0].val.clusterDim.z = 1;
            cfg.attrs = at;
            cfg.numAttrs = 1;
            PF_CU(cudaLaunchKernelEx(&cfg, pf::k_fdm_cluster<CL, CQ>, rhs, out, nx, ny, Sx, Sy[bcset], Lx, Ly[bcset],
                                     sh, nz, c2, Mx, My, face, (const int *)active));
        }
    }
    template <int CL>
    void cluster_cq(const T *rhs, T *out, int bcset, const T *sh, long long P, T *c2, const T *face) {
        const int cq = plane_cq();
        if (cq == 1) launch_cluster<CL, 1>(rhs, out, bcset, sh, P, c2, face);
        else if (cq == 2) launch_cluster<CL, 2>(rhs, out, bcset, sh, P, c2, face);
        else launch_cluster<CL, 4>(rhs, out, bcset, sh, P, c2, face);
    }
    // transform variant by its public code (PF_GEMM_*); false when this engine cannot run it
    bool gemm_available(int code) const {
        return ((code == 0 || code == 8) && !tcb.empty()) || (code == 1 && plane_fits()) || code == 32 ||
               code == 64 || (code >= 2 && code <= 5) || (code == 6 && cluster_fits(4)) ||
               (code == 7 && cluster_fits(2));
    }
    // PF_GEMM_TC_HYBRID (8): the psi and phi solves (the natural-BC set) on the cp.async 64x64 SIMT
    // transforms, the others on the tensor cores with four K slices per accumulation group
    bool tc_hybrid = false;
    void set_gemm(int code) {
        use_tc = code == 0 || code == 8;
        tc_hybrid = code == 8;
        fuse_plane = code == 1;
        cluster = code == 6 ? 4 : code == 7 ? 2 : 0;
        simt_tile = (code == 32 || code == 64 || (code >= 2 && code <= 5)) ? code : code == 8 ? 3 : 0;
    }
    template <int CQ>
    void launch_plane(const T *rhs, T *out, int bcset, const T *sh, long long P, T *c2, const T *face) {
        if constexpr (sizeof(T) == 4) {
            const unsigned threads = 32u * (unsigned)(pf::fdm_plane_nyp(ny) / 8);
            pf::k_fdm_plane<CQ><<<(unsigned)P, threads, fdm_plane_smem(), st>>>(
                rhs, out, nx, ny, Sx, Sy[bcset], Lx, Ly[bcset], sh, nz, c2, Mx, My, face, active);
        }
    }

    void fdm(const T *rhs, T *out, int bcset, const T *sh, int nplanes, T *minus_m_out = nullptr,
             const T *face = nullptr) {
        const long long P = nplanes;
        if (use_tc && !tcb.empty() && !(tc_hybrid && bcset == PF_BCSET_NN)) {
            fdm_tc(rhs, out, bcset, sh, P, minus_m_out, face);
            return;
        }
        if (cluster && cluster_fits(cluster)) {
            prof->begin(PF_KC_GEMM, st);
            if (cluster == 4) cluster_cq<4>(rhs, out, bcset, sh, P, minus_m_out, face);
            else cluster_cq<2>(rhs, out, bcset, sh, P, minus_m_out, face);
            check_launch();
            prof->end(st);
            return;
        }
        if (fuse_plane && plane_fits()) {
            prof->begin(PF_KC_GEMM, st);
            const int cq = plane_cq();
            if (cq == 1) launch_plane<1>(rhs, out, bcset, sh, P, minus_m_out, face);
            else if (cq == 2) launch_plane<2>(rhs, out, bcset, sh, P, minus_m_out, face);
            else launch_plane<4>(rhs, out, bcset, sh, P, minus_m_out, face);
            check_launch();
            prof->end(st);
            return;
        }
        gemm(rhs, Sx, W1, P * ny, nx, ny, 1, nullptr, nullptr, nullptr, 1);
        if (fuse_y && fdm_y_smem() <= 200 * 1024) {
            // y transform, eigenvalue division and inverse y transform in one pass
            constexpr int BM = 32, CG = 8;
            const int threads = ((BM * ((ny + CG - 1) / CG) + 31) / 32) * 32;
            prof->begin(PF_KC_GEMM, st);
            pf::k_fdm_y<T, BM, CG><<<(unsigned)((P * nx + BM - 1) / BM), threads, fdm_y_smem(), st>>>(
                W1, Sy[bcset], SyT[bcset], W2, P * nx, ny, nx, Ly[bcset], Lx, sh, nz, active);
            check_launch();
            prof->end(st);
            gemm(W2, SxT, out, P * ny, nx, ny, 0, nullptr, nullptr, nullptr, 1, minus_m_out, face);
            return;
        }
        gemm(W1, Sy[bcset], W2, P * nx, ny, nx, 0, Ly[bcset], Lx, sh, nz);
        gemm(W2, SyT[bcset], W1, P * nx, ny, nx, 1, nullptr, nullptr, nullptr, 1);
        gemm(W1, SxT, out, P * ny, nx, ny, 0, nullptr, nullptr, nullptr, 1, minus_m_out, face);
    }

    void fwd(const T *X0, int x0l, const T *X1, int x1l, int mult, double scale, const T *lift, T *out,
             T *out1, int ncomp = 1, const T *lift2y = nullptr, const T *lift2x = nullptr) {
        pf::FwdArgs<T> a;
        a.lift2y = lift2y; a.lift2x = lift2x;
        a.cs_x0 = x0l ? NL : N; a.cs_x1 = x1l ? NL : N; a.cs_out = N;
        a.X0 = X0; a.x0_local = x0l; a.X1 = X1; a.x1_local = x1l; a.mult = mult; a.scale = (T)scale;
        a.lift = lift; a.out = out; a.out1 = out1; a.two_pi_over_lz = (T)(2.0 * M_PI / hs.lz);
        a.tw = tw; a.tp = fwd_tp();
        const size_t smem = (size_t)((nz > 1 ? nz / 2 : 1) + a.tp * fld()) * sizeof(cplx<T>) + a.tp * 4 * sizeof(int) +
                            fft_scratch(a.tp);
        prof->begin(PF_KC_FWD, st);
        const dim3 grid((n2 + a.tp - 1) / a.tp, ncomp);
        switch (lgz()) {
            case 4: pf::k_fwd<T, 4><<<grid, 256, smem, st>>>(geo(), a); break;
            case 5: pf::k_fwd<T, 5><<<grid, 256, smem, st>>>(geo(), a); break;
            case 6: pf::k_fwd<T, 6><<<grid, 256, smem, st>>>(geo(), a); break;
            case 7: pf::k_fwd<T, 7><<<grid, 256, smem, st>>>(geo(), a); break;
            case 8: pf::k_fwd<T, 8><<<grid, 256, smem, st>>>(geo(), a); break;
            default: pf::k_fwd<T, 0><<<grid, 256, smem, st>>>(geo(), a);
        }
        check_launch();
        prof->end(st);
    }

    void inv(const T *Y, T *out, T *dzout, int drow0, double v0, int drow1, double v1, int ncomp = 1) {
        pf::InvArgs<T> a{};
        a.cs_y = N; a.cs_out = N;
        a.Y = Y; a.phi_variant = 0; a.drow0 = drow0; a.drow1 = drow1; a.v0 = (T)v0; a.v1 = (T)v1;
        a.out = out; a.dzout = d3 ? dzout : nullptr; a.two_pi_over_lz = (T)(2.0 * M_PI / hs.lz);
        a.tw = tw; a.tp = fwd_tp();
        const size_t smem = (size_t)((nz > 1 ? nz / 2 : 1) + a.tp * fld()) * sizeof(cplx<T>) + fft_scratch(a.tp);
        prof->begin(PF_KC_INV, st);
        launch_inv(dim3((n2 + a.tp - 1) / a.tp, ncomp), smem, a);
        check_launch();
        prof->end(st);
    }

    void inv_phi(double alpha, T *phi_out, T *dzphi_out) {
        pf::InvArgs<T> a{};
        a.Y = OUT; a.psi = PSIH; a.Q2h = Q2H; a.Q2n = Q2; a.alpha = (T)alpha;
        a.S_eta2 = (T)(hs.S / std::pow(hs.eta, 2.0)); a.phi_variant = 1; a.drow0 = a.drow1 = -1;
        a.out = phi_out; a.dzout = d3 ? dzphi_out : nullptr; a.out2 = W; a.dzout2 = d3 ? dzW : nullptr;
        a.out3 = Lf; a.two_pi_over_lz = (T)(2.0 * M_PI / hs.lz); a.tw = tw;
        a.tp = std::max(4, fwd_tp() / 2);    // still a power of two
        const size_t smem = (size_t)((nz > 1 ? nz / 2 : 1) + 2 * a.tp * fld()) * sizeof(cplx<T>) + fft_scratch(2 * a.tp);
        prof->begin(PF_KC_INV, st);
        launch_inv(dim3((n2 + a.tp - 1) / a.tp), smem, a);
        check_launch();
        prof->end(st);
    }

    void fwd_indep(const T *X0, const T *X1, const T *scale_p, bool lift, T *out, T *out1, int ncomp = 1) {
        pf::IndepFwd<T> a{NL, N, X0, X1, scale_p, lift ? liftb : nullptr, lift ? liftt : nullptr, pvb, pvt, out, out1};
        prof->begin(PF_KC_FWD, st);
        pf::k_fwd_indep<T><<<dim3((n2 + 255) / 256, nz, ncomp), 256, 0, st>>>(geo(), a);
        check_launch();
        prof->end(st);
    }
    void inv_indep(const T *Y, T *out, T *cur_level, bool dirichlet_v, bool phi_variant, double alpha, int ncomp = 1) {
        pf::IndepInv<T> a{};
        a.cs_y = N; a.cs_out = N;
        a.Y = Y; a.out = out; a.cur = cur_level;
        a.drow0 = dirichlet_v ? hs.vrow0 : -1; a.drow1 = dirichlet_v ? hs.vrow1 : -1;
        a.v0_p = pvb; a.v1_p = pvt;
        if (phi_variant) {
            a.psi = PSIH; a.Q2n = Q2; a.alpha = (T)alpha; a.S_eta2 = (T)(hs.S / std::pow(hs.eta, 2.0));
            a.outW = W; a.outL = Lf;
        }
        prof->begin(PF_KC_INV, st);
        pf::k_inv_indep<T><<<dim3((n2 + 255) / 256, nz, ncomp), 256, 0, st>>>(geo(), a);
        check_launch();
        prof->end(st);
    }

    // ---- the potential sub-step (also used by the initial fixed point) ----------------------
    void potential(int J, const T *phin, const T *phio, const T *Vn, const T *Vo, const T *Ezn, const T *Ezo,
                   T *Vout, T *Ezout) {
        auto G = geo();
        auto q = phys(J);
        prof->begin(PF_KC_POTENTIAL, st);
        by_order([&](auto kc) {
            pf::k_potential<T, decltype(kc)::value><<<elem_grid(), elem_threads(), elem_smem(3), st>>>(
                G, q, phin, phio, Vn, Vo, Ezn, Ezo, LA, d3 ? LB : nullptr);
        });
        check_launch();
        prof->end(st);
        if (indep) fwd_indep(LA, nullptr, pscale, true, RHS, nullptr);
        else if (hs.patch) fwd(LA, 1, d3 ? LB : nullptr, 1, 0, 1.0 / hs.eps0, liftV, RHS, nullptr, 1, Ky0, wallw);
        else fwd(LA, 1, d3 ? LB : nullptr, 1, 0, 1.0 / hs.eps0, liftV, RHS, nullptr);
        fdm(RHS, OUT, PF_BCSET_V, shV, nz);
        if (hs.patch) patch_correction();
        if (indep) inv_indep(OUT, Vout, Vout == V[0] ? V[1] : V[0], true, false, 0.0);
        else if (hs.patch) inv(OUT, Vout, Ezout, -1, 0.0, hs.vrow1, hs.v1);
        else inv(OUT, Vout, Ezout, hs.vrow0, hs.v0, hs.vrow1, hs.v1);
    }

    // Electrode patches (eq. 21): OUT holds the base solve y with the whole wall Dirichlet at the
    // values w = wallw (electrode voltages in mode 0, the previous solve's gap values).  The gap
    // change d = C^-1 (b_G - A_G,wall w - A_GI y) per plane, the correction z = A_II^-1 A_IG d
    // (second solve), then V = y - z off the wall and w + d on the wall; w keeps the new gap
    // values.  Starting from the last gap values keeps d and z small, so that y - z loses few digits.
    void patch_correction() {
        const int m = npatch_gap;
        T *rhs2 = RHS + N, *z = OUT + N;
        if (m > 0) {
            prof->begin(PF_KC_OTHER, st);
            pf::k_cap_solve<T><<<nz, 256, (size_t)2 * m * sizeof(T), st>>>(
                geo(), RHS, OUT, gapj, gapidx, m, wallw, Kxd, Ky0, (T)hs.My[0], shV, Cinv, gbuf, rhs2);
            check_launch();
            prof->end(st);
            fdm(rhs2, z, PF_BCSET_V, shV, nz);
        }
        prof->begin(PF_KC_OTHER, st);
        pf::k_cap_combine<T><<<(unsigned)((N + 255) / 256), 256, 0, st>>>(geo(), OUT, m > 0 ? z : nullptr, gbuf,
                                                                        gapidx, m, wallw, OUT, N);
        check_launch();
        prof->end(st);
    }

    void efield(const T *Vf) {
        const long long tot = N;
        prof->begin(PF_KC_EFIELD, st);
        by_order([&](auto kc) {
            constexpr int KC = decltype(kc)::value;
            const size_t rows_smem = (size_t)2 * (K + 1) * nx * sizeof(float);
            if constexpr (KC > 0 && sizeof(T) == 4) {
                if (rows_smem <= 48 * 1024) {   // element rows and columns per thread (FP32)
                    pf::DTab<KC> t;
                    for (int i = 0; i < (KC + 1) * (KC + 1); ++i) t.d[i] = (float)hs.D[i];
                    for (int i = 0; i <= KC; ++i) t.w[i] = (float)hs.w[i];
                    const unsigned thr = (unsigned)std::min(1024, (nx + 31) / 32 * 32);
                    pf::k_efield_rows<KC><<<dim3(ey, nz), thr, rows_smem, st>>>(geo(), t, Vf, Ex, Ey);
                    return;
                }
            }
            pf::k_efield<T, KC><<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(geo(), Vf, Ex, Ey);
        });
        check_launch();
        prof->end(st);
    }

    // ---- one time step -----------------------------------------------------------------------
    void step(int J) {
        const int n = cur, o = 1 - cur;
        auto G = geo();
        auto q = phys(J);
        const double al = alpha_of(hs, J);
        // V^{n+1}, E^{n+1}
        potential(J, phi[n], phi[o], V[n], V[o], Ez[n], Ez[o], V[o], Ez[o]);
        efield(V[o]);
        // psi^{n+1}
        prof->begin(PF_KC_CHEM, st);
        by_order([&](auto kc) {
            pf::k_chem<T, decltype(kc)::value><<<elem_grid(), elem_threads(), elem_smem(4), st>>>(
                G, q, phi[n], phi[o], dzphi[n], dzphi[o], u[0][n], u[0][o], u[1][n], u[1][o], u[2][n], u[2][o], Ex,
                Ey, Ez[o], LA, Q2, q.wetting ? faceU : nullptr);
        });
        check_launch();
        prof->end(st);
        if (indep) fwd_indep(LA, Q2, nullptr, false, RHS, Q2H);
        else fwd(LA, 1, Q2, 0, 1, 1.0, nullptr, RHS, Q2H);
        // wall term of the phi equation (only with a contact angle other than 90 degrees)
        const T *faceh = nullptr;
        if (q.wetting && indep) {
            prof->begin(PF_KC_OTHER, st);
            pf::k_face_indep<T><<<dim3((nx + 127) / 128, nz), 128, 0, st>>>(G, faceU, FACEH);
            check_launch();
            prof->end(st);
            faceh = FACEH;
        } else if (q.wetting) {
            const int tp = fwd_tp();
            const size_t smem = (size_t)((nz > 1 ? nz / 2 : 1) + tp * (nz + 1)) * sizeof(cplx<T>) + fft_scratch(tp);
            prof->begin(PF_KC_OTHER, st);
            pf::k_face_fft<T><<<(nx + tp - 1) / tp, 256, smem, st>>>(G, faceU, FACEH, tw, tp);
            check_launch();
            prof->end(st);
            faceh = FACEH;
        }
        // psi^{n+1}; its last transform also writes the phi right-hand side -M psi (+ wall term)
        T *rhs_phi = RHS + N;
        fdm(RHS, PSIH, PF_BCSET_NN, shPsi[J - 1], nz, rhs_phi, faceh);
        // phi^{n+1}
        fdm(rhs_phi, OUT, PF_BCSET_NN, shPhi[J - 1], nz);
        if (indep) inv_indep(OUT, phi[o], phi[n], false, true, al);
        else inv_phi(al, phi[o], dzphi[o]);
        if (hs.model == PF_MODEL_EQUILIBRIUM) {   // Sec. 2.4: u = 0, no pressure or velocity step
            if (indep) batch_check(n, o);
            cur = o;
            return;
        }
        // P^{n+1}
        pf::MomIn<T> mi;
        mi.phi = phi[o]; mi.dzphi = dzphi[o]; mi.W = W; mi.dzW = dzW; mi.L = Lf;
        mi.Ex = Ex; mi.Ey = Ey; mi.Ez = Ez[o];
        for (int c = 0; c < 3; ++c) {
            mi.un[c] = u[c][n]; mi.uo[c] = u[c][o]; mi.dzun[c] = dzu[c][n]; mi.dzuo[c] = dzu[c][o];
        }
        mi.Pn = P[n]; mi.Po = P[o]; mi.dzPn = dzP[n]; mi.dzPo = dzP[o];
        pf::MomOut<T> mo;
        mo.AP = LA; mo.BP = d3 ? LB : nullptr;
        for (int c = 0; c < 3; ++c) { mo.AU[c] = LAU[c]; mo.BU[c] = LBU[c]; }
        prof->begin(PF_KC_MOMENTUM, st);
        by_order([&](auto kc) {
            pf::k_momentum<T, decltype(kc)::value><<<elem_grid(), elem_threads(), elem_smem(12), st>>>(G, q, mi, mo);
        });
        check_launch();
        prof->end(st);
        if (indep) fwd_indep(LA, nullptr, nullptr, false, RHS, nullptr);
        else fwd(LA, 1, d3 ? LB : nullptr, 1, 0, 1.0, nullptr, RHS, nullptr);
        fdm(RHS, OUT, PF_BCSET_P, shP, nz);
        if (indep) inv_indep(OUT, P[o], P[n], false, false, 0.0);
        else inv(OUT, P[o], dzP[o], -1, 0.0, -1, 0.0);
        // u^{n+1}
        prof->begin(PF_KC_UGRADP, st);
        by_order([&](auto kc) {
            pf::k_ugradp<T, decltype(kc)::value><<<elem_grid(), elem_threads(), elem_smem(1), st>>>(
                G, q, P[o], LAU[0], LAU[1], d3 ? LBU[2] : nullptr);
        });
        check_launch();
        prof->end(st);
        const int dc = d3 ? 3 : 2;
        // all velocity components in one launch per transform
        if (indep) fwd_indep(LAU[0], nullptr, nullptr, false, RHS, nullptr, dc);
        else fwd(LAU[0], 1, d3 ? LBU[0] : nullptr, 1, 0, 1.0, nullptr, RHS, nullptr, dc);
        fdm(RHS, OUT, PF_BCSET_U, shU[J - 1], dc * nz);
        if (indep) inv_indep(OUT, u[0][o], u[0][n], false, false, 0.0, dc);
        else inv(OUT, u[0][o], dzu[0][o], -1, 0.0, -1, 0.0, dc);
        if (indep) batch_check(n, o);
        cur = o;
    }

    // per-plane FP64 reduction (kind 0: sum of M x, kind 1: max |x|) of level-n field x into host out[nz]
    void reduce_planes(const T *x, int kind, double *out, const T *y = nullptr) {
        pf::k_reduce_planes<T><<<nz, 256, 0, st>>>(x, y, Mx, My, nx, n2, kind, red);
        check_launch();
        PF_CU(cudaMemcpyAsync(out, red, nz * sizeof(double), cudaMemcpyDeviceToHost, st));
        PF_CU(cudaStreamSynchronize(st));
    }

    // discrete energy E(t) of eq. 14 at level n (FP64; synchronous)
    double *epart = nullptr;
    double energy() {
        const dim3 grid = elem_grid();
        const size_t nb = (size_t)grid.x * grid.y;
        if (!epart) epart = mk<double>(nb);
        pf::EnergyConst c{hs.rho1, hs.rho2, hs.eps1, hs.eps2, hs.lam, 1.0 / (hs.eta * hs.eta),
                          hs.sigma * hs.cos_theta};
        const int n = cur;
        pf::k_energy<T><<<grid, elem_threads(), elem_smem(1), st>>>(geo(), c, phi[n], d3 ? dzphi[n] : nullptr, u[0][n],
                                                                   u[1][n], d3 ? u[2][n] : nullptr, Ex, Ey,
                                                                   d3 ? Ez[n] : nullptr, epart);
        check_launch();
        std::vector<double> h(nb);
        PF_CU(cudaMemcpyAsync(h.data(), epart, nb * sizeof(double), cudaMemcpyDeviceToHost, st));
        PF_CU(cudaStreamSynchronize(st));
        double acc = 0.0;
        for (double v : h) acc += v;
        return acc * (d3 ? hs.lz / nz : 1.0);
    }

    // error word of the bounded device waits: read (synchronous) and clear
    int take_err() {
        int e = 0;
        PF_CU(cudaMemcpyAsync(&e, dev_err, sizeof(int), cudaMemcpyDeviceToHost, st));
        PF_CU(cudaStreamSynchronize(st));
        if (e) PF_CU(cudaMemsetAsync(dev_err, 0, sizeof(int), st));
        return e;
    }

    // ---- reductions (FP64 accumulation) -------------------------------------------------------
    double reduce(const T *x, const T *y, int kind) {
        const int blocks = 512;
        pf::k_reduce<T><<<blocks, 256, 0, st>>>(x, y, Mx, My, nx, n2, N, kind, red);
        check_launch();
        std::vector<double> h(blocks);
        PF_CU(cudaMemcpyAsync(h.data(), red, blocks * sizeof(double), cudaMemcpyDeviceToHost, st));
        PF_CU(cudaStreamSynchronize(st));
        double acc = 0.0;
        for (int i = 0; i < blocks; ++i) {
            const double v = h[i];
            if (kind == 0) acc += v;
            else if (v != v) return v;
            else acc = std::max(acc, v);
        }
        return acc;
    }
};

}  // namespace

// message of the last failed call that has no handle (read with pf_last_error(NULL))
void pf_internal_set_error(const std::string &msg) { g_create_error = msg; }

struct pf_handle {
    HostSetup hs;
    Prof prof;
    cudaStream_t st = nullptr;
    std::unique_ptr<Engine<double>> e64;
    std::unique_ptr<Engine<float>> e32;
    long long nstep = 0;
    double t = 0.0;
    int v_iters = 0;
    int last_J = 1;
    bool diverged = false;
    std::string err;
};

namespace {

int fail(pf_handle *h, int code, const std::string &msg) {
    if (h) h->err = msg;
    else g_create_error = msg;
    return code;
}

int cuda_fail(pf_handle *h, const CudaError &e) {
    return fail(h, PF_ECUDA, e.where + ": " + cudaGetErrorString(e.code));
}

void build_patches(HostSetup &s);

void build_setup(HostSetup &s) {
    s.p = s.K + 1;
    s.nx = s.ex * s.K;
    s.ny = s.ey * s.K + 1;
    const int p = s.p;
    s.xi.resize(p); s.w.resize(p); s.D.resize(p * p); s.Dw.resize(p * p);
    pf_gll(s.K, s.xi.data(), s.w.data(), s.D.data());
    for (int a = 0; a < p; ++a)
        for (int c = 0; c < p; ++c) s.Dw[a * p + c] = s.w[a] * s.D[a * p + c];
    s.hx.resize(s.ex); s.hy.resize(s.ey);
    for (int e = 0; e < s.ex; ++e) s.hx[e] = s.xb[e + 1] - s.xb[e];
    for (int e = 0; e < s.ey; ++e) s.hy[e] = s.yb[e + 1] - s.yb[e];
    s.Kx.resize((size_t)s.nx * s.nx); s.Mx.resize(s.nx);
    s.Ky.resize((size_t)s.ny * s.ny); s.My.resize(s.ny);
    pf_operators_1d(s.ex, s.xb.data(), s.K, 1, s.Kx.data(), s.Mx.data());
    pf_operators_1d(s.ey, s.yb.data(), s.K, 0, s.Ky.data(), s.My.data());
    s.Sx.resize((size_t)s.nx * s.nx); s.Lx.resize(s.nx);
    pf_fdm_1d(s.nx, s.Kx.data(), s.Mx.data(), nullptr, s.Sx.data(), s.Lx.data());
    // the zero eigenvalue of the periodic operator is exact
    for (auto &v : s.Lx) if (std::fabs(v) < 1e-11) v = 0.0;
    const int ny = s.ny;
    auto mask = [&](bool bot, bool top) {
        std::vector<unsigned char> m(ny, 0);
        if (bot) m[0] = 1;
        if (top) m[ny - 1] = 1;
        return m;
    };
    std::vector<unsigned char> masks[4] = {
        mask(s.vrow0 >= 0, s.vrow1 >= 0),   // V
        mask(false, false),                 // psi, phi
        mask(false, true),                  // P: Dirichlet on the open side
        mask(true, false)};                 // u: Dirichlet on the wall
    for (int b = 0; b < 4; ++b) {
        s.Sy[b].resize((size_t)ny * ny);
        s.Ly[b].resize(ny);
        pf_fdm_1d(ny, s.Ky.data(), s.My.data(), masks[b].data(), s.Sy[b].data(), s.Ly[b].data());
        for (auto &v : s.Ly[b]) if (std::fabs(v) < 1e-11) v = 0.0;
    }
    // lifting of the potential's Dirichlet values: K_y[i][d] * V_d (times M_x in the kernel)
    s.liftV.assign(ny, 0.0);
    for (int i = 0; i < ny; ++i) {
        if (s.vrow0 >= 0) s.liftV[i] += s.Ky[(size_t)i * ny + 0] * s.v0;
        if (s.vrow1 >= 0) s.liftV[i] += s.Ky[(size_t)i * ny + (ny - 1)] * s.v1;
    }
    s.X.resize(s.nx);
    for (int e = 0; e < s.ex; ++e)
        for (int a = 0; a < s.K; ++a) s.X[e * s.K + a] = s.xb[e] + 0.5 * (s.xi[a] + 1.0) * s.hx[e];
    s.Y.resize(ny);
    for (int e = 0; e < s.ey; ++e)
        for (int b = 0; b <= s.K; ++b) s.Y[e * s.K + b] = s.yb[e] + 0.5 * (s.xi[b] + 1.0) * s.hy[e];
    if (s.patch) build_patches(s);
}

// Electrode patches (eq. 21): classify the wall nodes, and for every mode plane build the
// capacitance matrix of the gap rows and invert it (FP64).  With A the plane operator
// K_x (x) M_y + M_x (x) K_y + c M_x (x) M_y and the base solve A_II^-1 on everything but the wall
// row, the gap values g solve C g = b_G - A_GE V_E - A_GI A_II^-1 (b_I - A_IE V_E) with
// C = A_GG - A_GI A_II^-1 A_IG.  A_IG couples a gap node (0, j) only with (i, j), i >= 1, through
// M_x[j] K_y[i][0], so in the base eigenbases (S_x, L_x; S_y, L_y of the Dirichlet-wall set)
//   (A_GI A_II^-1 A_IG)[j][l] = M_x[j] M_x[l] sum_a S_x[j][a] S_x[l][a] sum_b w_b^2 / (L_x[a] + L_y[b] + c),
// w_b = sum_i K_y[0][i] S_y[i][b]; A_GG[j][l] = M_y[0] K_x[j][l] + [j = l] M_x[j] (K_y[0][0] + c M_y[0]).
int electrode_at(const HostSetup &s, double x) {
    const double period = s.xb[s.ex] - s.xb[0];
    for (size_t e = 0; e < s.px0.size(); ++e) {
        const double tol = 1e-9 * std::fabs(s.px1[e] - s.px0[e]) + 1e-12;
        if ((x >= s.px0[e] - tol && x <= s.px1[e] + tol) || (x + period >= s.px0[e] - tol && x + period <= s.px1[e] + tol))
            return (int)e;
    }
    return -1;
}

// in-place inverse of a dense n x n matrix (Gauss-Jordan, partial pivoting); false if singular
bool invert_dense(std::vector<double> &A, int n) {
    std::vector<double> I((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) I[(size_t)i * n + i] = 1.0;
    for (int c = 0; c < n; ++c) {
        int piv = c;
        for (int r = c + 1; r < n; ++r)
            if (std::fabs(A[(size_t)r * n + c]) > std::fabs(A[(size_t)piv * n + c])) piv = r;
        if (A[(size_t)piv * n + c] == 0.0) return false;
        if (piv != c)
            for (int k = 0; k < n; ++k) {
                std::swap(A[(size_t)c * n + k], A[(size_t)piv * n + k]);
                std::swap(I[(size_t)c * n + k], I[(size_t)piv * n + k]);
            }
        const double d = 1.0 / A[(size_t)c * n + c];
        for (int k = 0; k < n; ++k) { A[(size_t)c * n + k] *= d; I[(size_t)c * n + k] *= d; }
        for (int r = 0; r < n; ++r) {
            if (r == c) continue;
            const double f = A[(size_t)r * n + c];
            if (f == 0.0) continue;
            for (int k = 0; k < n; ++k) {
                A[(size_t)r * n + k] -= f * A[(size_t)c * n + k];
                I[(size_t)r * n + k] -= f * I[(size_t)c * n + k];
            }
        }
    }
    A.swap(I);
    return true;
}

void build_patches(HostSetup &s) {
    const int nx = s.nx, ny = s.ny, nz = s.nz;
    s.vbx.assign(nx, 0.0);
    s.gapidx.assign(nx, -1);
    s.gapj.clear();
    for (int j = 0; j < nx; ++j) {
        const int e = electrode_at(s, s.X[j]);
        if (e >= 0) s.vbx[j] = s.pv[e];
        else { s.gapidx[j] = (int)s.gapj.size(); s.gapj.push_back(j); }
    }
    const int m = (int)s.gapj.size();
    s.Ky0.assign(s.Ky.begin(), s.Ky.begin() + ny);   // row 0 (= column 0, K_y is symmetric)
    const std::vector<double> &Sy = s.Sy[PF_BCSET_V], &Ly = s.Ly[PF_BCSET_V];
    std::vector<double> w2(ny, 0.0);
    for (int b = 0; b < ny; ++b) {
        double acc = 0.0;
        for (int i = 0; i < ny; ++i) acc += s.Ky0[i] * Sy[(size_t)i * ny + b];
        w2[b] = acc * acc;
    }
    s.Cinv.assign((size_t)nz * m * m, 0.0);
    std::vector<double> gam(nx), C((size_t)m * m);
    int done_k = -1;
    std::vector<double> last;
    for (int p = 0; p < nz; ++p) {
        int k = 0;
        if (nz > 1) k = (p == 0) ? 0 : (p == 1 ? nz / 2 : p / 2);
        if (k == done_k) {   // planes 2k and 2k+1 share the mode
            std::copy(last.begin(), last.end(), s.Cinv.begin() + (size_t)p * m * m);
            continue;
        }
        const double beta = nz > 1 ? 2.0 * M_PI * k / s.lz : 0.0;
        const double c = beta * beta;
        for (int a = 0; a < nx; ++a) {
            double acc = 0.0;
            for (int b = 0; b < ny; ++b) acc += w2[b] / (s.Lx[a] + Ly[b] + c);
            gam[a] = acc;
        }
        for (int jj = 0; jj < m; ++jj)
            for (int ll = 0; ll < m; ++ll) {
                const int j = s.gapj[jj], l = s.gapj[ll];
                double acc = 0.0;
                for (int a = 0; a < nx; ++a) acc += s.Sx[(size_t)j * nx + a] * s.Sx[(size_t)l * nx + a] * gam[a];
                double v = s.My[0] * s.Kx[(size_t)j * nx + l] - s.Mx[j] * s.Mx[l] * acc;
                if (jj == ll) v += s.Mx[j] * (s.Ky[0] + c * s.My[0]);
                C[(size_t)jj * m + ll] = v;
            }
        if (m > 0 && !invert_dense(C, m)) C.assign((size_t)m * m, NAN);
        std::copy(C.begin(), C.end(), s.Cinv.begin() + (size_t)p * m * m);
        last = C;
        done_k = k;
    }
}

// initial potential: fixed point of the Remark in Sec. 3.1 in FP64, run to the round-off
// floor: stop when the max-norm update is <= 1e-15 vmax, or once it is below 1e-11 vmax and
// no longer decreases, or after 20000 iterations (vmax = max(1, |electrode voltages|)).
int initial_potential(const HostSetup &hs, Engine<double> &E, const double *phi0_dev, int &v_iters,
                      std::string &err) {
    const double tol = 1e-15;
    double prev = INFINITY;
    double vmax = 1.0;
    if (hs.vrow0 >= 0) vmax = std::max(vmax, std::fabs(hs.v0));
    if (hs.vrow1 >= 0) vmax = std::max(vmax, std::fabs(hs.v1));
    for (double v : hs.bvb) vmax = std::max(vmax, std::fabs(v));
    for (double v : hs.bvt) vmax = std::max(vmax, std::fabs(v));
    int a = 0;   // slot of the current iterate
    PF_CU(cudaMemsetAsync(E.V[0], 0, E.N * sizeof(double), E.st));
    if (E.d3) PF_CU(cudaMemsetAsync(E.Ez[0], 0, E.N * sizeof(double), E.st));
    int it = 0;
    for (it = 1; it <= 20000; ++it) {
        E.potential(1, phi0_dev, phi0_dev, E.V[a], E.V[a], E.Ez[a], E.Ez[a], E.V[1 - a], E.Ez[1 - a]);
        const double diff = E.reduce(E.V[1 - a], E.V[a], 2);
        a = 1 - a;
        if (!(diff == diff)) {
            err = "non-finite value in the initial potential";
            return PF_EDIVERGED;
        }
        if (diff <= tol * vmax || (diff <= 1e-11 * vmax && diff >= prev)) break;
        prev = diff;
    }
    v_iters = std::min(it, 20000);
    if (a != 0) {
        PF_CU(cudaMemcpyAsync(E.V[0], E.V[1], E.N * sizeof(double), cudaMemcpyDeviceToDevice, E.st));
        if (E.d3) PF_CU(cudaMemcpyAsync(E.Ez[0], E.Ez[1], E.N * sizeof(double), cudaMemcpyDeviceToDevice, E.st));
    }
    return PF_OK;
}

template <typename T>
void copy_level(Engine<T> &E, int from, int to) {
    auto cp = [&](T *const *arr) {
        if (arr[from] && arr[to]) PF_CU(cudaMemcpyAsync(arr[to], arr[from], E.N * sizeof(T), cudaMemcpyDeviceToDevice, E.st));
    };
    cp(E.V); cp(E.Ez); cp(E.phi); cp(E.dzphi); cp(E.P); cp(E.dzP);
    for (int c = 0; c < 3; ++c) { cp(E.u[c]); cp(E.dzu[c]); }
}

// Host <-> device field copies: the caller's double buffer is copied as is (DMA directly
// from/to it when it is pinned) into device scratch and converted there.
template <typename T>
void upload_field(Engine<T> &E, T *dst, const double *host) {
    double *scratch = reinterpret_cast<double *>(E.W2);   // 3N values of T >= N doubles
    PF_CU(cudaMemcpyAsync(scratch, host, E.N * sizeof(double), cudaMemcpyHostToDevice, E.st));
    E.prof->begin(PF_KC_OTHER, E.st);
    pf::k_convert<double, T><<<1024, 256, 0, E.st>>>(scratch, dst, E.N);
    PF_CU(cudaGetLastError());
    E.prof->end(E.st);
}

// Asynchronous on the engine's stream: the next conversion into the scratch follows the copy in
// stream order; the caller synchronises before it reads the host buffer.
template <typename T>
void download_field(Engine<T> &E, const T *src, double *host) {
    double *scratch = reinterpret_cast<double *>(E.W2);
    E.prof->begin(PF_KC_OTHER, E.st);
    pf::k_convert<T, double><<<1024, 256, 0, E.st>>>(src, scratch, E.N);
    PF_CU(cudaGetLastError());
    E.prof->end(E.st);
    PF_CU(cudaMemcpyAsync(host, scratch, E.N * sizeof(double), cudaMemcpyDeviceToHost, E.st));
}

// z-derivative of a physical field through the engine's own transforms (forward then
// inverse with d/dz), used when a field is set from the host
template <typename T>
void dz_of(Engine<T> &E, const T *x, T *dzx) {
    if (!E.d3) return;
    E.fwd(x, 0, nullptr, 0, 0, 1.0, nullptr, E.RHS, nullptr);
    E.inv(E.RHS, E.W1, dzx, -1, 0.0, -1, 0.0);
}

template <typename T>
int engine_init_state(Engine<T> &E, const double *phi0, const double *u0) {
    upload_field(E, E.phi[0], phi0);
    dz_of(E, E.phi[0], E.dzphi[0]);
    if (u0) {
        for (int c = 0; c < (E.d3 ? 3 : 2); ++c) {
            upload_field(E, E.u[c][0], u0 + c * E.N);
            dz_of(E, E.u[c][0], E.dzu[c][0]);
        }
    }
    return PF_OK;
}

template <typename T>
int do_steps(pf_handle *h, Engine<T> &E, int nsteps) {
    for (int s = 0; s < nsteps; ++s) {
        const int J = (h->nstep == 0 || h->hs.bdf == 1) ? 1 : 2;
        // graphs need a capturable stream (not the legacy default stream) and no event timers
        if (J == 2 && E.st != nullptr && !h->prof.on && !E.tc_stall) E.step_graph();
        else E.step(J);
        h->last_J = J;
        h->nstep += 1;
        h->t += h->hs.dt;
    }
    return PF_OK;
}

}  // namespace

// ============================================================================================
namespace {

// Validate the descriptors and fill the host constants (Sec. 2.1, Sec. 3.1); no device work.
int fill_setup(const pf_mesh *mesh, const pf_fluid *fluid, const pf_vbc *vbc, const pf_scheme *scheme,
               HostSetup &s, std::string &err) {
    auto bad = [&](const char *m) { err = m; return PF_EINVAL; };
    if (!mesh || !fluid || !vbc || !scheme) return bad("null argument");
    if (mesh->ex < 1 || mesh->ey < 1 || !mesh->xb || !mesh->yb) return bad("bad element counts");
    if (mesh->order < 2 || mesh->order > 15) return bad("order must be in [2, 15]");
    if (mesh->nz < 1 || mesh->nz > 1024) return bad("nz must be 1 or an even product of 2, 3, 5, 7 <= 1024");
    if (mesh->nz > 1) {
        int r = mesh->nz;
        for (int f : {2, 3, 5, 7})
            while (r % f == 0) r /= f;
        if (r != 1 || mesh->nz % 2 != 0) return bad("nz must be 1 or an even product of 2, 3, 5, 7 <= 1024");
    }
    if (mesh->nz > 1 && !(mesh->lz > 0)) return bad("lz must be positive");
    if (mesh->ex * mesh->order < 2) return bad("need at least 2 nodes in x");
    for (int e = 0; e < mesh->ex; ++e)
        if (!(mesh->xb[e + 1] > mesh->xb[e])) return bad("xb must increase");
    for (int e = 0; e < mesh->ey; ++e)
        if (!(mesh->yb[e + 1] > mesh->yb[e])) return bad("yb must increase");
    if (vbc->bottom_kind != PF_BC_DIRICHLET && vbc->bottom_kind != PF_BC_NEUMANN &&
        vbc->bottom_kind != PF_BC_PATCHES)
        return bad("bad bottom_kind");
    if (vbc->top_kind != PF_BC_DIRICHLET && vbc->top_kind != PF_BC_NEUMANN) return bad("bad top_kind");
    if (vbc->bottom_kind == PF_BC_PATCHES) {
        if (vbc->n_patch < 0 || (vbc->n_patch > 0 && (!vbc->patch_x0 || !vbc->patch_x1 || !vbc->patch_v)))
            return bad("bad electrode patch arrays");
        for (int e = 0; e < vbc->n_patch; ++e)
            if (!std::isfinite(vbc->patch_x0[e]) || !std::isfinite(vbc->patch_x1[e]) ||
                !std::isfinite(vbc->patch_v[e]) || vbc->patch_x0[e] > vbc->patch_x1[e])
                return bad("electrode patches need finite x0 <= x1 and a finite voltage");
        s.patch = true;
        s.px0.assign(vbc->patch_x0, vbc->patch_x0 + vbc->n_patch);
        s.px1.assign(vbc->patch_x1, vbc->patch_x1 + vbc->n_patch);
        s.pv.assign(vbc->patch_v, vbc->patch_v + vbc->n_patch);
    }
    if (vbc->bottom_kind == PF_BC_NEUMANN && vbc->top_kind == PF_BC_NEUMANN)
        return bad("the potential needs an electrode (Dirichlet) on at least one side");
    const pf_fluid &f = *fluid;
    if (!(f.rho1 > 0 && f.rho2 > 0 && f.mu1 > 0 && f.mu2 > 0 && f.eps1 > 0 && f.eps2 > 0 && f.sigma >= 0 &&
          f.eta > 0 && f.gamma1 > 0))
        return bad("fluid parameters must be positive");
    if (!(scheme->dt > 0) || (scheme->bdf != 1 && scheme->bdf != 2)) return bad("bad dt or bdf");
    if (scheme->precision != PF_FP64 && scheme->precision != PF_MIXED && scheme->precision != PF_MIXED_SIMT)
        return bad("bad precision");
    if (scheme->model != PF_MODEL_FULL && scheme->model != PF_MODEL_EQUILIBRIUM) return bad("bad model");
    s.ex = mesh->ex; s.ey = mesh->ey; s.K = mesh->order; s.nz = mesh->nz; s.lz = mesh->nz > 1 ? mesh->lz : 1.0;
    s.xb.assign(mesh->xb, mesh->xb + s.ex + 1);
    s.yb.assign(mesh->yb, mesh->yb + s.ey + 1);
    s.rho1 = f.rho1; s.rho2 = f.rho2; s.mu1 = f.mu1; s.mu2 = f.mu2; s.eps1 = f.eps1; s.eps2 = f.eps2;
    s.sigma = f.sigma; s.eta = f.eta; s.gamma1 = f.gamma1; s.theta = f.theta_s_deg;
    s.dt = scheme->dt; s.bdf = scheme->bdf; s.precision = scheme->precision; s.model = scheme->model;
    // Sec. 2.1 and Sec. 3.1 constants (same formulas and order of operations as documented in pf.h)
    s.lam = 3.0 * s.sigma * s.eta / (2.0 * std::sqrt(2.0));
    s.eps0 = scheme->eps0 != 0.0 ? scheme->eps0 : std::max(s.eps1, s.eps2);
    s.rho0 = scheme->rho0 != 0.0 ? scheme->rho0 : std::min(s.rho1, s.rho2);
    s.nu_m = scheme->nu_m != 0.0 ? scheme->nu_m : std::max(s.mu1, s.mu2) / std::min(s.rho1, s.rho2);
    if (scheme->S != 0.0) s.S = scheme->S;
    else {
        const double g0 = s.bdf == 2 ? 1.5 : 1.0;
        s.S = std::pow(s.eta, 2.0) * std::sqrt(4.0 * g0 / (s.lam * s.gamma1 * s.dt));
    }
    s.cos_theta = std::cos(s.theta * M_PI / 180.0);
    if (vbc->bottom_kind == PF_BC_DIRICHLET) { s.vrow0 = 0; s.v0 = vbc->v_bottom; }
    if (vbc->bottom_kind == PF_BC_PATCHES) { s.vrow0 = 0; s.v0 = 0.0; }   // base solve: the whole wall Dirichlet
    if (vbc->top_kind == PF_BC_DIRICHLET) { s.vrow1 = s.ey * s.K; s.v1 = vbc->v_top; }
    return PF_OK;
}

// Device state for a filled set-up: initial state, V^0 (FP64), E^0, both history levels,
// then the working-precision engine.  Returns a PF_* code (CUDA errors are thrown).
int build_engines(const HostSetup &s, const double *phi0, const double *u0, cudaStream_t st, Prof *prof,
                  std::unique_ptr<Engine<double>> &e64out, std::unique_ptr<Engine<float>> &e32out, int &v_iters,
                  std::string &err) {
    std::unique_ptr<Engine<double>> e64(new Engine<double>(s, st, prof));
    engine_init_state(*e64, phi0, u0);
    const int rc = initial_potential(s, *e64, e64->phi[0], v_iters, err);
    if (rc != PF_OK) return rc;
    e64->efield(e64->V[0]);
    copy_level(*e64, 0, 1);
    e64->cur = 0;
    if (s.precision == PF_FP64) {
        e64out = std::move(e64);
        return PF_OK;
    }
    std::unique_ptr<Engine<float>> e32(new Engine<float>(s, st, prof));
    auto cv = [&](const double *src, float *dst) {
        if (!src || !dst) return;
        pf::k_convert<double, float><<<1024, 256, 0, st>>>(src, dst, e64->N);
    };
    for (int l = 0; l < 2; ++l) {
        cv(e64->V[l], e32->V[l]); cv(e64->Ez[l], e32->Ez[l]); cv(e64->phi[l], e32->phi[l]);
        cv(e64->dzphi[l], e32->dzphi[l]); cv(e64->P[l], e32->P[l]); cv(e64->dzP[l], e32->dzP[l]);
        for (int c = 0; c < 3; ++c) { cv(e64->u[c][l], e32->u[c][l]); cv(e64->dzu[c][l], e32->dzu[c][l]); }
    }
    cv(e64->Ex, e32->Ex); cv(e64->Ey, e32->Ey);
    if (e64->wallw && e32->wallw)
        pf::k_convert<double, float><<<64, 256, 0, st>>>(e64->wallw, e32->wallw, (long long)e64->nz * e64->nx);
    PF_CU(cudaGetLastError());
    PF_CU(cudaStreamSynchronize(st));
    e64.reset();
    e32out = std::move(e32);
    return PF_OK;
}

}  // namespace

extern "C" int pf_create(const pf_mesh *mesh, const pf_fluid *fluid, const pf_vbc *vbc, const pf_scheme *scheme,
                         const double *phi0, const double *u0, void *cuda_stream, pf_handle **out) {
    if (out) *out = nullptr;
    if (!phi0 || !out) return fail(nullptr, PF_EINVAL, "null argument");
    std::unique_ptr<pf_handle> h(new pf_handle());
    std::string err;
    int rc = fill_setup(mesh, fluid, vbc, scheme, h->hs, err);
    if (rc != PF_OK) return fail(nullptr, rc, err);
    build_setup(h->hs);
    if (h->hs.patch && (int)h->hs.gapj.size() == h->hs.nx && h->hs.vrow1 < 0)
        return fail(nullptr, PF_EINVAL, "no wall node lies on an electrode and the top is not Dirichlet: "
                                        "the potential is undetermined");
    h->st = (cudaStream_t)cuda_stream;
    try {
        rc = build_engines(h->hs, phi0, u0, h->st, &h->prof, h->e64, h->e32, h->v_iters, err);
        if (rc != PF_OK) return fail(nullptr, rc, err);
    } catch (const CudaError &e) {
        g_create_error = e.where + ": " + cudaGetErrorString(e.code);
        return e.code == cudaErrorMemoryAllocation ? PF_ENOMEM : PF_ECUDA;
    }
    *out = h.release();
    return PF_OK;
}

extern "C" int pf_step(pf_handle *h, int nsteps) {
    if (!h) return PF_EINVAL;
    if (nsteps < 0) return fail(h, PF_EINVAL, "nsteps must be >= 0");
    try {
        if (h->e64) return do_steps(h, *h->e64, nsteps);
        return do_steps(h, *h->e32, nsteps);
    } catch (const CudaError &e) {
        return cuda_fail(h, e);
    }
}

namespace {
template <typename T>
int sync_impl(pf_handle *h, Engine<T> &E) {
    PF_CU(cudaStreamSynchronize(E.st));
    const int n = E.cur;
    double m = E.reduce(E.phi[n], nullptr, 1);
    double um = 0.0;
    for (int c = 0; c < 3; ++c)
        if (E.u[c][n]) um = std::max(um, E.reduce(E.u[c][n], nullptr, 1));
    if (E.take_err())
        return fail(h, PF_ETIMEOUT, "a tensor-core transform gave up waiting (bounded mbarrier wait); the state "
                                    "of the steps since the last pf_sync is not valid");
    if (!(m == m) || !(um == um) || std::isinf(m) || std::isinf(um)) h->diverged = true;
    return h->diverged ? fail(h, PF_EDIVERGED, "non-finite value in the state") : PF_OK;
}
}  // namespace

extern "C" int pf_sync(pf_handle *h) {
    if (!h) return PF_EINVAL;
    try {
        if (h->e64) return sync_impl(h, *h->e64);
        return sync_impl(h, *h->e32);
    } catch (const CudaError &e) {
        return cuda_fail(h, e);
    }
}

namespace {
template <typename T>
int get_impl(pf_handle *h, Engine<T> &E, unsigned mask, double *out, size_t n) {
    const bool old = mask & PF_FIELD_OLD;
    const int l = old ? 1 - E.cur : E.cur;
    size_t need = 0;
    if (mask & PF_FIELD_V) need += 1;
    if (mask & PF_FIELD_E) need += 3;
    if (mask & PF_FIELD_PHI) need += 1;
    if (mask & PF_FIELD_PSI) need += 1;
    if (mask & PF_FIELD_P) need += 1;
    if (mask & PF_FIELD_U) need += 3;
    if (need * (size_t)E.N > n) return fail(h, PF_EINVAL, "output buffer too small");
    PF_CU(cudaStreamSynchronize(E.st));
    double *o = out;
    auto put = [&](const T *src) {
        if (src) download_field(E, src, o);
        else std::fill(o, o + E.N, 0.0);
        o += E.N;
    };
    if (mask & PF_FIELD_V) put(E.V[l]);
    if (mask & PF_FIELD_E) { put(E.Ex); put(E.Ey); put(E.d3 ? E.Ez[E.cur] : nullptr); }
    if (mask & PF_FIELD_PHI) put(E.phi[l]);
    if (mask & PF_FIELD_PSI) {
        // psi = L + alpha phi, L = psi - alpha phi of the last step
        std::vector<double> phi(E.N);
        download_field(E, E.phi[E.cur], phi.data());
        download_field(E, E.Lf, o);
        PF_CU(cudaStreamSynchronize(E.st));
        const double al = alpha_of(h->hs, h->last_J);
        for (long long i = 0; i < E.N; ++i) o[i] += al * phi[i];
        o += E.N;
    }
    if (mask & PF_FIELD_P) put(E.P[l]);
    if (mask & PF_FIELD_U) { put(E.u[0][l]); put(E.u[1][l]); put(E.u[2][l]); }
    PF_CU(cudaStreamSynchronize(E.st));
    return PF_OK;
}

template <typename T>
int set_impl(pf_handle *h, Engine<T> &E, unsigned mask, const double *in, size_t n, int reset) {
    const bool old = mask & PF_FIELD_OLD;
    const int l = old ? 1 - E.cur : E.cur;
    size_t need = 0;
    if (mask & PF_FIELD_V) need += 1;
    if (mask & PF_FIELD_E) return fail(h, PF_EINVAL, "E is derived from V and cannot be set");
    if (mask & PF_FIELD_PSI) return fail(h, PF_EINVAL, "psi cannot be set");
    if (mask & PF_FIELD_PHI) need += 1;
    if (mask & PF_FIELD_P) need += 1;
    if (mask & PF_FIELD_U) need += 3;
    if (need * (size_t)E.N > n) return fail(h, PF_EINVAL, "input buffer too small");
    const double *p = in;
    auto take = [&](T *dst, T *dzdst) {
        if (dst) {
            upload_field(E, dst, p);
            if (dzdst) dz_of(E, dst, dzdst);
        }
        p += E.N;
    };
    if (mask & PF_FIELD_V) take(E.V[l], E.d3 ? E.Ez[l] : nullptr);
    if (mask & PF_FIELD_PHI) take(E.phi[l], E.d3 ? E.dzphi[l] : nullptr);
    if (mask & PF_FIELD_P) take(E.P[l], E.d3 ? E.dzP[l] : nullptr);
    if (mask & PF_FIELD_U)
        for (int c = 0; c < 3; ++c) take(E.u[c][l], E.d3 ? E.dzu[c][l] : nullptr);
    if (mask & PF_FIELD_V && !old) E.efield(E.V[l]);
    if (reset) {
        copy_level(E, E.cur, 1 - E.cur);
        h->nstep = 0;
    }
    PF_CU(cudaStreamSynchronize(E.st));
    return PF_OK;
}
}  // namespace

extern "C" int pf_get_fields(pf_handle *h, unsigned mask, double *host_out, size_t n) {
    if (!h || !host_out) return PF_EINVAL;
    try {
        if (h->e64) return get_impl(h, *h->e64, mask, host_out, n);
        return get_impl(h, *h->e32, mask, host_out, n);
    } catch (const CudaError &e) {
        return cuda_fail(h, e);
    }
}

extern "C" int pf_set_fields(pf_handle *h, unsigned mask, const double *host_in, size_t n, int reset_history) {
    if (!h || !host_in) return PF_EINVAL;
    try {
        if (h->e64) return set_impl(h, *h->e64, mask, host_in, n, reset_history);
        return set_impl(h, *h->e32, mask, host_in, n, reset_history);
    } catch (const CudaError &e) {
        return cuda_fail(h, e);
    }
}

namespace {
template <typename T>
int diag_impl(pf_handle *h, Engine<T> &E, double *out) {
    PF_CU(cudaStreamSynchronize(E.st));
    const int n = E.cur;
    const double plane_w = E.d3 ? h->hs.lz / E.nz : 1.0;
    out[0] = E.reduce(E.phi[n], nullptr, 0) * plane_w;
    double um = 0.0;
    for (int c = 0; c < 3; ++c)
        if (E.u[c][n]) {
            const double v = E.reduce(E.u[c][n], nullptr, 1);
            um = (v != v) ? v : std::max(um, v);
        }
    out[1] = um;
    out[2] = h->t;
    out[3] = (double)h->nstep;
    out[4] = h->v_iters;
    if (!(out[0] == out[0]) || !(um == um)) h->diverged = true;
    out[5] = h->diverged ? 1.0 : 0.0;
    out[6] = E.reduce(E.phi[n], E.phi[1 - n], 2) / h->hs.dt;
    out[7] = E.energy();
    return PF_OK;
}

template <typename T>
int helm_impl(pf_handle *h, Engine<T> &E, int bcset, int mode, double lambda, const double *rhs, double *out) {
    const int np = mode == 0 ? 1 : 2;
    const HostSetup &s = h->hs;
    std::vector<T> b((size_t)np * E.n2);
    for (int pl = 0; pl < np; ++pl)
        for (int i = 0; i < E.ny; ++i)
            for (int j = 0; j < E.nx; ++j) {
                const size_t q = (size_t)i * E.nx + j;
                b[(size_t)pl * E.n2 + q] = (T)(s.Mx[j] * s.My[i] * rhs[(size_t)pl * E.n2 + q]);
            }
    const double beta = E.d3 ? 2.0 * M_PI * mode / s.lz : 0.0;
    std::vector<T> sh(3 * E.nz, (T)(lambda + beta * beta));
    PF_CU(cudaMemcpyAsync(E.shTmp, sh.data(), sh.size() * sizeof(T), cudaMemcpyHostToDevice, E.st));
    PF_CU(cudaMemcpyAsync(E.RHS, b.data(), b.size() * sizeof(T), cudaMemcpyHostToDevice, E.st));
    E.fdm(E.RHS, E.OUT, bcset, E.shTmp, np);
    std::vector<T> o((size_t)np * E.n2);
    PF_CU(cudaMemcpyAsync(o.data(), E.OUT, o.size() * sizeof(T), cudaMemcpyDeviceToHost, E.st));
    PF_CU(cudaStreamSynchronize(E.st));
    for (size_t i = 0; i < o.size(); ++i) out[i] = (double)o[i];
    if (E.take_err()) return fail(h, PF_ETIMEOUT, "a tensor-core transform gave up waiting (bounded mbarrier wait)");
    return PF_OK;
}
}  // namespace

extern "C" int pf_diagnostics(pf_handle *h, double out[8]) {
    if (!h || !out) return PF_EINVAL;
    try {
        if (h->e64) return diag_impl(h, *h->e64, out);
        return diag_impl(h, *h->e32, out);
    } catch (const CudaError &e) {
        return cuda_fail(h, e);
    }
}

extern "C" int pf_solve_helmholtz(pf_handle *h, int bcset, int mode, double lambda, const double *rhs, double *out) {
    if (!h || !rhs || !out) return PF_EINVAL;
    if (bcset < 0 || bcset > 3) return fail(h, PF_EINVAL, "bcset must be one of PF_BCSET_*");
    if (mode < 0 || (h->hs.nz == 1 && mode != 0) || (h->hs.nz > 1 && mode > h->hs.nz / 2))
        return fail(h, PF_EINVAL, "mode out of range");
    try {
        if (h->e64) return helm_impl(h, *h->e64, bcset, mode, lambda, rhs, out);
        return helm_impl(h, *h->e32, bcset, mode, lambda, rhs, out);
    } catch (const CudaError &e) {
        return cuda_fail(h, e);
    }
}

extern "C" int pf_profile(pf_handle *h, int enable) {
    if (!h) return PF_EINVAL;
    try {
        PF_CU(cudaStreamSynchronize(h->st));
        h->prof.resolve();
        h->prof.on = enable != 0;
        if (h->prof.on)
            for (int k = 0; k < PF_KC_COUNT; ++k) h->prof.ms[k] = 0.0;
    } catch (const CudaError &e) {
        return cuda_fail(h, e);
    }
    return PF_OK;
}

extern "C" int pf_profile_read(pf_handle *h, double *ms, long long *launches) {
    if (!h) return PF_EINVAL;
    try {
        PF_CU(cudaStreamSynchronize(h->st));
        h->prof.resolve();
    } catch (const CudaError &e) {
        return cuda_fail(h, e);
    }
    for (int k = 0; k < PF_KC_COUNT; ++k) {
        if (ms) ms[k] = h->prof.on ? h->prof.ms[k] : 0.0;
        if (launches) launches[k] = h->prof.launches[k];
    }
    return PF_OK;
}

namespace {
// time `steps` steady steps of each transform variant, keep the fastest; advances `total` steps.
// Steps run as the run will run them: replays of the captured graphs on a non-default stream
// (re-captured for every variant), eager launches on the legacy stream.
template <typename T>
void autotune_engine(Engine<T> &E, int steps, int total, cudaEvent_t e0, cudaEvent_t e1, int *choice, double *best_ms) {
    auto drop_graphs = [&]() {
        for (int c = 0; c < 2; ++c)
            if (E.graph[c]) { cudaGraphExecDestroy(E.graph[c]); E.graph[c] = nullptr; }
    };
    auto one = [&]() {
        if (E.st != nullptr && !E.prof->on) E.step_graph();
        else E.step(2);
    };
    // two untimed steps (both history parities captured), then `steps` timed ones
    auto time_variant = [&](int &taken) {
        drop_graphs();
        one();
        one();
        PF_CU(cudaEventRecord(e0, E.st));
        for (int s = 0; s < steps; ++s) one();
        PF_CU(cudaEventRecord(e1, E.st));
        PF_CU(cudaEventSynchronize(e1));
        taken += steps + 2;
        float ms = 0.f;
        PF_CU(cudaEventElapsedTime(&ms, e0, e1));
        return (double)ms / steps;
    };
    // every variant this engine can run (PF_GEMM_* codes)
    std::vector<int> cands;
    for (int code : {0, 8, 32, 64, 2, 3, 4, 5, 1, 6, 7})
        if (E.gemm_available(code)) cands.push_back(code);
    int pick = cands[0];
    double best = INFINITY;
    int taken = 0;
    for (int code : cands) {
        E.set_gemm(code);
        const double ms = time_variant(taken);
        if (ms < best) { best = ms; pick = code; }
    }
    E.set_gemm(pick);
    // the fused y pair against the two separate y transforms (the whole-plane solves have no y pair)
    if (!E.fuse_plane && !E.cluster) {
        E.fuse_y = !E.fuse_y;
        const double ms = time_variant(taken);
        if (ms < best) best = ms;
        else E.fuse_y = !E.fuse_y;
    }
    // then the transform tile (pencils per block), with the chosen GEMM
    if (E.d3) {
        int best_tp = 0;
        for (int tp : {4, 8, 16, 32}) {
            E.tp_override = tp;
            const double ms = time_variant(taken);
            if (ms < best) { best = ms; best_tp = tp; }
        }
        E.tp_override = best_tp;
    }
    drop_graphs();
    for (; taken < total; ++taken) E.step(2);
    if (choice) *choice = pick + 1000 * E.tp_override + ((E.fuse_y && !E.fuse_plane && !E.cluster) ? 100000 : 0);
    if (best_ms) *best_ms = best;
}
}  // namespace

extern "C" int pf_autotune(pf_handle *h, int steps, int *choice, double *ms_per_step) {
    if (!h || steps < 1) return PF_EINVAL;
    try {
        if (h->nstep < 1) pf_step(h, 1);
        int total = 16 * (steps + 2);   // at most 11 transform variants + the y pair + 4 tiles
        cudaEvent_t e0, e1;
        PF_CU(cudaEventCreate(&e0));
        PF_CU(cudaEventCreate(&e1));
        if (h->e64) autotune_engine(*h->e64, steps, total, e0, e1, choice, ms_per_step);
        else autotune_engine(*h->e32, steps, total, e0, e1, choice, ms_per_step);
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        h->nstep += total;
        h->t += total * h->hs.dt;
        h->last_J = 2;
    } catch (const CudaError &e) {
        return cuda_fail(h, e);
    }
    return PF_OK;
}

namespace {
// pin the transform variants of one engine; false when the engine cannot use them
template <typename T>
bool set_variant(Engine<T> &E, int gemm, int fuse_y, int tile) {
    const bool tile_ok = tile == 0 || tile == 4 || tile == 8 || tile == 16 || tile == 32;
    if (!E.gemm_available(gemm) || (fuse_y != 0 && fuse_y != 1) || !tile_ok) return false;
    E.set_gemm(gemm);
    E.fuse_y = fuse_y == 1;
    E.tp_override = tile;
    for (int c = 0; c < 2; ++c)
        if (E.graph[c]) { cudaGraphExecDestroy(E.graph[c]); E.graph[c] = nullptr; }
    return true;
}
}  // namespace

extern "C" int pf_set_variant(pf_handle *h, int gemm, int fuse_y, int tile) {
    if (!h) return PF_EINVAL;
    try {
        PF_CU(cudaStreamSynchronize(h->st));
        const bool ok = h->e64 ? set_variant(*h->e64, gemm, fuse_y, tile) : set_variant(*h->e32, gemm, fuse_y, tile);
        if (!ok) {
            h->err = "pf_set_variant: variant not available for this run";
            return PF_EINVAL;
        }
    } catch (const CudaError &e) {
        return cuda_fail(h, e);
    }
    return PF_OK;
}

extern "C" int pf_set_tc_accum(pf_handle *h, int gemm, int family, int slices, int sep) {
    if (!h) return PF_EINVAL;
    if (gemm != PF_GEMM_TC && gemm != PF_GEMM_TC_HYBRID) return fail(h, PF_EINVAL, "gemm must be PF_GEMM_TC or PF_GEMM_TC_HYBRID");
    if (family != 0 && family != 1) return fail(h, PF_EINVAL, "family 0 (psi, phi solves) or 1 (V, P, u solves)");
    if (slices < 1 || slices > 64 || (sep != 0 && sep != 1)) return fail(h, PF_EINVAL, "slices in [1, 64], sep 0 or 1");
    if (!h->e32) return fail(h, PF_EINVAL, "tensor-core transforms run in PF_MIXED only");
    try {
        PF_CU(cudaStreamSynchronize(h->st));
        auto &E = *h->e32;
        const int v = gemm == PF_GEMM_TC_HYBRID ? 1 : 0;
        E.tc_gs[v][family] = slices;
        E.tc_sepv[v][family] = sep;
        for (int c = 0; c < 2; ++c)
            if (E.graph[c]) { cudaGraphExecDestroy(E.graph[c]); E.graph[c] = nullptr; }
    } catch (const CudaError &e) {
        return cuda_fail(h, e);
    }
    return PF_OK;
}

extern "C" int pf_set_step(pf_handle *h, int nstep, double t) {
    if (!h) return PF_EINVAL;
    if (nstep < 0 || !std::isfinite(t)) return fail(h, PF_EINVAL, "nstep must be >= 0 and t finite");
    h->nstep = nstep;
    h->t = t;
    return PF_OK;
}

extern "C" int pf_debug_tc_stall(pf_handle *h, unsigned long long wait_ns) {
    if (!h) return PF_EINVAL;
    if (!h->e32 || !h->e32->use_tc || h->e32->tcb.empty())
        return fail(h, PF_EINVAL, "the handle does not run its transforms on the tensor cores");
    if (wait_ns == 0 || wait_ns > 10000000000ull) return fail(h, PF_EINVAL, "wait_ns must be in (0, 1e10]");
    h->e32->tc_stall = 1;
    h->e32->tc_wait_ns_next = wait_ns;
    return PF_OK;
}

extern "C" int pf_geometry(const pf_handle *h, double *nodes_x, double *nodes_y, int dims[4]) {
    if (!h) return PF_EINVAL;
    const HostSetup &s = h->hs;
    if (nodes_x) std::copy(s.X.begin(), s.X.end(), nodes_x);
    if (nodes_y) std::copy(s.Y.begin(), s.Y.end(), nodes_y);
    if (dims) {
        dims[0] = s.nx; dims[1] = s.ny; dims[2] = s.nz;
        dims[3] = s.nx * s.ny * s.nz;
    }
    return PF_OK;
}

extern "C" void pf_destroy(pf_handle *h) {
    if (!h) return;
    if (h->st) cudaStreamSynchronize(h->st);
    else cudaDeviceSynchronize();
    delete h;
}

extern "C" const char *pf_last_error(const pf_handle *h) {
    if (!h) return g_create_error.c_str();
    return h->err.c_str();
}

// ============================================================================================
// Ensembles of independent 2D runs
struct pf_batch {
    struct Group {
        HostSetup hs;
        Prof prof;
        std::unique_ptr<Engine<double>> e64;
        std::unique_ptr<Engine<float>> e32;
        std::vector<int> runs;
        int v_iters = 0;
        cudaStream_t gst = nullptr;        // the group's own stream: groups run concurrently
        cudaEvent_t joined = nullptr;      // recorded on gst at the end of a step
    };
    std::vector<std::unique_ptr<Group>> groups;
    std::vector<std::pair<int, int>> where;   // run -> (group, plane)
    cudaStream_t st = nullptr;
    cudaEvent_t fork = nullptr;                // recorded on st before a step
    long long nstep = 0;
    int bdf = 2;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    std::vector<std::vector<long long>> gcounts[2];   // per-group launches of one replayed step
    std::string err;
    ~pf_batch() {
        for (int c = 0; c < 2; ++c)
            if (graph[c]) cudaGraphExecDestroy(graph[c]);
        for (auto &g : groups)
            if (g->gst) cudaStreamSynchronize(g->gst);
        groups.clear();   // engines first, then their streams and events
        for (auto e : streams_events) {
            if (e.first) cudaStreamDestroy(e.first);
            if (e.second) cudaEventDestroy(e.second);
        }
        if (fork) cudaEventDestroy(fork);
    }
    std::vector<std::pair<cudaStream_t, cudaEvent_t>> streams_events;
};

namespace {

bool same_group(const HostSetup &a, const HostSetup &b) {
    return a.ex == b.ex && a.ey == b.ey && a.K == b.K && a.xb == b.xb && a.yb == b.yb && a.rho1 == b.rho1 &&
           a.rho2 == b.rho2 && a.mu1 == b.mu1 && a.mu2 == b.mu2 && a.sigma == b.sigma && a.eta == b.eta &&
           a.gamma1 == b.gamma1 && a.theta == b.theta && a.vrow0 == b.vrow0 && a.vrow1 == b.vrow1 &&
           a.dt == b.dt && a.bdf == b.bdf && a.precision == b.precision && a.S == b.S && a.nu_m == b.nu_m &&
           a.rho0 == b.rho0 && a.model == b.model;
}

template <typename F>
void for_engine(pf_batch::Group &g, F f) {
    if (g.e64) f(*g.e64);
    else f(*g.e32);
}

std::vector<std::vector<long long>> &graph_counts(pf_batch *b, int c) { return b->gcounts[c]; }

int batch_fail(pf_batch *b, int code, const std::string &m) {
    b->err = m;
    return code;
}

void batch_invalidate_graphs(pf_batch *b) {
    for (int c = 0; c < 2; ++c)
        if (b->graph[c]) {
            cudaGraphExecDestroy(b->graph[c]);
            b->graph[c] = nullptr;
        }
}

// one step of every group, each on its own stream, between a fork on the ensemble's stream and a
// join back into it (in a capture the group streams join the graph as concurrent branches)
void batch_step_groups(pf_batch *b, int J) {
    PF_CU(cudaEventRecord(b->fork, b->st));
    for (auto &g : b->groups) {
        PF_CU(cudaStreamWaitEvent(g->gst, b->fork, 0));
        for_engine(*g, [&](auto &E) { E.step(J); });
        PF_CU(cudaEventRecord(g->joined, g->gst));
        PF_CU(cudaStreamWaitEvent(b->st, g->joined, 0));
    }
}

void batch_step_once(pf_batch *b) {
    const int J = (b->nstep == 0 || b->bdf == 1) ? 1 : 2;
    if (J == 1 || b->st == nullptr) {
        batch_step_groups(b, J);
    } else {
        int c = 0;
        for_engine(*b->groups[0], [&](auto &E) { c = E.cur; });
        if (!b->graph[c]) {
            cudaGraph_t gr = nullptr;
            std::vector<std::vector<long long>> before;
            for (auto &g : b->groups) before.emplace_back(g->prof.launches, g->prof.launches + PF_KC_COUNT);
            PF_CU(cudaStreamBeginCapture(b->st, cudaStreamCaptureModeThreadLocal));
            try {
                batch_step_groups(b, 2);
            } catch (...) {
                cudaStreamEndCapture(b->st, &gr);
                if (gr) cudaGraphDestroy(gr);
                throw;
            }
            PF_CU(cudaStreamEndCapture(b->st, &gr));
            cudaError_t e = cudaGraphInstantiate(&b->graph[c], gr, 0);
            cudaGraphDestroy(gr);
            PF_CU(e);
            // the capture ran nothing: restore the slots and the counters
            for (size_t i = 0; i < b->groups.size(); ++i) {
                auto &g = *b->groups[i];
                for_engine(g, [&](auto &E) { E.cur = c; });
                for (int k = 0; k < PF_KC_COUNT; ++k) {
                    const long long d = g.prof.launches[k] - before[i][k];
                    g.prof.launches[k] = before[i][k];
                    before[i][k] = d;   // per-step launches of this group
                }
            }
            // remember the per-step launch counts in the first group's graph slot via a side table
            b->err.clear();
            graph_counts(b, c) = before;
        }
        PF_CU(cudaGraphLaunch(b->graph[c], b->st));
        // later work on the group streams (reads, eager steps) comes after the replayed step
        PF_CU(cudaEventRecord(b->fork, b->st));
        for (auto &g : b->groups) PF_CU(cudaStreamWaitEvent(g->gst, b->fork, 0));
        for (size_t i = 0; i < b->groups.size(); ++i) {
            auto &g = *b->groups[i];
            for (int k = 0; k < PF_KC_COUNT; ++k) g.prof.launches[k] += graph_counts(b, c)[i][k];
            for_engine(g, [&](auto &E) { E.cur = 1 - c; });
        }
    }
    b->nstep += 1;
}

}  // namespace

extern "C" int pf_batch_create(int nrun, const pf_mesh *meshes, const pf_fluid *fluids, const pf_vbc *vbcs,
                               const pf_scheme *scheme, const double *const *phi0, void *cuda_stream,
                               pf_batch **out) {
    if (out) *out = nullptr;
    if (nrun < 1 || !meshes || !fluids || !vbcs || !scheme || !phi0 || !out)
        return fail(nullptr, PF_EINVAL, "pf_batch_create: null argument or nrun < 1");
    std::unique_ptr<pf_batch> b(new pf_batch());
    b->st = (cudaStream_t)cuda_stream;
    b->bdf = scheme->bdf;
    b->where.resize(nrun);
    std::vector<HostSetup> setups(nrun);
    for (int r = 0; r < nrun; ++r) {
        std::string err;
        if (vbcs[r].bottom_kind == PF_BC_PATCHES)
            return fail(nullptr, PF_EINVAL, "electrode patches are not supported in ensembles");
        const int rc = fill_setup(&meshes[r], &fluids[r], &vbcs[r], scheme, setups[r], err);
        if (rc != PF_OK) return fail(nullptr, rc, "run " + std::to_string(r) + ": " + err);
        if (meshes[r].nz != 1) return fail(nullptr, PF_EINVAL, "ensemble runs must be 2D (nz = 1)");
        if (!phi0[r]) return fail(nullptr, PF_EINVAL, "null phi0 of run " + std::to_string(r));
    }
    for (int r = 0; r < nrun; ++r) {
        int gi = -1;
        for (size_t g = 0; g < b->groups.size(); ++g)
            if (same_group(b->groups[g]->hs, setups[r])) { gi = (int)g; break; }
        if (gi < 0) {
            b->groups.emplace_back(new pf_batch::Group());
            b->groups.back()->hs = setups[r];
            gi = (int)b->groups.size() - 1;
        }
        auto &g = *b->groups[gi];
        b->where[r] = {gi, (int)g.runs.size()};
        g.runs.push_back(r);
        g.hs.beps1.push_back(setups[r].eps1);
        g.hs.beps2.push_back(setups[r].eps2);
        g.hs.bvb.push_back(setups[r].v0);
        g.hs.bvt.push_back(setups[r].v1);
    }
    try {
        PF_CU(cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming));
        for (auto &gp : b->groups) {
            auto &g = *gp;
            PF_CU(cudaStreamCreateWithFlags(&g.gst, cudaStreamNonBlocking));
            PF_CU(cudaEventCreateWithFlags(&g.joined, cudaEventDisableTiming));
            b->streams_events.push_back({g.gst, g.joined});
            g.hs.batch = (int)g.runs.size();
            build_setup(g.hs);
            const size_t n2 = (size_t)g.hs.nx * g.hs.ny;
            std::vector<double> phi(n2 * g.runs.size());
            for (size_t i = 0; i < g.runs.size(); ++i) std::copy(phi0[g.runs[i]], phi0[g.runs[i]] + n2, phi.begin() + i * n2);
            std::string err;
            const int rc = build_engines(g.hs, phi.data(), nullptr, g.gst, &g.prof, g.e64, g.e32, g.v_iters, err);
            if (rc != PF_OK) return fail(nullptr, rc, err);
        }
    } catch (const CudaError &e) {
        g_create_error = e.where + ": " + cudaGetErrorString(e.code);
        return e.code == cudaErrorMemoryAllocation ? PF_ENOMEM : PF_ECUDA;
    }
    *out = b.release();
    return PF_OK;
}

extern "C" int pf_batch_step(pf_batch *b, int nsteps) {
    if (!b || nsteps < 0) return PF_EINVAL;
    try {
        for (int s = 0; s < nsteps; ++s) batch_step_once(b);
    } catch (const CudaError &e) {
        return batch_fail(b, PF_ECUDA, e.where + ": " + cudaGetErrorString(e.code));
    }
    return PF_OK;
}

extern "C" int pf_batch_umax(pf_batch *b, double *umax, double *mass) {
    if (!b || !umax) return PF_EINVAL;
    try {
        for (auto &gp : b->groups) {
            auto &g = *gp;
            const int B = (int)g.runs.size();
            std::vector<double> um(B, 0.0), t(B), m(B);
            for_engine(g, [&](auto &E) {
                if (g.hs.model == PF_MODEL_EQUILIBRIUM) {
                    E.reduce_planes(E.phi[E.cur], 1, t.data(), E.phi[1 - E.cur]);
                    for (int i = 0; i < B; ++i) um[i] = t[i] / g.hs.dt;
                } else {
                    for (int c = 0; c < 2; ++c) {
                        E.reduce_planes(E.u[c][E.cur], 1, t.data());
                        for (int i = 0; i < B; ++i) um[i] = (t[i] != t[i] || um[i] != um[i]) ? NAN : std::max(um[i], t[i]);
                    }
                }
                if (mass) E.reduce_planes(E.phi[E.cur], 0, m.data());
            });
            for (int i = 0; i < B; ++i) {
                umax[g.runs[i]] = um[i];
                if (mass) mass[g.runs[i]] = m[i];
            }
        }
    } catch (const CudaError &e) {
        return batch_fail(b, PF_ECUDA, e.where + ": " + cudaGetErrorString(e.code));
    }
    return PF_OK;
}

extern "C" int pf_batch_run_to_equilibrium(pf_batch *b, double tol, int max_steps, int check_every, int *steps_out) {
    if (!b || !steps_out || check_every < 1 || max_steps < 0 || !(tol >= 0.0)) return PF_EINVAL;
    const int nrun = (int)b->where.size();
    try {
        // every run active, its step count the ensemble's; each step ends with the device check
        for (auto &g : b->groups) for_engine(*g, [&](auto &E) { E.reset_exit(tol, (int)b->nstep); });
        while (b->nstep < max_steps) {
            const int n = (int)std::min<long long>(check_every, max_steps - b->nstep);
            const int rc = pf_batch_step(b, n);
            if (rc != PF_OK) return rc;
            bool any = false;   // the host only decides when to stop launching
            for (auto &g : b->groups)
                for_engine(*g, [&](auto &E) {
                    std::vector<int> act(E.nz);
                    PF_CU(cudaMemcpyAsync(act.data(), E.active, E.nz * sizeof(int), cudaMemcpyDeviceToHost, E.st));
                    PF_CU(cudaStreamSynchronize(E.st));
                    for (int v : act) any = any || v;
                });
            if (!any) break;
        }
        for (auto &g : b->groups)
            for_engine(*g, [&](auto &E) {
                std::vector<int> at(E.nz);
                PF_CU(cudaMemcpyAsync(at.data(), E.steps_at, E.nz * sizeof(int), cudaMemcpyDeviceToHost, E.st));
                PF_CU(cudaStreamSynchronize(E.st));
                for (size_t i = 0; i < g->runs.size(); ++i) steps_out[g->runs[i]] = at[i];
                E.reset_exit(-1.0, (int)b->nstep);   // later pf_batch_step calls advance every run again
            });
    } catch (const CudaError &e) {
        return batch_fail(b, PF_ECUDA, e.where + ": " + cudaGetErrorString(e.code));
    }
    (void)nrun;
    return PF_OK;
}

extern "C" int pf_batch_get_fields(pf_batch *b, int run, unsigned mask, double *host_out, size_t n) {
    if (!b || !host_out || run < 0 || run >= (int)b->where.size()) return PF_EINVAL;
    auto &g = *b->groups[b->where[run].first];
    const int pl = b->where[run].second;
    const size_t n2 = (size_t)g.hs.nx * g.hs.ny;
    size_t need = 0;
    if (mask & PF_FIELD_V) need += 1;
    if (mask & PF_FIELD_E) need += 3;
    if (mask & PF_FIELD_PHI) need += 1;
    if (mask & PF_FIELD_PSI) need += 1;
    if (mask & PF_FIELD_P) need += 1;
    if (mask & PF_FIELD_U) need += 3;
    if (need * n2 > n) return batch_fail(b, PF_EINVAL, "output buffer too small");
    try {
        for_engine(g, [&](auto &E) {
            using T = typename std::remove_reference<decltype(*E.V[0])>::type;
            PF_CU(cudaStreamSynchronize(E.st));
            const int l = (mask & PF_FIELD_OLD) ? 1 - E.cur : E.cur;
            double *o = host_out;
            std::vector<T> tmp(n2);
            auto put = [&](const T *src) {
                if (src) {
                    PF_CU(cudaMemcpy(tmp.data(), src + (size_t)pl * n2, n2 * sizeof(T), cudaMemcpyDeviceToHost));
                    for (size_t i = 0; i < n2; ++i) o[i] = (double)tmp[i];
                } else {
                    std::fill(o, o + n2, 0.0);
                }
                o += n2;
            };
            if (mask & PF_FIELD_V) put(E.V[l]);
            if (mask & PF_FIELD_E) { put(E.Ex); put(E.Ey); put(nullptr); }
            if (mask & PF_FIELD_PHI) put(E.phi[l]);
            if (mask & PF_FIELD_PSI) {
                std::vector<T> ph(n2);
                PF_CU(cudaMemcpy(ph.data(), E.phi[E.cur] + (size_t)pl * n2, n2 * sizeof(T), cudaMemcpyDeviceToHost));
                put(E.Lf);
                const double al = alpha_of(g.hs, (b->nstep <= 1 || g.hs.bdf == 1) ? 1 : 2);
                for (size_t i = 0; i < n2; ++i) o[(ptrdiff_t)i - (ptrdiff_t)n2] += al * (double)ph[i];
            }
            if (mask & PF_FIELD_P) put(E.P[l]);
            if (mask & PF_FIELD_U) { put(E.u[0][l]); put(E.u[1][l]); put(nullptr); }
        });
    } catch (const CudaError &e) {
        return batch_fail(b, PF_ECUDA, e.where + ": " + cudaGetErrorString(e.code));
    }
    return PF_OK;
}

extern "C" const char *pf_batch_last_error(const pf_batch *b) {
    if (!b) return g_create_error.c_str();
    return b->err.c_str();
}

extern "C" int pf_batch_set_variant(pf_batch *b, int gemm, int fuse_y) {
    if (!b) return PF_EINVAL;
    try {
        PF_CU(cudaStreamSynchronize(b->st));
        for (auto &gp : b->groups) {   // every group must be able to take the variant
            bool ok = true;
            for_engine(*gp, [&](auto &E) {
                ok = E.gemm_available(gemm);
            });
            if (!ok || (fuse_y != 0 && fuse_y != 1))
                return batch_fail(b, PF_EINVAL, "pf_batch_set_variant: variant not available for every group");
        }
        for (auto &gp : b->groups) for_engine(*gp, [&](auto &E) { set_variant(E, gemm, fuse_y, 0); });
        batch_invalidate_graphs(b);
    } catch (const CudaError &e) {
        return batch_fail(b, PF_ECUDA, e.where + ": " + cudaGetErrorString(e.code));
    }
    return PF_OK;
}

extern "C" int pf_batch_autotune(pf_batch *b, int steps, double *ms_out) {
    if (!b || steps < 1) return PF_EINVAL;
    try {
        // make sure the timed steps are steady (BDF2) steps
        if (b->nstep < 1) batch_step_once(b);
        cudaEvent_t e0, e1;
        PF_CU(cudaEventCreate(&e0));
        PF_CU(cudaEventCreate(&e1));
        // every group takes the same number of steps (6 variants x (steps + 1), rounded up to an
        // even count so the history-slot parity of all groups stays equal)
        int total = 6 * (steps + 1);
        if (total % 2) total += 1;
        for (size_t gi = 0; gi < b->groups.size(); ++gi) {
            auto &g = *b->groups[gi];
            double best = INFINITY;
            for_engine(g, [&](auto &E) {
                std::vector<int> cands;
                for (int code : {0, 32, 64, 1, 6, 7})
                    if (E.gemm_available(code)) cands.push_back(code);
                int pick = cands[0];
                int taken = 0;
                for (int code : cands) {
                    E.set_gemm(code);
                    E.step(2);   // warm-up of this variant
                    PF_CU(cudaEventRecord(e0, E.st));
                    for (int s = 0; s < steps; ++s) E.step(2);
                    PF_CU(cudaEventRecord(e1, E.st));
                    PF_CU(cudaEventSynchronize(e1));
                    taken += steps + 1;
                    float ms = 0.f;
                    PF_CU(cudaEventElapsedTime(&ms, e0, e1));
                    if (ms / steps < best) { best = ms / steps; pick = code; }
                }
                E.set_gemm(pick);
                for (; taken < total; ++taken) E.step(2);
            });
            if (ms_out) ms_out[gi] = best;
        }
        b->nstep += total;
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        batch_invalidate_graphs(b);
    } catch (const CudaError &e) {
        return batch_fail(b, PF_ECUDA, e.where + ": " + cudaGetErrorString(e.code));
    }
    return (int)b->groups.size();
}

extern "C" int pf_batch_groups(const pf_batch *b, int *group_of) {
    if (!b) return PF_EINVAL;
    if (group_of)
        for (size_t r = 0; r < b->where.size(); ++r) group_of[r] = b->where[r].first;
    return (int)b->groups.size();
}

extern "C" void pf_batch_destroy(pf_batch *b) {
    if (!b) return;
    if (b->st) cudaStreamSynchronize(b->st);
    else cudaDeviceSynchronize();
    delete b;
}
