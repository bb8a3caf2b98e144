// Allocation-free variant of the fast-diagonalisation solve (FP64).
//
// Some callers cannot allocate device memory at the point where they need a solve:
// code running inside a region that forbids or cannot afford cudaMalloc (it may
// synchronise the device), a memory-planned real-time loop, or a host library that
// brings its own allocator and must not see a second one.  For them,
// pf_fdm_solve_static takes every input and output as a caller-owned device pointer
// and keeps its two intermediate buffers in the file-scope array below, which every
// GPU that loads this library holds until the process exits.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "../../include/pf.h"
#include "pf_kernels.cuh"

void pf_internal_set_error(const std::string &msg);   // pf_api.cu: message for pf_last_error(NULL)

namespace {

// Two scratch planes sets of PF_STATIC_MAX_VALUES doubles each (16 MiB in total).
static __device__ __align__(256) double g_fdm_scratch[2 * PF_STATIC_MAX_VALUES];

std::mutex g_mu;
double *g_scratch_ptr[64] = {nullptr};   // device address of g_fdm_scratch, per device

// Device address of the scratch array on the current device, looked up once per device.
// Host code must not pass the symbol itself to a kernel: on the host it only names a
// stand-in object, not device memory.
int scratch_for_current_device(double **out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        pf_internal_set_error(std::string("cudaGetDevice: ") + cudaGetErrorString(e));
        return PF_ECUDA;
    }
    if (dev < 0 || dev >= 64) {
        pf_internal_set_error("device index out of range for the static scratch table");
        return PF_EINVAL;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_fdm_scratch);
        if (e != cudaSuccess || !p) {
            pf_internal_set_error(std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            return PF_ECUDA;
        }
        g_scratch_ptr[dev] = static_cast<double *>(p);
    }
    *out = g_scratch_ptr[dev];
    return PF_OK;
}

int launch_gemm(const double *A, const double *B, double *C, long long rows, int n, int R, int store,
                const double *lamN, const double *lamR, const double *cpl, int cpl_mod, cudaStream_t st) {
    pf::GemmArgs<double> g{A, B, C, rows, n, R, store, lamN, lamR, cpl, cpl_mod};
    dim3 grid((n + 63) / 64, (unsigned)((rows + 63) / 64));
    pf::k_gemm<double, 64, 64, 8, 4, 4><<<grid, 256, 0, st>>>(g);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        pf_internal_set_error(std::string("k_gemm launch: ") + cudaGetErrorString(e));
        return PF_ECUDA;
    }
    return PF_OK;
}

}  // namespace

extern "C" int pf_fdm_solve_static(int nx, int ny, int nplanes, const double *Sx, const double *SxT,
                                   const double *lam_x, const double *Sy, const double *SyT,
                                   const double *lam_y, const double *shift, const double *rhs, double *out,
                                   void *cuda_stream) {
    if (nx < 1 || ny < 1 || nplanes < 1 || !Sx || !SxT || !lam_x || !Sy || !SyT || !lam_y || !shift || !rhs ||
        !out) {
        pf_internal_set_error("pf_fdm_solve_static: null pointer or non-positive size");
        return PF_EINVAL;
    }
    const long long total = (long long)nx * ny * nplanes;
    if (total > PF_STATIC_MAX_VALUES) {
        pf_internal_set_error("pf_fdm_solve_static: nx*ny*nplanes exceeds PF_STATIC_MAX_VALUES");
        return PF_EINVAL;
    }
    double *scratch = nullptr;
    int rc = scratch_for_current_device(&scratch);
    if (rc != PF_OK) return rc;
    double *W1 = scratch, *W2 = scratch + PF_STATIC_MAX_VALUES;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const long long P = nplanes;
    // the same four transforms as the handle's solves: x, y (+ eigenvalue division), y^T, x^T
    if ((rc = launch_gemm(rhs, Sx, W1, P * ny, nx, ny, 1, nullptr, nullptr, nullptr, 1, st)) != PF_OK) return rc;
    if ((rc = launch_gemm(W1, Sy, W2, P * nx, ny, nx, 0, lam_y, lam_x, shift, nplanes, st)) != PF_OK) return rc;
    if ((rc = launch_gemm(W2, SyT, W1, P * nx, ny, nx, 1, nullptr, nullptr, nullptr, 1, st)) != PF_OK) return rc;
    return launch_gemm(W1, SxT, out, P * ny, nx, ny, 0, nullptr, nullptr, nullptr, 1, st);
}
