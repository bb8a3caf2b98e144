/*
 * pf.h -- C-ABI of the GB300 (sm_103a) implementation of the decoupled
 * phase-field scheme for two immiscible dielectric fluids
 * (Yang, Christov & Dong, arXiv 2305.09020).
 *
 * The library advances the per-time-step path of Algorithm 1 (2D, eqs. 54-59)
 * and Algorithm 2 (3D hybrid Fourier/spectral element, eqs. 74-78):
 *   potential V -> field E -> auxiliary psi -> phase field phi -> pressure P
 *   -> velocity u, each a constant-coefficient Helmholtz problem per Fourier
 * mode (Remark after Algorithm 2), solved by fast diagonalisation with 1D
 * generalised eigenbases computed once at set-up.
 *
 * Conventions shared by every entry point
 *  - Return 0 (PF_OK) on success, a negative PF_E* code on failure; the
 *    handle's message is then readable with pf_last_error().
 *  - Host buffers are always owned by the caller; the library never keeps a
 *    pointer to them after the call returns.
 *  - Device memory is owned by the handle (allocated in pf_create, freed in
 *    pf_destroy); all work is issued on the stream given to pf_create.
 *  - Field layout: values at the unique tensor-product GLL nodes, ordered
 *    [z][y][x] with x fastest.  n_x = ex*order (x is periodic),
 *    n_y = ey*order + 1, Nz planes in z (Nz = 1 for 2D).  Public values are
 *    double precision whatever the internal precision.
 *  - Boundaries: x (and z) periodic; y = yb[0] is the solid wall
 *    (u = 0, wetting condition eq. 19 with contact angle theta_s), y = yb[ey]
 *    is the open side (eqs. a19, a24: P = 0, du/dn = 0).  The potential takes
 *    a whole-side Dirichlet (electrode) or homogeneous Neumann condition on
 *    each of the two sides (eq. 21 with an electrode covering the side).
 */
#ifndef PF_H
#define PF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------------------------- */
#define PF_OK             0
#define PF_EINVAL        -1   /* invalid argument (sizes, pointers, parameters)            */
#define PF_ENOMEM        -2   /* device or host allocation failed                          */
#define PF_ECUDA         -3   /* a CUDA runtime call or kernel launch failed              */
#define PF_ENOTSEPARABLE -4   /* boundary data that is not a whole-side condition         */
#define PF_EDIVERGED     -5   /* a non-finite value appeared in the state                  */
#define PF_ETIMEOUT      -6   /* a bounded device-side wait gave up                        */
#define PF_ESTATE        -7   /* call not valid in the handle's current state              */

/* ---- enumerations ---------------------------------------------------------------------- */
#define PF_BC_DIRICHLET 0
#define PF_BC_NEUMANN   1
#define PF_BC_PATCHES   2   /* wall only: electrodes on parts of the wall (eq. 21), see pf_vbc */

#define PF_FP64  0   /* every kernel in double precision                                  */
#define PF_MIXED 1   /* node-wise kernels and FFT in FP32, eigenbasis GEMMs in 3xTF32 on   */
                     /* the tensor cores (FP32 accumulation); set-up, the initial-potential */
                     /* fixed point and reductions in FP64                                  */
#define PF_MIXED_SIMT 2  /* as PF_MIXED but the eigenbasis GEMMs on the FP32 SIMT pipe     */

/* boundary-condition sets of the Helmholtz solves (y-direction; x is periodic) */
#define PF_BCSET_V   0   /* the potential: per-side Dirichlet/Neumann from pf_vbc           */
#define PF_BCSET_NN  1   /* psi and phi: natural (Neumann) on both sides, eq. 56-57        */
#define PF_BCSET_P   2   /* pressure: natural on the wall, Dirichlet on the open side, 58  */
#define PF_BCSET_U   3   /* velocity: Dirichlet on the wall, natural on the open side, 59  */

/* field selection mask for pf_get_fields / pf_set_fields, in this order */
#define PF_FIELD_V    1u    /* potential V                                                 */
#define PF_FIELD_E    2u    /* electric field Ex, Ey, Ez (3 blocks; Ez = 0 in 2D)         */
#define PF_FIELD_PHI  4u    /* phase field phi                                             */
#define PF_FIELD_PSI  8u    /* auxiliary psi of eq. 44 (get only)                         */
#define PF_FIELD_P   16u    /* pressure P                                                  */
#define PF_FIELD_U   32u    /* velocity ux, uy, uz (3 blocks; uz = 0 in 2D)               */
#define PF_FIELD_OLD 64u    /* with PF_FIELD_V/PHI/P/U: the level n-1 copies (restart)   */

/* ---- descriptors ----------------------------------------------------------------------- */
typedef struct pf_handle pf_handle;   /* opaque; owns all device memory */

typedef struct {
    int ex, ey;            /* elements in x (periodic) and y                               */
    const double *xb;      /* ex+1 increasing breakpoints in x (period xb[ex]-xb[0])       */
    const double *yb;      /* ey+1 increasing breakpoints in y (graded meshes allowed)     */
    int order;             /* element order K (K+1 GLL nodes per direction), 2 <= K <= 15  */
    int nz;                /* Fourier planes in z: 1 (2D) or an even 2^a 3^b 5^c 7^d <= 1024 */
    double lz;             /* period in z (ignored when nz == 1)                           */
} pf_mesh;

typedef struct {
    double rho1, rho2;     /* densities of fluid 1 (phi = +1) and fluid 2 (phi = -1)       */
    double mu1, mu2;       /* dynamic viscosities                                          */
    double eps1, eps2;     /* relative permittivities (mixture law eq. interpolation)     */
    double sigma;          /* surface tension; lambda = 3 sigma eta / (2 sqrt 2)           */
    double eta;            /* interface thickness (Cahn number)                            */
    double gamma1;         /* mobility                                                     */
    double theta_s_deg;    /* static contact angle on the wall, eq. theta_def (90 = none)  */
} pf_fluid;

/* Potential boundary conditions (eq. 21 on the wall, eq. a25 or a Dirichlet top).  Each side is
 * Dirichlet (an electrode over the whole side, voltage v_bottom / v_top) or Neumann (dV/dn = 0);
 * the wall may instead carry electrode patches, bottom_kind = PF_BC_PATCHES: n_patch electrodes on
 * the closed x-intervals [patch_x0[e], patch_x1[e]] (uniform in z: stripes along z in 3D) at
 * voltage patch_v[e], and dV/dn = 0 on the gaps.  A wall node is on electrode e when its x (or
 * x + the x-period) lies in the interval to 1e-9 of its length plus 1e-12.  The patch arrays are
 * host memory, read during pf_create only, and ignored for other kinds.  The patch solve is the
 * base solve with the whole wall Dirichlet plus a capacitance (Schur-complement) correction on
 * the gap nodes, per Fourier mode: two fast-diagonalisation solves per potential solve. */
typedef struct {
    int bottom_kind, top_kind;   /* PF_BC_DIRICHLET, PF_BC_NEUMANN, or PF_BC_PATCHES (wall)  */
    double v_bottom, v_top;      /* electrode voltages for Dirichlet sides                 */
    int n_patch;                 /* PF_BC_PATCHES: number of electrodes (>= 0)              */
    const double *patch_x0, *patch_x1, *patch_v;   /* PF_BC_PATCHES: n_patch each          */
} pf_vbc;

typedef struct {
    double dt;          /* time step                                                       */
    int bdf;            /* 1 or 2 (BDF order J of Sec. 3.1; J = 1 is used for step 1)      */
    int precision;      /* PF_FP64, PF_MIXED or PF_MIXED_SIMT                              */
    double S;           /* stabiliser; 0 -> eta^2 sqrt(4 gamma0 / (lambda gamma1 dt))      */
    double nu_m;        /* 0 -> max(mu1,mu2)/min(rho1,rho2)                                */
    double rho0;        /* 0 -> min(rho1,rho2)                                             */
    double eps0;        /* 0 -> max(eps1,eps2)                                             */
    int model;          /* PF_MODEL_FULL, or PF_MODEL_EQUILIBRIUM: the simpler system of     */
                        /* Sec. 2.4 (eq. 16 with eq. 15c, 15d, u = 0; only the V and phi     */
                        /* sub-steps run, P and u stay 0)                                    */
} pf_scheme;

#define PF_MODEL_FULL        0
#define PF_MODEL_EQUILIBRIUM 1

/* ---- host-only set-up helpers (no GPU needed) ------------------------------------------ */

/* GLL tables of order K (Sec. 3.2.1 element basis): nodes[K+1], weights[K+1] and the
 * differentiation matrix D[(K+1)*(K+1)], D[i*(K+1)+j] = l_j'(x_i).  Returns PF_EINVAL
 * for K < 1 or K > 31 or null pointers. */
int pf_gll(int K, double *nodes, double *weights, double *D);

/* GLL node coordinates of ne elements of order K with breakpoints br[ne+1] along one
 * direction (the unique nodes of Sec. 3.2.1): n = ne*K values when periodic != 0 (the
 * last node is the first one shifted by the period), else ne*K + 1. */
int pf_nodes_1d(int ne, const double *br, int K, int periodic, double *nodes);

/* Assembled 1D stiffness (dense n x n, row-major) and diagonal GLL mass (n) of
 * ne elements of order K with breakpoints br[ne+1]; periodic != 0 identifies the
 * last node with the first (n = ne*K), else n = ne*K + 1.  These are the 1D
 * factors of the tensor-product operators of eqs. 54-59. */
int pf_operators_1d(int ne, const double *br, int K, int periodic, double *Kmat, double *Mdiag);

/* Generalised eigenbasis of the 1D operator restricted to the free nodes:
 * Kmat s = lambda Mdiag s with s^T Mdiag s = 1 (fast-diagonalisation factor of the
 * constant matrices of the Remark after Algorithm 2).  dirichlet[n] flags removed
 * nodes.  Output S[n*n] row-major: column c is the c-th eigenvector (ascending
 * lambda), rows of Dirichlet nodes are zero and the last (#Dirichlet) columns are
 * zero padding with lam = 1.  Returns PF_EINVAL on bad sizes. */
int pf_fdm_1d(int n, const double *Kmat, const double *Mdiag, const unsigned char *dirichlet,
              double *S, double *lam);

/* ---- handle life cycle ------------------------------------------------------------------ */

/* Validate the descriptors, build the 1D tables and eigenbases (FP64), allocate
 * the device state, set phi^0 (host, [z][y][x], required) and u^0 (host, three
 * consecutive blocks ux,uy,uz, nullable -> 0), P^0 = 0, compute V^0 by the fixed
 * point of the Remark in Sec. 3.1 (FP64 on the device) and E^0.
 * cuda_stream: a cudaStream_t (NULL = legacy default stream).
 * Errors: PF_EINVAL (bad descriptor, including patch intervals that are not finite with
 * x0 <= x1, PF_BC_PATCHES on the top, or a potential with no Dirichlet node at all),
 * PF_ENOMEM, PF_ECUDA. *out is NULL on error. */
int pf_create(const pf_mesh *mesh, const pf_fluid *fluid, const pf_vbc *vbc,
              const pf_scheme *scheme, const double *phi0, const double *u0,
              void *cuda_stream, pf_handle **out);

/* Advance nsteps time steps (Algorithm 1 / 2).  The first step of a run uses
 * BDF1; later steps the scheme's order.  Asynchronous on the handle's stream
 * except when it returns an error found on the host.  nsteps >= 0. */
int pf_step(pf_handle *h, int nsteps);

/* Synchronise the handle's stream and check the state for non-finite values:
 * returns PF_EDIVERGED if any was found since creation.  Returns PF_ETIMEOUT (and clears the
 * condition) when a bounded device-side wait of the tensor-core transforms gave up since the
 * last pf_sync; the fields computed by those steps are then not valid. */
int pf_sync(pf_handle *h);

/* Copy fields to the host (synchronous).  mask: PF_FIELD_* bits; blocks of
 * n_x*n_y*Nz doubles in the order V, Ex, Ey, Ez, phi, psi, P, ux, uy, uz for
 * the bits set (PF_FIELD_OLD selects level n-1 of V, phi, P, u).  n = capacity of
 * host_out in doubles; PF_EINVAL if too small. */
int pf_get_fields(pf_handle *h, unsigned mask, double *host_out, size_t n);

/* Overwrite fields from host data, same layout as pf_get_fields (restart or warm
 * start).  Setting PHI without OLD also sets level n-1 of phi; after a set the
 * next step restarts the BDF history only if reset_history != 0. */
int pf_set_fields(pf_handle *h, unsigned mask, const double *host_in, size_t n, int reset_history);

/* Restart bookkeeping (Sec. 3.1: the BDF order J of a step is 1 for the first step of a run and
 * the scheme's order afterwards): set the handle's step count and time.  With both history levels
 * written by pf_set_fields (mask with and without PF_FIELD_OLD, reset_history = 0) and the step
 * count and time of the run that wrote them (pf_diagnostics out[3], out[2]), a fresh handle of the
 * same descriptors continues that run.  PF_EINVAL for nstep < 0 or a non-finite t. */
int pf_set_step(pf_handle *h, int nstep, double t);

/* FP64 diagnostics (synchronous): out[0] = int phi (phase mass), out[1] = max|u|,
 * out[2] = time t, out[3] = step count, out[4] = number of V^0 fixed-point
 * iterations, out[5] = 1 if a non-finite value was seen, out[6] = max|phi^n - phi^{n-1}| / dt
 * (the pseudo-time rate of the equilibrium model), out[7] = the discrete energy E(t) of eq. 14
 * at the current level: GLL quadrature of rho|u|^2/2 + lambda|grad phi|^2/2 +
 * lambda (phi^2-1)^2/(4 eta^2) + eps(phi)|E|^2/2 with element-local derivatives (d/dz spectral),
 * plus the wall energy sigma cos(theta_s) phi (phi^2-3)/4 integrated over the wall (its constant
 * dropped); FP64 arithmetic and accumulation whatever the precision of the state. */
int pf_diagnostics(pf_handle *h, double out[8]);

/* One fast-diagonalisation solve on a user right-hand side (synchronous):
 *   (K + (lambda + beta_k^2) M) x = M f,   beta_k = 2 pi mode / lz,
 * with homogeneous Dirichlet values on the Dirichlet sides of bcset
 * (PF_BCSET_*; for PF_BCSET_V the handle's potential sides).  rhs/out are host
 * arrays of n_x*n_y doubles ([y][x]) for mode 0 (and always in 2D) and two such
 * planes (real, imaginary) for 0 < mode <= Nz/2.  Runs in the handle's precision.
 * Errors: PF_EINVAL for a bad bcset or mode; PF_ETIMEOUT when a bounded device-side wait of the
 * tensor-core transforms gave up (the output is then not valid). */
int pf_solve_helmholtz(pf_handle *h, int bcset, int mode, double lambda,
                       const double *rhs, double *out);

/* Kernel classes of the per-class launch counters and timers (pf_profile_read). */
#define PF_KC_GEMM      0   /* fast-diagonalisation transforms (4 per solve batch)          */
#define PF_KC_FWD       1   /* direct stiffness summation + forward z FFT + combination     */
#define PF_KC_INV       2   /* inverse z FFT (+ d/dz, Dirichlet values)                     */
#define PF_KC_POTENTIAL 3   /* eq. 54a/74a right-hand side                                  */
#define PF_KC_CHEM      4   /* eq. 56/75 right-hand side                                    */
#define PF_KC_MOMENTUM  5   /* eq. 49, 58a/77a, 59a/78a right-hand sides                    */
#define PF_KC_UGRADP    6   /* new-pressure term of eq. 59a/78a                             */
#define PF_KC_EFIELD    7   /* eq. 55/78 projection                                         */
#define PF_KC_OTHER     8   /* phi right-hand side, wall-face transform, conversions        */
#define PF_KC_COUNT     9

/* Enable (1) or disable (0) per-class CUDA-event timing of the kernels this handle
 * launches (events bracket every launch on the handle's stream, so enabling it adds a
 * little host overhead).  Enabling resets the timers.  Launch counters always run. */
int pf_profile(pf_handle *h, int enable);

/* Read the counters (synchronous): ms[PF_KC_COUNT] = summed device time per class since
 * timing was enabled (0 when disabled), launches[PF_KC_COUNT] = kernels launched per
 * class since creation.  Either pointer may be NULL. */
int pf_profile_read(pf_handle *h, double *ms, long long *launches);

/* Transform variants of the fast-diagonalisation solves (Sec. 3.1 solves, Eq. 44/48/52), as
 * codes for pf_set_variant and pf_autotune:
 *   PF_GEMM_TC       3xTF32 tcgen05 tensor-core transforms: persistent warp-specialised kernel,
 *                    TMA-staged operands, FP32 sums of per-K-chunk TMEM accumulators (PF_MIXED
 *                    only; n_x a multiple of 4, for the 16-byte row pitch TMA needs)
 *   PF_GEMM_TC_HYBRID
 *                    the psi and phi solves (the Cahn-Hilliard pair of eq. 44, whose rounding drives the
 *                    phase field's error) on the cp.async 64x64 CUDA-core transforms; the potential,
 *                    pressure and velocity solves on the tensor cores with four 8-wide K slices per
 *                    TMEM accumulation group (1.6x faster, less accurate; PF_MIXED only)
 *   PF_GEMM_PLANE    the whole solve of a mode plane in one thread block, plane and eigenbases
 *                    in shared memory (FP32 precisions; n_x <= 128, n_y <= 128)
 *   PF_GEMM_SIMT32 / PF_GEMM_SIMT64 / PF_GEMM_SIMT32X64
 *                    CUDA-core transforms with 32x32, 64x64 or 32x64 output tiles, the next k
 *                    tile prefetched through registers
 *   PF_GEMM_PIPE64 / PF_GEMM_PIPE32 / PF_GEMM_PIPE32X64
 *                    the same tiles with a four-stage cp.async pipeline (three k tiles in flight)
 *   PF_GEMM_CLUSTER4 / PF_GEMM_CLUSTER2
 *                    the whole solve of a mode plane on a cluster of 4 / 2 thread blocks that
 *                    exchange the plane through distributed shared memory (FP32 precisions;
 *                    n_x <= 128, n_y <= 128)
 * All give the same result up to rounding order; in FP64 the CUDA-core variants sum in the same
 * order and agree bit for bit. */
#define PF_GEMM_TC 0
#define PF_GEMM_PLANE 1
#define PF_GEMM_SIMT32 32
#define PF_GEMM_SIMT64 64
#define PF_GEMM_SIMT32X64 2
#define PF_GEMM_PIPE64 3
#define PF_GEMM_PIPE32 4
#define PF_GEMM_PIPE32X64 5
#define PF_GEMM_CLUSTER4 6
#define PF_GEMM_CLUSTER2 7
#define PF_GEMM_TC_HYBRID 8

/* Autotuner of a single run: time `steps` steady steps with each transform variant available to
 * the run (PF_GEMM_*), keep the fastest, then (unless a whole-plane variant won) whether the y transforms
 * run fused (one pass, eigenbasis in shared memory), then (3D) the z-transform tile of 4, 8, 16
 * or 32 pencils per block.  Each candidate is timed as the run executes its steady steps: graph
 * replays when the run has its own stream, eager launches on the legacy stream.  The run advances
 * by 16 (steps + 2) steps.  choice (nullable) receives gemm + 1000 * tile + 100000 * fused_y with
 * gemm a PF_GEMM_* code, tile the pencils per z-transform block (0: size heuristic, always 0 in
 * 2D) and fused_y 1 when the y pair runs fused; ms_per_step (nullable) the best time. */
int pf_autotune(pf_handle *h, int steps, int *choice, double *ms_per_step);

/* Pin the transform variant without timing (to reproduce an autotuned choice or to compare
 * variants): gemm a PF_GEMM_* code, fuse_y 1 to run the y transform pair fused where it fits
 * (0 separately; ignored by the whole-plane variants), tile the pencils per z-transform block (4, 8, 16,
 * 32) or 0 for the size heuristic.  Synchronises the run's stream and drops its captured
 * graphs.  PF_EINVAL (nothing changed) when a value is outside these sets or the run cannot use
 * the variant (PF_GEMM_TC outside PF_MIXED, the whole-plane variants in FP64 or on a plane too
 * large). */
int pf_set_variant(pf_handle *h, int gemm, int fuse_y, int tile);

/* Accumulation of the 3xTF32 tensor-core transforms (the constant eigenbasis products of the
 * Remark after Algorithm 2) for variant gemm (PF_GEMM_TC or PF_GEMM_TC_HYBRID) and solve family
 * (0: the psi and phi solves of the split Cahn-Hilliard step, eq. 44, and with electrode patches
 * the potential solves, whose capacitance correction subtracts two solutions; 1: the other V, P
 * and u solves):
 * every `slices` 8-wide K slices (1..64) accumulate in a tensor-memory region of their own,
 * drained into FP32 registers with rounding to nearest; sep = 1 chains the two small correction
 * products of a whole output tile in a separate region (drained once per tile), so that a group's
 * region holds only the main products.  The tensor core truncates its FP32 sums: longer groups
 * run faster and lose more digits.  Defaults: PF_GEMM_TC 2 slices with sep for psi, phi and 8
 * with sep for the others; PF_GEMM_TC_HYBRID (psi, phi on CUDA cores) 4 without sep.  Applies
 * from the next step (captured graphs are dropped).  PF_EINVAL when h is not a PF_MIXED run or a
 * value is outside these sets. */
int pf_set_tc_accum(pf_handle *h, int gemm, int family, int slices, int sep);

/* Test hook of the failure detection (Sec. 3 has no counterpart): the next tensor-core transform
 * launch of h waits on a device barrier that nothing arrives at, gives up after wait_ns
 * nanoseconds (0 < wait_ns <= 1e10), records the time-out in the handle's error word and returns
 * without touching tensor memory; pf_sync (after pf_step) or pf_solve_helmholtz then return
 * PF_ETIMEOUT.  The next pf_step runs without its captured graph so that the hook applies.
 * PF_EINVAL when the handle does not use the tensor-core transforms. */
int pf_debug_tc_stall(pf_handle *h, unsigned long long wait_ns);

/* Geometry queries: nodes_x[n_x], nodes_y[n_y] (either may be NULL), sizes in dims[4]
 * = {n_x, n_y, Nz, number of real values per field}. */
int pf_geometry(const pf_handle *h, double *nodes_x, double *nodes_y, int dims[4]);

/* ---- ensembles of independent 2D runs ---------------------------------------------- */

/* Opaque ensemble: nrun independent 2D runs (nz = 1 meshes) advanced together.  Runs that
 * share the mesh (breakpoints, order), the fluid constants other than eps1/eps2, the kinds of
 * the potential sides and the scheme are grouped; each group's runs are the planes of one
 * engine (per-run permittivities and electrode voltages), and one CUDA graph replays a time
 * step of every group. */
typedef struct pf_batch pf_batch;

/* meshes/fluids/vbcs: nrun descriptors each (nz must be 1); scheme shared by all runs;
 * phi0[r]: host array of run r's n_x*n_y initial phase field.  Each group computes its
 * initial potentials by the fixed point of the Remark in Sec. 3.1 (FP64).  Errors: PF_EINVAL
 * (message in pf_last_error(NULL)), PF_ENOMEM, PF_ECUDA. */
int pf_batch_create(int nrun, const pf_mesh *meshes, const pf_fluid *fluids, const pf_vbc *vbcs,
                    const pf_scheme *scheme, const double *const *phi0, void *cuda_stream, pf_batch **out);

/* Advance every run nsteps time steps (Algorithm 1; BDF1 for the first step). */
int pf_batch_step(pf_batch *b, int nsteps);

/* Per-run FP64 max |u| (out[nrun]) and phase mass int phi (mass[nrun], nullable); synchronous.
 * For PF_MODEL_EQUILIBRIUM (u = 0) umax[r] is the pseudo-time rate max|phi^n - phi^{n-1}| / dt,
 * so pf_batch_run_to_equilibrium stops on it. */
int pf_batch_umax(pf_batch *b, double *umax, double *mass);

/* Step until every run has max|u| < tol, checking every check_every steps, or until the
 * ensemble has taken max_steps steps.  steps_out[r] = the step count at which run r was first
 * seen below tol, -1 if it never was, or -2 if its velocity became non-finite (runs are
 * independent: a diverged run does not affect the others, which keep stepping). */
int pf_batch_run_to_equilibrium(pf_batch *b, double tol, int max_steps, int check_every, int *steps_out);

/* Copy run r's fields to the host; mask and layout as pf_get_fields for one 2D run. */
int pf_batch_get_fields(pf_batch *b, int run, unsigned mask, double *host_out, size_t n);

/* Autotuner: for every group, time `steps` steps with each transform variant (tensor cores
 * where the precision has them, SIMT with 32x32 and 64x64 tiles, the whole-plane solves on one
 * block or a cluster where they fit) and keep the fastest.  It advances the ensemble by
 * 6 (steps + 1) steps (rounded up to even).  ms_out[g] (nullable, capacity >= number of groups) receives the best time per step of
 * group g; returns the number of groups (>= 0) or an error code. */
int pf_batch_autotune(pf_batch *b, int steps, double *ms_out);

/* Pin the transform variant of every group (codes as pf_set_variant); PF_EINVAL, nothing
 * changed, when some group cannot use it. */
int pf_batch_set_variant(pf_batch *b, int gemm, int fuse_y);

/* Message of the ensemble's last failed call (empty if none; pf_last_error(NULL)'s message for
 * b == NULL).  The string is owned by the ensemble and valid until its next call. */
const char *pf_batch_last_error(const pf_batch *b);

/* Number of groups and, per run, its group (group_of[nrun], nullable). */
int pf_batch_groups(const pf_batch *b, int *group_of);

void pf_batch_destroy(pf_batch *b);

/* ---- learned warm start --------------------------------------------------------------- */

/* A small neural operator (the paper has no counterpart): a tanh multilayer perceptron with
 * layer widths dims[0..nlayer-1] maps dims[0] run parameters (standardised with feat_mean /
 * feat_std) to the phase field on a gnx x gny grid (dims[nlayer-1] = gnx*gny; x periodic
 * on [x0, x1) with cells starting at x0 + i (x1-x0)/gnx, y from y0 to y1 inclusive), which a
 * fixed bilinear map carries to the nqx x nqy nodes (node_x[nqx], node_y[nqy]; [y][x] order).
 * Weights are BF16 in the products (FP32 master copies), activations and sums FP32; Glorot
 * initialisation from seed.  The forward products of hidden and output layers whose input width
 * is a multiple of 64 up to 384 and whose output width is a multiple of 128 run on the tensor
 * cores (tcgen05.mma kind::f16: the BF16 weights times the inputs split into BF16 head and tail,
 * FP32 accumulation); the first layer and the backward products run on the CUDA cores.  All work
 * runs on cuda_stream.  Errors: PF_EINVAL, PF_ENOMEM, PF_ECUDA, PF_ETIMEOUT when a tensor-core
 * layer's bounded wait gave up (messages in pf_last_error(NULL)). */
typedef struct pf_no pf_no;
int pf_no_create(int nlayer, const int *dims, const double *feat_mean, const double *feat_std, int gnx, int gny,
                 double x0, double x1, double y0, double y1, int nqx, int nqy, const double *node_x,
                 const double *node_y, uint64_t seed, void *cuda_stream, pf_no **out);
/* Number of parameters: for each layer its weights (dims[l] x dims[l+1], row-major) then
 * its biases, layer after layer. */
long long pf_no_param_count(const pf_no *h);
/* FP32 master parameters to / from host doubles (n >= pf_no_param_count). */
int pf_no_get_params(pf_no *h, double *host, size_t n);
int pf_no_set_params(pf_no *h, const double *host, size_t n);
/* Phase field at the nodes (B x nq, host) for B feature rows (B x dims[0], host). */
int pf_no_predict(pf_no *h, int B, const double *feat, double *phi_nodes);
/* As pf_no_predict, then each sample's field is shifted by a constant so that its phase mass
 * sum_ij wx[j] wy[i] phi_ij equals mass[b] (FP64 sums on the device): the equilibrium system of
 * Sec. 2.4 conserves int phi, so a warm start carries the run's own mass.  wx[nqx], wy[nqy] are
 * the quadrature weights of the node grid (the assembled 1D GLL masses), mass[B] the targets. */
int pf_no_predict_mass(pf_no *h, int B, const double *feat, const double *mass, const double *wx,
                       const double *wy, double *phi_nodes);
/* Mean squared error against target node fields (B x nq) and the gradient of every
 * parameter (grad nullable; layout of pf_no_get_params). */
int pf_no_loss_grad(pf_no *h, int B, const double *feat, const double *target, double *loss, double *grad);
/* Adam training (beta 0.9 / 0.999, eps 1e-8) on nsample rows resident on the device for
 * `epochs` epochs of shuffled minibatches of `batch` rows; loss_per_epoch[epochs] nullable. */
int pf_no_train(pf_no *h, int nsample, const double *feat, const double *target, int batch, int epochs,
                double lr, uint64_t seed, double *loss_per_epoch);
void pf_no_destroy(pf_no *h);

/* ---- allocation-free solve ---------------------------------------------------------- */

/* Capacity, in doubles, of each of the two scratch buffers of pf_fdm_solve_static. */
#define PF_STATIC_MAX_VALUES (1 << 20)

/* A fast-diagonalisation solve that allocates nothing, for callers that cannot call
 * cudaMalloc where they need it (inside a region where allocation is forbidden or would
 * synchronise the device, a memory-planned real-time loop, a host library that brings its
 * own allocator).  The paper has no counterpart: it is a packaging of the solve above.
 *
 * For each of nplanes planes p ([p][y][x], x fastest, device memory) it computes
 *   out[p] = Sy [ (Sy^T rhs[p] Sx) / (lam_y[i] + lam_x[j] + shift[p]) ] Sx^T
 * in FP64, i.e. the solution of (K + shift[p] M) x = rhs[p] when rhs[p] is the weak-form
 * (mass-weighted) right-hand side and Sx, Sy, lam_x, lam_y are the factors returned by
 * pf_fdm_1d (SxT, SyT their transposes, row-major; a zero denominator gives 0).
 * Every pointer is a caller-owned device pointer; the call is asynchronous on cuda_stream.
 *
 * Its two intermediate buffers live in one file-scope device array of
 * 2 * PF_STATIC_MAX_VALUES doubles (16 MiB) that every GPU loading this library holds
 * until exit.  nx*ny*nplanes > PF_STATIC_MAX_VALUES returns PF_EINVAL (message in
 * pf_last_error(NULL)).  The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current and keeps it for the life of the process;
 * make that first call before any stream capture.  Resetting the device (cudaDeviceReset) or
 * calling from another context on that device after the first call is not supported: the kept
 * address would belong to the old context.  Every call shares the array, so calls that overlap
 * on the GPU (other streams, other threads) race; each call fully overwrites the buffers before
 * reading them. */
int pf_fdm_solve_static(int nx, int ny, int nplanes, const double *Sx, const double *SxT,
                        const double *lam_x, const double *Sy, const double *SyT, const double *lam_y,
                        const double *shift, const double *rhs, double *out, void *cuda_stream);

/* ---- measured peaks ------------------------------------------------------------------- */

/* Compute peaks of the current device, measured by microbenchmark kernels (the paper has no
 * counterpart; these are the denominators of the benchmark's roofline fractions), in TFLOP/s:
 * out[0] = TF32 tensor cores (tcgen05.mma kind::tf32, M = 128, N = 256, K = 8, one CTA per SM),
 * out[1] = FP32 FFMA on the CUDA cores, out[2] = FP64 DFMA.  Best of five timed launches each;
 * synchronous, takes a few milliseconds.  PF_ECUDA without a device, PF_ETIMEOUT if the tensor-core
 * loop's bounded wait gave up (messages in pf_last_error(NULL)). */
int pf_measure_peaks(double out[3]);

/* Release all device memory of the handle (NULL is a no-op). */
void pf_destroy(pf_handle *h);

/* Last error message of the handle, or of the last failed pf_create when h is NULL. */
const char *pf_last_error(const pf_handle *h);

#ifdef __cplusplus
}
#endif

#endif /* PF_H */
