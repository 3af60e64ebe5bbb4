/*
 * hmg -- FFT-based (Eyre-Milton accelerated) thermal homogenization of coated-sphere
 * composites on one NVIDIA GB300.  C ABI of libhmg.so.
 *
 * The method is that of Lemaitre, Salnikov, Choi & Karamian, "Computation of thermal
 * properties via 3D homogenization of multiphase materials using FFT-based
 * accelerated scheme" (arXiv:1504.07499):
 *   - §2 / Fig. 1: identical non-overlapping spheres (centre, outer radius r_s), each
 *     with a coating of width l * r_s (0 < l < 1); three phases: matrix (0),
 *     inclusion core (1), coating shell (2); isotropic conductivities k I (§2, §5).
 *   - §3, eq. 1-3: periodic cell problem in polarization form with a constant
 *     reference medium L0 = -k0 I, k0 = sqrt(min k * max k) (§5), and the Green
 *     operator Gamma0(xi) = xi xi^T / (xi . L0 xi), Gamma0(0) = 0.
 *   - §3 Algorithm, steps 1-7: the accelerated iteration and its two-stage
 *     convergence test (eps_comp, then eps_eq).
 *   - §3 last paragraph: <phi> = -L_hom grad Theta gives the 3x3 effective tensor.
 *
 * Conventions shared by every call
 *   - Grids are N x N x N voxels stored z-major, x fastest: index (z*N + y)*N + x.
 *     N must be even, N = 2 * 2^a * 3^b, 8 <= N <= 512.
 *   - Phase ids: 0 matrix, 1 inclusion, 2 coating (uint8 per voxel).
 *   - Vector fields hold components x, y, z as three consecutive N^3 blocks.
 *   - A pointer argument may be host memory or device memory of the context's GPU;
 *     the library detects which and copies as needed.  All buffers are owned by the
 *     caller and are only read (inputs) or written (outputs) during the call.
 *   - Every call returns an hmg_status; nothing aborts, throws or traps.  On error
 *     hmg_last_error() describes the failure (thread-local, valid until the next call).
 *   - A context is not thread-safe: serialize calls on one context.
 *   - Wavevectors are xi_j = 2 pi m_j / N with m_j in (-N/2, N/2].  Nyquist components
 *     (m_j = N/2) are dropped from xi except in a mode whose only nonzero component is
 *     a Nyquist one; Gamma0 is zero where the resulting xi is zero.
 */
#ifndef HMG_H
#define HMG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hmg_ctx hmg_ctx;

/* One coated sphere (§2): centre in the periodic unit cube, r = OUTER radius r_s. */
typedef struct {
    double cx, cy, cz, r;
} hmg_sphere;

/* One coated cylinder (§6 outlook: RVEs with cylinders, or spheres and cylinders):
 * centre in the periodic unit cube, unit axis (ux, uy, uz), OUTER radius r and OUTER
 * length h (coating included).  The coating has the same thickness l r on the lateral
 * surface and on the flat ends: the core has radius (1 - l) r and length h - 2 l r.
 * A cylinder of length at least 1 + 2 l r along a grid axis is a continuous fiber. */
typedef struct {
    double cx, cy, cz, ux, uy, uz, r, h;
} hmg_cylinder;

typedef enum {
    HMG_OK = 0,
    HMG_PENDING = 1,          /* hmg_poll: request not finished yet */
    HMG_INVALID_ARG = -1,     /* bad size, value or pointer; nothing was launched */
    HMG_OUT_OF_MEMORY = -2,   /* device allocation failed or the HBM budget is exceeded */
    HMG_NOT_CONVERGED = -3,   /* max_iter reached; outputs hold the last iterate's values */
    HMG_DIVERGED = -4,        /* a residual became NaN or Inf */
    HMG_CUDA_ERROR = -5,      /* a CUDA runtime call failed; see hmg_last_error() */
    HMG_BUSY = -6,            /* hmg_submit: queue full */
    HMG_UNKNOWN_TICKET = -7   /* hmg_poll: no such request (or already collected) */
} hmg_status;

/* Arithmetic of the solve.
 * HMG_FP64: every step in FP64 (the plain method of §3).
 * HMG_FP32_BULK: FFTs and pointwise updates in FP32; residual norms, the convergence
 *   tests, the flux average and a few defect-correction sweeps in FP64, so that the
 *   same tolerance as HMG_FP64 is met (eps_eq < tol computed in FP64). */
typedef enum { HMG_FP64 = 0, HMG_FP32_BULK = 1 } hmg_precision;

/* Iterative scheme for the periodic cell problem (§3 lists the FFT-based schemes and
 * picks the accelerated one).
 *   HMG_SCHEME_EYRE_MILTON: the accelerated scheme of the §3 Algorithm (steps 1-7),
 *     reference k0 = sqrt(min k * max k) (§5); contraction (sqrt c - 1)/(sqrt c + 1)
 *     per sweep for contrast c = max k / min k.
 *   HMG_SCHEME_BASIC: the basic scheme, the plain fixed-point iteration of the
 *     Lippmann-Schwinger equation of §3 (eqs. 1-3), e^{n+1} = E - Gamma0 * ((k - k0) e^n)
 *     with a positive reference k0 = (min k + max k) / 2 and Gamma0 = P / k0
 *     (P = xi xi^T / |xi|^2); contraction (c - 1)/(c + 1) per sweep.  Steps 1 and 6
 *     (the two convergence tests) are those of the §3 Algorithm; its new iterate is the
 *     compatible field of step 5.
 *   HMG_SCHEME_AUGMENTED_LAGRANGIAN: the augmented Lagrangian scheme (Michel, Moulinec
 *     & Suquet 2001, cited in §5 for the choice of k0): alternate minimization of the
 *     Lagrangian <d.k d>/2 + <lambda.(e - d)> + k0 <|e - d|^2>/2 over a compatible field e
 *     (mean grad Theta) and a free field d, then the multiplier update
 *     lambda += k0 (e - d), with k0 = sqrt(min k * max k).  Its iterate d (and flux
 *     lambda = k d) moves half the Eyre-Milton step: step 7 with the factor 1 in place
 *     of 2, contraction (1 + rho)/2 per sweep with rho = (sqrt c - 1)/(sqrt c + 1), so it
 *     needs about twice the sweeps but also converges when rho -> 1 (infinite contrast).
 *     Steps 1 and 6 test its iterate d (eps_comp = |d - e|, eps_eq on lambda = k d).
 * All converge to the same discrete solution (the fixed point of each is the
 * compatible field with divergence-free flux), so K agrees to the tolerance. */
typedef enum {
    HMG_SCHEME_EYRE_MILTON = 0,
    HMG_SCHEME_BASIC = 1,
    HMG_SCHEME_AUGMENTED_LAGRANGIAN = 2
} hmg_scheme;

/* Per-solve report.  Index j is the macroscopic gradient e_j. */
typedef struct {
    int iters[3];          /* sweeps of steps 2-7 (FP32 and FP64 together) */
    int iters_fp64[3];     /* of which in FP64 */
    double eps_comp[3];    /* last compatibility residual (§3 step 6) */
    double eps_eq[3];      /* last equilibrium residual (§3 step 1) */
    double seconds;        /* wall time of the call */
    int fp64_rounds;       /* FP64 defect-correction rounds (HMG_FP32_BULK) */
    int status[3];         /* hmg_status per gradient */
} hmg_info;

/* Library version string (static storage). */
const char* hmg_version(void);

/* Thread-local description of the last failure in this thread ("" if none). */
const char* hmg_last_error(void);

/* Create a context on CUDA device `device`.  `hbm_budget_bytes` caps the device
 * memory the context may hold for solve state (0 = 90 % of the free memory at
 * creation).  *ctx receives the handle; destroy it with hmg_destroy. */
hmg_status hmg_create(hmg_ctx** ctx, int device, size_t hbm_budget_bytes);

/* Release every resource of the context (waits for in-flight work). */
hmg_status hmg_destroy(hmg_ctx* ctx);

/* Voxelize coated spheres into a three-phase grid (§2, Fig. 1).
 * spheres: n entries (host or device).  layer: l in (0, 1), core radius (1-l) r_s.
 * phase_out: N^3 bytes (host or device), written with 0/1/2.
 * Rule (bit-exact, integer): coordinates are quantized to S = 2 N 4096 units; voxel
 * (i,j,k) has centre ((2i+1) 4096, ...); a centre c maps to floor(c' S + 1/2) mod S
 * with c' = c - floor(c); squared radii are floor((r S)^2 + 1/2) and
 * floor(((1-l) r S)^2 + 1/2); distances are periodic minimum-image; a voxel is
 * inclusion if inside any core, else coating if inside any sphere, else matrix
 * (boundaries inclusive).
 * Errors: HMG_INVALID_ARG for n = 0 or n > 100000, non-finite values, r <= 0 or
 * r >= 0.5, layer outside (0,1), a bad N, or overlapping spheres (§2: the spheres
 * do not overlap). */
hmg_status hmg_voxelize(hmg_ctx* ctx, const hmg_sphere* spheres, size_t n, double layer,
                        int N, uint8_t* phase_out);

/* hmg_voxelize for coated spheres and coated cylinders together (§6 outlook).  The
 * spheres follow the rule of hmg_voxelize; the cylinders the integer rule: coordinates in
 * units of 1 / (2 N 256) (voxel centres at odd multiples of 256), a centre c mapped as a
 * sphere's, the axis to A = floor(1024 u + 1/2) per component, squared radii
 * floor((r S)^2 + 1/2) and floor(((1-l) r S)^2 + 1/2), half-lengths floor((h/2) S + 1/2) and
 * floor((h/2 - l r) S + 1/2) (S = 2 N 256); with d the signed minimum-image offset of a
 * voxel centre from the centre (components in [-S/2, S/2)) and t = d . A, the voxel lies in
 * the cylinder when |d|^2 |A|^2 - t^2 <= R^2 |A|^2 and t^2 <= H^2 |A|^2 (int64).  A voxel is
 * inclusion inside any core (sphere or cylinder), else coating inside any outer shape, else
 * matrix.  Either count may be 0 (not both); spheres and cylinders: host or device.
 * Overlaps are checked between spheres only (the generator keeps cylinders apart).
 * Errors: HMG_INVALID_ARG as hmg_voxelize, and for a cylinder with a non-finite value,
 * r outside (0, 0.5), h outside (0, 2] or an axis of length other than 1. */
hmg_status hmg_voxelize_mixed(hmg_ctx* ctx, const hmg_sphere* spheres, size_t n_spheres,
                              const hmg_cylinder* cylinders, size_t n_cylinders, double layer, int N,
                              uint8_t* phase_out);

/* Seeded placement of n identical, non-overlapping spheres of outer radius r in the
 * periodic unit cube, computed on the GPU (§2: the RVEs come from random sequential
 * adsorption, up to 100 spheres and 40 % volume fraction).  For n spheres filling a
 * volume fraction f (coating included), r = (3 f / (4 pi n))^(1/3).
 * Steps: RSA at radius r (candidates uniform in the cube, accepted in draw order when
 * farther than 2r from every accepted centre, periodic minimum image); if it cannot
 * place n spheres (RSA jams near 38 %), RSA at 0.85 r followed by Monte-Carlo
 * displacement sweeps that grow the radius back to r.  Random numbers come from the
 * counter-based SplitMix64 stream of `seed` (streams 0, 2 and 1 for the three steps);
 * every squared distance is (dx^2 + dy^2) + dz^2 with each operation rounded on its own,
 * so the result is reproducible bit for bit on any machine.
 * max_candidates: RSA candidate cap (drawn in blocks of 8192, so up to the next multiple).
 * spheres_out: n entries (host or device), radius r.  generator: NULL, or 0 (RSA) /
 * 1 (reduced-radius RSA + growth sweeps).  Every loop is bounded (candidate cap, 20000
 * growth sweeps).
 * Errors: HMG_INVALID_ARG for n outside 1..1024, r outside (0, 0.5) or a cap below 1;
 * HMG_NOT_CONVERGED when neither step places the spheres (nothing is written). */
hmg_status hmg_rsa(hmg_ctx* ctx, uint64_t seed, int n, double r, long long max_candidates,
                   hmg_sphere* spheres_out, int* generator);

/* The RVE of §2 as a phase grid: hmg_rsa followed by hmg_voxelize with layer l.
 * phase_out: N^3 bytes (host or device); spheres_out: NULL or n entries (host or
 * device).  Errors as hmg_rsa and hmg_voxelize. */
hmg_status hmg_rve(hmg_ctx* ctx, uint64_t seed, int n, double r, long long max_candidates, double layer,
                   int N, uint8_t* phase_out, hmg_sphere* spheres_out, int* generator);

/* Effective conductivity tensor of a three-phase grid (§3 Algorithm, steps 1-7, run
 * for the three unit gradients; §3 last paragraph for L_hom).
 * phase: N^3 bytes (host or device).  k_*: phase conductivities (> 0).
 * tol: the convergence criterion acc of §3, used for both eps_comp and eps_eq.
 * max_iter: cap on sweeps per gradient (<= 0 selects 20000).
 * K_out: 9 doubles (host), row-major, K_out[3*i + j] = <k e_i> for gradient e_j,
 *   i.e. L_hom with <phi> = -L_hom grad Theta (not symmetrized).
 * info: optional (may be NULL).
 * Returns HMG_OK when all three gradients converged, else the first failure. */
hmg_status hmg_solve(hmg_ctx* ctx, const uint8_t* phase, int N, double k_matrix,
                     double k_incl, double k_coat, double tol, hmg_precision precision,
                     int max_iter, double K_out[9], hmg_info* info);

/* hmg_solve that also returns the converged gradient fields.
 * e_out: NULL or 9 N^3 doubles (host or device): gradient j's field, components
 * x, y, z, at offset 3 j N^3.  Other arguments as hmg_solve. */
hmg_status hmg_solve_fields(hmg_ctx* ctx, const uint8_t* phase, int N, double k_matrix,
                            double k_incl, double k_coat, double tol,
                            hmg_precision precision, int max_iter, double K_out[9],
                            hmg_info* info, double* e_out);

/* hmg_solve_fields with a choice of iterative scheme (hmg_scheme, above).  The plain
 * FP64 form and the FP32-bulk form (FP32 sweeps with FP64 defect correction) are
 * available for both schemes; HMG_SCHEME_EYRE_MILTON is exactly hmg_solve_fields.
 * The basic scheme needs about ln(1/tol) (c + 1) / 2 sweeps per gradient at contrast c
 * (18 500 at c = 2000, tol 1e-8): raise max_iter above its default of 20000 for
 * contrasts beyond ~2000.
 * The augmented Lagrangian scheme needs about twice the sweeps of the accelerated one.
 * Errors: HMG_INVALID_ARG for an unknown scheme, otherwise as hmg_solve. */
hmg_status hmg_solve_scheme(hmg_ctx* ctx, const uint8_t* phase, int N, double k_matrix,
                            double k_incl, double k_coat, double tol,
                            hmg_precision precision, hmg_scheme scheme, int max_iter,
                            double K_out[9], hmg_info* info, double* e_out);

/* The polarization scheme named in §3 (beside the basic, dual, augmented Lagrangian and
 * accelerated schemes; the paper prints no formula).  Read here as the relaxed
 * iteration on the polarization tau = (k + k0) e with relaxation beta,
 *   tau^{n+1} = (1 - beta/2) tau^n + (beta/2) [(I - 2P)(Y tau^n) + 2 k0 E],
 * i.e. step 7 of the §3 Algorithm with the factor beta in place of 2:
 * e^{n+1} = e^n + beta k0 / (k + k0) (e_comp - e^n).  beta = 2 is the accelerated
 * (Eyre-Milton) scheme, beta = 1 the augmented Lagrangian scheme; every beta in (0, 2]
 * has the same fixed point and contracts by 1 - beta (1 - rho) / 2 per sweep.
 * Errors: HMG_INVALID_ARG for beta outside (0, 2], otherwise as hmg_solve_scheme. */
hmg_status hmg_solve_polarization(hmg_ctx* ctx, const uint8_t* phase, int N, double k_matrix,
                                  double k_incl, double k_coat, double tol,
                                  hmg_precision precision, double beta, int max_iter,
                                  double K_out[9], hmg_info* info, double* e_out);

/* Run `n_iter` sweeps of steps 2-7 of §3 (no convergence test) on a given gradient
 * field, for one macroscopic gradient grad_Theta (3 doubles, host).
 * e_inout: 3 N^3 doubles (host or device), the current iterate e^n on entry and
 * e^{n + n_iter} on return.  eps_comp_out: NULL or n_iter doubles (host), the
 * step-6 residual of each sweep.  precision selects FP64 or FP32 arithmetic for
 * the sweeps (the field is rounded to FP32 on entry in that case). */
hmg_status hmg_em_iterate(hmg_ctx* ctx, const uint8_t* phase, int N, double k_matrix,
                          double k_incl, double k_coat, const double grad_Theta[3],
                          hmg_precision precision, int n_iter, double* e_inout,
                          double* eps_comp_out);

/* Equilibrium residual of step 1 of §3 for a gradient field e (3 N^3 doubles, host
 * or device): phi = -k e, phi_hat = DFT(phi)/N^3,
 * eps_eq = sqrt(sum_{xi != 0} |xi . phi_hat|^2) / |phi_hat(0)|.
 * eps_eq_out: 1 double (host).  flux_mean_out: NULL or 3 doubles (host), <k e>
 * (minus the mean flux of §3).  Arithmetic in FP64 or FP32 (accumulation in FP64). */
hmg_status hmg_equilibrium(hmg_ctx* ctx, const uint8_t* phase, int N, double k_matrix,
                           double k_incl, double k_coat, hmg_precision precision,
                           const double* e, double* eps_eq_out, double* flux_mean_out);

/* Unnormalized forward 3D DFT (§3 step 3) of `count` real N^3 grids.
 * x: count N^3 doubles (host or device).
 * X_out: count * N^3 complex values as interleaved (re, im) doubles (host or
 * device), N*N*(N/2) complex per grid, index (kz*N + ky)*(N/2) + kx, kx in [0, N/2).
 * For kx > 0 the entry is the DFT coefficient X(kx, ky, kz).  The kx = 0 entry packs
 * two planes: Z = A + i B with A(ky,kz) = X(0, ky, kz) and B(ky,kz) = X(N/2, ky, kz);
 * A = (Z(k) + conj Z(-k))/2 and B = (Z(k) - conj Z(-k))/(2i) recover them. */
hmg_status hmg_fft_forward(hmg_ctx* ctx, int N, int count, hmg_precision precision,
                           const double* x, double* X_out);

/* Unnormalized inverse of hmg_fft_forward (kernel exp(+2 pi i k.n/N), no 1/N^3):
 * X: packed spectra as produced by hmg_fft_forward; x_out: count N^3 doubles. */
hmg_status hmg_fft_inverse(hmg_ctx* ctx, int N, int count, hmg_precision precision,
                           const double* X, double* x_out);

/* Largest N accepted by hmg_equilibrium_noalloc. */
#define HMG_NOALLOC_MAX_N 64

/* hmg_equilibrium for callers that cannot allocate device memory.  The paper has no
 * counterpart; this entry point exists for hosts that own all device memory through
 * their own pool, or that must not risk an allocation failure or the implicit device
 * synchronization of cudaMalloc/cudaFree in the middle of a run.  It needs no context
 * and calls no cudaMalloc, cudaFree or allocating library routine: its scratch (about
 * 13 MB: the field, the packed spectrum, partial sums and the twiddle table of one
 * N <= HMG_NOALLOC_MAX_N grid) is a set of static device arrays that every GPU which
 * loads libhmg holds until the process exits (the CUDA driver maps them in with the
 * library's code, not this call).
 * Same arithmetic as hmg_equilibrium with precision HMG_FP64: phase (N^3 bytes) and e
 * (3 N^3 doubles) may be host or device pointers of the current device;
 * eps_eq_out (1 double) and flux_mean_out (NULL or 3 doubles, <k e>) are host memory.
 * Work runs on the current device's legacy default stream and the call returns when
 * it has finished.  Every call looks up the arrays' device addresses in the current
 * context (cudaGetSymbolAddress) and rewrites the twiddle table and the sums it
 * uses, so it also works after cudaDeviceReset.  All calls share the arrays, which
 * keep the last call's contents: two calls overlapping on the GPU would race, so the
 * library serializes them (a lock held until the call's GPU work has finished).  Work
 * the caller runs on other streams is not ordered against this call (the legacy
 * default stream does not wait for non-blocking streams): finish writing phase and e
 * before the call.
 * Errors: HMG_INVALID_ARG for N > HMG_NOALLOC_MAX_N (or any argument hmg_equilibrium
 * rejects), HMG_CUDA_ERROR if a CUDA call fails. */
hmg_status hmg_equilibrium_noalloc(const uint8_t* phase, int N, double k_matrix,
                                   double k_incl, double k_coat, const double* e,
                                   double* eps_eq_out, double* flux_mean_out);

/* ---- many RVEs: batched solves and the request loop ------------------------- */

/* Solve `count` RVEs (possibly of different N) together: each batched sweep
 * advances every unfinished RVE and gradient in one launch per FFT pass.
 * phases[i]: N_list[i]^3 bytes (host or device).  k3: 3 count doubles
 * (k_matrix, k_incl, k_coat per RVE).  K_out: 9 count doubles (host).
 * info: NULL or count entries.  Other arguments as hmg_solve. */
hmg_status hmg_solve_batch(hmg_ctx* ctx, int count, const uint8_t* const* phases,
                           const int* N_list, const double* k3, double tol,
                           hmg_precision precision, int max_iter, double* K_out,
                           hmg_info* info);

/* Queue one solve request (copies the phase grid; returns without waiting for the
 * GPU).  A worker thread with its own CUDA stream runs the request loop: between
 * engine ticks it retires finished requests (freeing their device state) and admits
 * queued ones while their footprint (hmg_footprint) fits the context's budget; every
 * tick advances all admitted HMG_FP32_BULK requests of a lane together in one
 * CUDA-graph launch (continuous batching).  HMG_FP64 requests run one at a time.
 * Grids of 192^3 voxels and more and smaller grids run in two lanes (each a worker
 * thread with its own streams and engine), so small requests do not wait for the ticks
 * of large ones and the kernels of both lanes share the GPU; the large lane runs its
 * requests one at a time in arrival order, the small lane up to 64 at once.
 * The loop and the caller's context share one budget: the first hmg_submit on a
 * context releases the context's own solve state, and device memory that later calls
 * on the context hold counts against the loop's admissions (a request that cannot get
 * its state waits in the queue while other requests or the caller hold memory, and
 * finishes with HMG_OUT_OF_MEMORY after about 10 s of waiting).  The first hmg_submit
 * starts the loop; concurrent first calls start one loop.
 * *ticket identifies the request.
 * Returns HMG_BUSY when the queue is full, HMG_INVALID_ARG for bad arguments, and
 * HMG_OUT_OF_MEMORY when the request alone exceeds the budget. */
hmg_status hmg_submit(hmg_ctx* ctx, const uint8_t* phase, int N, double k_matrix,
                      double k_incl, double k_coat, double tol, hmg_precision precision,
                      uint64_t* ticket);

/* hmg_submit for an RVE that the request loop generates on the device when it admits
 * the request: placement as hmg_rsa (seed, n spheres of outer radius r, candidate cap
 * 400000), voxelization with layer l on an N^3 grid, then the solve -- no phase grid
 * crosses the host.  A placement that fails finishes the request with its status
 * (HMG_NOT_CONVERGED).  Errors as hmg_submit and hmg_rsa. */
hmg_status hmg_submit_rve(hmg_ctx* ctx, uint64_t seed, int n, double r, double layer, int N,
                          double k_matrix, double k_incl, double k_coat, double tol,
                          hmg_precision precision, uint64_t* ticket);

/* Result of a submitted request: HMG_PENDING while queued or running; otherwise the
 * request's final status with K_out (9 doubles, host) and info (nullable) filled in.
 * A finished ticket is released by the call that returns its result. */
hmg_status hmg_poll(hmg_ctx* ctx, uint64_t ticket, double K_out[9], hmg_info* info);

/* ---- kernel variants (autotuning) --------------------------------------------- */

/* The FP32 path has kernel variants for grid sizes 64, 96, 128, 192 and 256, chosen by
 * timing on the device at the first FP32 solve of a size and kept per context:
 *   bit 0: z pass -- 0: one thread holds the three components of its modes; 1: one
 *          thread group per component, projections summed through shared memory;
 *   bit 1: x and y passes (sizes 128, 192, 256) -- 0: separate passes; 1: one
 *          thread-block-cluster kernel per direction (distributed shared memory);
 *   bit 2: with separate passes, the sweeps of a block of FP32 sweeps are chained
 *          (0, the default: the x inverse of one sweep and the x forward of the next
 *          are one kernel and the field is stored only before the residual sweep) or
 *          not (1).  Chained and unchained sweeps give bit-identical results.
 *   bit 3: with chained sweeps, the x round trip runs as one launch per CTA of each
 *          row block (0) or as a persistent kernel (1) whose CTAs stage the spectrum
 *          and phase rows of their next row block in shared memory with bulk copies
 *          while they transform the current one (bit-identical results).
 *   bit 4: with bit 0 clear, the z pass of plain and correction sweeps runs as a
 *          persistent kernel whose CTAs stage the next column block (three tiled tensor
 *          copies) in shared memory while they transform the current one (sizes up to
 *          256; bit-identical results).
 *   bit 5: with chained sweeps (sizes 64, 128, 192, 256), the y inverse of one sweep, the
 *          x round trip and the y forward of the next sweep run as one persistent kernel
 *          whose CTAs take whole (component, z) planes, so that each plane stays in L2
 *          between the three passes (bit-identical results; bit 3 then has no effect).
 * The autotuner chooses bits 0, 1, 3 and 4 and leaves bits 2 and 5 clear (the plane kernel
 * times faster alone than the passes it replaces but is even with them inside a solve).
 * hmg_set_variant pins
 * `variant` (0 .. 63) for size N, or clears the choice (-1) so that the next solve
 * times them again.  All give the same results to rounding.
 * When the environment variable HMG_TUNE_CACHE names a file, a context takes the choice
 * recorded there for its GPU (device name and SM count) and N instead of timing, and
 * appends the choices it times, one line "<device name>|<SM count>|<N>|<variant>" each
 * (the last line for a key wins). */
hmg_status hmg_set_variant(hmg_ctx* ctx, int N, int variant);

/* The variant chosen for size N (-1 if none yet). */
hmg_status hmg_get_variant(hmg_ctx* ctx, int N, int* variant);

/* ---- tracing ------------------------------------------------------------------ */

/* Kernel kinds reported by the tracer. */
typedef enum {
    HMG_K_X_FORWARD = 0,   /* x pass, real -> complex, polarization fused (step 2 + 3) */
    HMG_K_Y_FORWARD = 1,   /* y pass forward (step 3) */
    HMG_K_Z_GREEN = 2,     /* z forward + Green operator + z inverse (steps 3-5) */
    HMG_K_Y_INVERSE = 3,   /* y pass inverse (step 5) */
    HMG_K_X_INVERSE = 4,   /* x pass, complex -> real, update and residual (steps 5-7) */
    HMG_K_EQ_X = 5,        /* equilibrium check: x pass with the flux average (step 1) */
    HMG_K_EQ_Z = 6,        /* equilibrium check: z pass with the divergence norm (step 1) */
    HMG_K_OTHER = 7,       /* reductions, conversions, voxelization */
    HMG_K_X_ROUND = 8,     /* x pass inverse + update of one sweep fused with the
                              polarization + x pass forward of the next (steps 5-7, 2-3) */
    HMG_K_FP64 = 9,        /* every pass of an FP64 sweep or FP64 equilibrium test */
    HMG_K_YXY = 10,        /* y pass inverse + x round trip + y pass forward of the next sweep,
                              one persistent kernel over (component, z) planes (steps 5-7, 2-3) */
    HMG_K_COUNT = 11
} hmg_kernel_kind;

/* Start (enable = 1, counters reset) or stop (0) timing every kernel the solver
 * launches with CUDA events recorded on the context's stream around each launch. */
hmg_status hmg_trace_enable(hmg_ctx* ctx, int enable);

/* Accumulated trace of one kernel kind: total device time (ms), launches, and the
 * algorithmic bytes those launches had to move (fields read and written once each). */
hmg_status hmg_trace_read(hmg_ctx* ctx, int kind, double* total_ms, long long* launches,
                          double* algo_bytes);

/* Measured FP64 fused-multiply-add rate of the context's GPU (flop/s, 2 per FMA): long
 * register-only chains over the whole device, best of five timed launches.  The plain
 * FP64 form of the solver is bound by this rate rather than by HBM bandwidth; the
 * paper has no counterpart (a measurement aid for the roofline of that form). */
hmg_status hmg_fp64_rate(hmg_ctx* ctx, double* flops_out);

/* Request-loop counters (zeros before the first hmg_submit): out[0] submitted,
 * out[1] completed, out[2] most requests resident on the device at once, out[3]
 * engine ticks, out[4] CUDA-graph captures, out[5] CUDA-graph launches. */
hmg_status hmg_server_stats(hmg_ctx* ctx, long long out[6]);

/* Device memory the solver state of one N^3 request occupies (bytes). */
size_t hmg_footprint(int N, hmg_precision precision);

#ifdef __cplusplus
}
#endif

#endif /* HMG_H */
