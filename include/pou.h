/*
 * pou.h -- C-ABI of the GB300-native parallel orbital-updating solver.
 *
 * Method: Dai, Liu, Zhang, Zhou, "A Parallel Orbital-updating Based
 * Optimization Method for Electronic Structure Calculations" (arXiv 1510.07230).
 *
 * Problem statement (Sec. 2.1, Eq. emin and Eq. energy; the initialisation of Algorithm B):
 * given a uniform periodic grid, the external potential (or Gaussian-well
 * atoms), the number N of doubly occupied orbitals and an initial block U,
 * minimise the discrete Kohn-Sham energy
 *
 *   E(U) = f sum_i <u_i, -1/2 Lap_h u_i> + dV sum_r rho Vext
 *          + 1/2 dV sum_r rho V_H + dV sum_r eps_x(rho) rho,   f = 2,
 *
 * over orthonormal U (<u_i, u_j> = dV sum_r u_i u_j = delta_ij), with
 * rho = f sum_i u_i^2, V_H the periodic Hartree potential of rho (zero mean,
 * neutralising background) and Slater LDA exchange.  The solver returns the
 * energy, the orbitals and the density.
 *
 * Each iteration (Algorithm E, i.e. Algorithm M with n_org = 1; Sec. 3.2;
 * Algorithm M's n_org > 1 and subspace diagonalisation are options below):
 * HW = H(rho) W, sigma_ii = <H w_i, w_i>, direction z_i = H w_i - sigma_ii w_i,
 * a shared Barzilai-Borwein step, nonmonotone backtracking (Eq. ene-de) and
 * Orth by Cholesky-QR (S = <Wt^T Wt>, S = R^T R, W = Wt R^-1), then the new
 * density and the Hartree potential by an FFT Poisson solve.
 *
 * Conventions (every call):
 *  - Units: Hartree and bohr.
 *  - Orbital blocks are laid out [N][nz][ny][nx], x fastest, one orbital
 *    after another; fields (Vext, rho) are [nz][ny][nx].
 *  - Grid point (i, j, k) sits at (i*hx, j*hy, k*hz), h_a = L_a / n_a,
 *    dV = hx*hy*hz.
 *  - dtype codes: POU_DT_F64 (double) or POU_DT_F32 (float).
 *  - on_device = 1: the pointer is CUDA device memory (for example a torch
 *    tensor's data_ptr) and is used on the context's stream; 0: host memory.
 *  - Ownership: the caller owns every pointer it passes; the library copies
 *    what it needs and retains no caller pointer after the call returns.
 *  - Errors: every call returns a pou_status; no call aborts the process or
 *    traps the device.  pou_last_error() gives a one-line description of the
 *    last failure of that context.
 *  - Calls on one context are not thread-safe; distinct contexts are
 *    independent.
 */
#ifndef POU_H
#define POU_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pou_ctx pou_ctx;

typedef enum {
  POU_OK = 0,
  POU_EINVAL = 1,   /* bad argument or configuration */
  POU_ENOMEM = 2,   /* device or host allocation failed */
  POU_ECUDA = 3,    /* a CUDA runtime call failed */
  POU_ENOTSPD = 4,  /* Gram matrix not positive definite in Cholesky-QR */
  POU_ENAN = 5,     /* non-finite energy or step */
  POU_ENOCONV = 6   /* stopping tolerance not met within max_iter */
} pou_status;

/* Arithmetic of the bulk (orbital blocks, stencil, Gram, rotation). */
typedef enum {
  POU_FP64 = 0,         /* plain method: everything in FP64 */
  POU_FP32 = 1,         /* mixed: FP32 orbitals/stencil/potential; Gram and rotation on the
                           tensor cores with TF32 split products (three per product, about
                           2^-21 relative) and FP64 promotion; FP64 Cholesky, density,
                           Hartree solve, energies and traces */
  POU_FP32_TF32X3 = 1,  /* the same form, named by its Gram */
  POU_FP32_TF32 = 2     /* as POU_FP32 with a single TF32 product (hi hi) in the iteration's
                           Gram matrices: a third of the tensor-core work of the Gram; its
                           rounding errors are zero-mean and average over the grid points (the
                           trial Gram's diagonal stays the FP64 norm of the H-apply sums); the
                           rotation keeps the split products */
} pou_precision;

typedef enum { POU_DT_F64 = 0, POU_DT_F32 = 1 } pou_dtype;

typedef struct {
  int n[3];           /* grid points nx, ny, nz (each >= 2; FFT sizes 2^a 3^b 5^c) */
  double L[3];        /* periodic box edges, bohr */
  int stencil_order;  /* 2: 7-point Laplacian, 4: 13-point Laplacian */
  int N;              /* number of doubly occupied orbitals, 1..POU_MAX_N */
  int precision;      /* pou_precision */
  int hartree;        /* 1: Hartree term on; 0: off (closed-form tests) */
  int exchange;       /* 1: Slater exchange on; 0: off */
  int bb_variant;     /* 1: tau1 = tr<S^T S>/|tr<S^T Y>|, 2: tau2 = |tr<S^T Y>|/tr<Y^T Y>,
                         3 (default): tau1 on even steps l, tau2 on odd steps */
  double rho1;        /* backtracking constants of Eq. ene-de: 1e-4 */
  double delta;       /* 0.1 */
  double eta;         /* 0.85 */
  int max_backtrack;  /* after this many reductions the trial is accepted: 10 */
  double tau0;        /* first step; <= 0 selects 1 / lambda_max(-1/2 Lap_h) */
  double tau_min;     /* step clamp: 1e-12 */
  double tau_max;     /* step clamp: 1e3 */
  int n_org;          /* Algorithm M: Orth every n_org steps (>= 1; 1 = Algorithm E).  The
                         steps in between take W - tau Z as it is (no Orth, no Eq. ene-de test,
                         no backtracking); their history entries are NaN and pou_energy
                         reports the last orthonormalised step's energy until the next one */
  int n_diag;         /* Algorithm M: subspace diagonalisation every n_diag steps
                         (Sec. 3.3: Sigma = <W^T H W>, P^T Sigma P diagonal, W <- W P);
                         0 = off */
  void* stream;       /* cudaStream_t to run on; NULL: the library creates one */
  int direction;      /* search direction (Sec. 3.1): 0 (default) Opt-Par, z_i = H w_i - sigma_ii w_i;
                         1 OptM-QR, the comparison method of Table 1, Z = HW - W Sigma with the full
                         Sigma = <W^T H W>, its own Barzilai-Borwein differences Y = Z - Z'.  1 needs
                         n_org = 1 and n_diag = 0, and two more orbital blocks of device memory */
  int tau_mode;       /* 0 (default): one Barzilai-Borwein step for all orbitals; 1: a step tau_i per
                         orbital from its own s_i, y_i (Sec. 3.2's tau_i); backtracking scales all by
                         delta^s and Eq. ene-de takes sum_i tau_i ||z_i||^2.  1 needs direction = 0,
                         solver = 0, n_org = 1, n_diag = 0 */
  int solver;         /* per-orbital subproblem solver (Sec. 3.1): 0 (default) steepest descent;
                         1 conjugate gradient: d_i = z_i + beta_i (d_i' - <w_i,d_i'> w_i), Polak-Ribiere
                         beta_i >= 0 capped so that <z_i,d_i> >= <z_i,z_i>/2, and the Newton step
                         tau_i = <z_i,d_i> / <d_i,(H - sigma_ii) d_i> of each orbital's frozen-potential
                         Rayleigh quotient; Eq. ene-de takes sum_i tau_i <z_i,d_i>.  1 needs direction = 0,
                         tau_mode = 0, n_org = 1, n_diag = 0, and four more orbital blocks */
} pou_config;

#define POU_MAX_N 512      /* FP32 forms (without the subspace diagonalisation) */
#define POU_MAX_N_FP64 128 /* FP64 form, the subspace diagonalisation, FP64 pou_rotate */

typedef struct {
  double kinetic;   /* f sum_i <w_i, -1/2 Lap_h w_i> */
  double external;  /* dV sum rho Vext */
  double hartree;   /* 1/2 dV sum rho V_H */
  double exchange;  /* dV sum eps_x(rho) rho */
  double total;
} pou_energy_terms;

typedef struct {
  int iterations;        /* accepted steps taken by this call */
  int passes;            /* trial evaluations by this call (accepted + rejected) */
  int backtracks;        /* step reductions by this call (Eq. ene-de failures) */
  int forced;            /* trials accepted after max_backtrack reductions */
  int total_iterations;  /* accepted steps since pou_set_orbitals */
  int converged;         /* 0: no, 1: energy criterion met, 2: gradient criterion met */
  double energy;         /* E of the current orbitals, Ha (n_org > 1: of the last orthonormalised step) */
  double tau;            /* last accepted step */
  double df_mean3;       /* (df^l + df^(l-1) + df^(l-2)) / 3 of Sec. 4.2 */
  double grad_norm;      /* ||HW - W Sigma||_F (Eq. gra) when computed, else -1 */
  double gram_offdiag;   /* max |S - I| of the last accepted trial Gram matrix */
  int second_passes;     /* FP32 form: trials orthonormalised twice by this call (Cholesky-QR
                            repeated when max |S - I| > 0.02); 0 in the FP64 form */
  int diagonalisations;  /* subspace diagonalisations (Algorithm M) by this call */
} pou_report;

/* Fill a config with the paper's constants (Sec. 3.2) and FP64 defaults. */
void pou_config_default(pou_config* cfg);

/* Validate cfg, allocate the device buffers (four orbital blocks, fields,
 * FFT and reduction workspaces) and return a context.  EINVAL on a bad
 * configuration, ENOMEM if the device cannot hold the buffers. */
pou_status pou_create(const pou_config* cfg, pou_ctx** out);

/* Release the context and all of its device memory. NULL is a no-op. */
void pou_destroy(pou_ctx* ctx);

/* One-line description of the last error on this context ("" if none). */
const char* pou_last_error(const pou_ctx* ctx);

/* Set the external potential Vext(r) (Sec. 2.1), nx*ny*nz doubles. */
pou_status pou_set_vext(pou_ctx* ctx, const double* vext, int on_device);

/* Set Vext from M Gaussian wells, Vext(r) = -sum_I Z_I sum_n
 * exp(-|r - R_I - nL|^2 / (2 width^2)), n over the 27 nearest images of R_I
 * folded into [0, L) (a local pseudopotential, Sec. 2.1).  R: M*3 host
 * doubles (x, y, z per atom), Z: M host doubles; width > 0. */
pou_status pou_set_atoms(pou_ctx* ctx, int M, const double* R, const double* Z, double width);

/* Nonlocal part of the pseudopotential (Sec. 2.1): V_nloc u = sum_p <xi_p, u> xi_p
 * with P synthetic Gaussian projectors xi_p(r) = amps[p] sum_n
 * exp(-|r - c_p - nL|^2 / (2 widths[p]^2)) (n over the 27 nearest images of
 * the centre folded into [0, L)).  centres: P*3 host doubles (x, y, z),
 * widths, amps: P host doubles; P = 0 removes them (P <= 256).  H gains the
 * term and the energy's external part gains f sum_i sum_p <xi_p, w_i>^2.
 * The projectors do not move with the atoms of pou_set_atoms, so dE/dR of
 * pou_backward covers the local wells only.  Like pou_set_vext, the current
 * orbitals must be set again afterwards.  EINVAL with solver = 1. */
#define POU_MAX_PROJ 256
pou_status pou_set_projectors(pou_ctx* ctx, int P, const double* centres, const double* widths, const double* amps);

/* Load N orbitals (the initialisation of Algorithm B) and orthonormalise them by one
 * Cholesky-QR; then build rho, V and E of the orthonormal block and reset
 * the iteration history (C^0 = E, Q^0 = 1, Sec. 3.2).  U: [N][nz][ny][nx]
 * in dtype.  ENOTSPD if U is rank deficient. */
pou_status pou_set_orbitals(pou_ctx* ctx, const void* U, int dtype, int on_device);

/* Run up to max_iter accepted steps of Algorithm E (Algorithm M with the
 * config's n_org and n_diag, Sec. 3.3).  Stops early when
 * e_tol > 0 and the mean of the last three relative energy changes is below
 * e_tol (Sec. 4.2), or when grad_tol > 0 and ||grad E||_F < grad_tol
 * (Eq. gra; checked every 10 steps).  rep may be NULL.  Returns ENOCONV if a
 * tolerance was given and not met, ENOTSPD / ENAN on breakdown. */
pou_status pou_iterate(pou_ctx* ctx, int max_iter, double e_tol, double grad_tol, pou_report* rep);

/* Energy terms of the current orbitals (FP64); with n_org > 1, those of the
 * last orthonormalised step (the steps in between are not orthonormal). */
pou_status pou_energy(pou_ctx* ctx, pou_energy_terms* out);

/* Copy out the current orbitals, converted to dtype. */
pou_status pou_get_orbitals(pou_ctx* ctx, void* U, int dtype, int on_device);

/* Copy out the density rho = f sum_i w_i^2 (FP64, nx*ny*nz). */
pou_status pou_get_density(pou_ctx* ctx, double* rho, int on_device);

/* Copy out the local potential V = Vext + V_H + v_x of the current density (FP64). */
pou_status pou_get_potential(pou_ctx* ctx, double* V, int on_device);

/* ||grad E||_F = sqrt(tr<G^T G>), G = HW - W Sigma, Sigma = <(HW)^T W>
 * (Eq. gra, Sec. 2.2), of the current orbitals W and their HW, into *out
 * (host).  Sigma is formed on the device in the working precision; G is
 * formed point by point and its squares summed in FP64.  Synchronises the
 * context's stream.  POU_EINVAL when no orbitals are set.  Overwrites the
 * context's N x N scratch matrix (not part of the iteration state).  */
pou_status pou_gradient_norm(pou_ctx* ctx, double* out);

/* Energy of an arbitrary block U (not orthonormalised, Eq. energy) without
 * touching the iteration state: builds rho(U), V_H, v_x and the four terms.
 * A device block of the context's dtype is read in place: it needs only the
 * element's own alignment (a block off the 16-byte boundary is served by a
 * kernel with narrower accesses, at some cost in speed). */
pou_status pou_evaluate(pou_ctx* ctx, const void* U, int dtype, int on_device, pou_energy_terms* out);

/* Adjoint of pou_evaluate: with g = dL/dE,
 *   dEdU = g * 2 f dV H(rho_U) U            (E_{u_i} = H u_i, Sec. 2.1),
 *   dEdR[I][a] = g * dV sum_r rho dVext/dR_I,a,  dEdZ[I] = g * dV sum_r rho dVext/dZ_I
 * for the atoms of pou_set_atoms.  V_H and v_x are rebuilt from rho(U); no
 * per-orbital intermediate is stored.  U == NULL uses the current orbitals.
 * dEdU (same dtype/location as U, or device/host per on_device when U is
 * NULL), dEdR (M*3 host doubles) and dEdZ (M host doubles) may each be NULL.
 * As for pou_evaluate, device blocks need only element alignment.
 * EINVAL if dEdR/dEdZ are requested without atoms. */
pou_status pou_backward(pou_ctx* ctx, const void* U, int dtype, int on_device, double g,
                        void* dEdU, double* dEdR, double* dEdZ);

/* Per-iteration history since pou_set_orbitals (Fig. 3 style curves):
 * up to max_entries accepted energies and steps, oldest first (NaN energy
 * for the steps between orthonormalisations when n_org > 1); *count gets
 * the number written.  E, tau may be NULL. */
pou_status pou_get_history(pou_ctx* ctx, double* E, double* tau, int max_entries, int* count);

/* Checkpoint / resume: the scalar history (tau, C, Q, sigma, step counters)
 * and the current and previous orbital blocks with their H-products.
 * pou_get_state with blob == NULL writes the required size to *size. */
pou_status pou_get_state(pou_ctx* ctx, void* blob, size_t* size);
pou_status pou_set_state(pou_ctx* ctx, const void* blob, size_t size);

/* Diagnostics (no counterpart in the paper): every wait of the tensor-core
 * kernels on a shared-memory barrier gives up after a time limit, records it
 * and lets the kernel return, so that a lost arrival surfaces as POU_ECUDA
 * instead of a hang.  This runs that bounded wait on a barrier that nothing
 * arrives at, with limit_s seconds (0 < limit_s <= 10), on the current device
 * and its legacy default stream; *timed_out = 1 when it gave up as designed.
 * POU_ECUDA if the launch failed; the device stays usable either way. */
pou_status pou_selftest_wait_timeout(double limit_s, int* timed_out);

/* Block until all work queued by the context has finished. */
pou_status pou_synchronize(pou_ctx* ctx);

/* Number of kernels launched by the library in this process since the
 * context was created. */
long long pou_launch_count(const pou_ctx* ctx);

/* Per-kernel timing, the tracing counterpart of the paper's par-time /
 * total-time split (Sec. 4.2).  While enabled, passes are launched one
 * kernel at a time (no graph replay) and every kernel is bracketed by CUDA
 * events on the context's stream.  Disabling discards the counters. */
pou_status pou_set_profiling(pou_ctx* ctx, int enable);

/* Read the counters: up to max_entries kernels, each with its name (32 bytes
 * per entry in names, NUL-terminated), number of launches and total
 * milliseconds.  Synchronises the context's stream.  Any output may be NULL. */
pou_status pou_get_profile(pou_ctx* ctx, int max_entries, char* names, long long* launches, double* ms,
                           int* count);

/* ------------------------------------------------------------------------
 * Stand-alone operations on caller-owned device buffers.  These run the
 * same kernels as the iteration, one step of Sec. 3.2 each.  Pointers are
 * device pointers (a pointer that is not CUDA device or managed memory
 * returns POU_EINVAL before any launch; so does on_device = 1 with such a
 * pointer in the calls above), stream is a cudaStream_t (NULL = legacy
 * default stream).
 * ------------------------------------------------------------------------ */

/* Gram matrix S = dV * A^T A (Sec. 3.2, Cholesky-based QR, first step) of a
 * block A of N <= POU_MAX_N columns of length Ng, stored [N][Ng] in dtype.
 * S: N*N device doubles, row-major and symmetric.  workspace: device memory of at least
 * pou_gram_workspace_bytes(dtype, Ng, N) bytes, 256-byte aligned. */
size_t pou_gram_workspace_bytes(int dtype, long long Ng, int N);
pou_status pou_gram(int dtype, long long Ng, int N, const void* A, double dV, double* S,
                    void* workspace, size_t workspace_bytes, void* stream);

/* Allocation-free Gram matrix: the result of pou_gram (same arguments
 * without the workspace), for callers that cannot allocate device memory:
 * hosts that give this library a fixed device-memory budget, and loops that
 * must not call cudaMalloc once they run (it can synchronise the device and
 * stall every stream).  The paper has no counterpart: this is a library
 * service, not a step of the method.
 *  - The per-split partial sums live in one fixed buffer of static device
 *    memory of POU_GRAM_NOALLOC_MAX_BYTES, which every GPU that loads the
 *    library holds until the process exits; the call allocates nothing.
 *  - The first call on a device looks up the buffer's device address, with
 *    that device current, and keeps it for the life of the process; make
 *    that first call before any stream capture.  The kept address assumes
 *    the device's primary context: after cudaDeviceReset, or from another
 *    driver context on the same device, the buffer moves and the kept
 *    address is stale.
 *  - The number of splits is capped to what fits the buffer, so results may
 *    differ from pou_gram by rounding; N > POU_MAX_N (or a split that does
 *    not fit) returns POU_EINVAL.
 *  - Every call shares the buffer, and each call overwrites every part of
 *    it that it reads, so nothing has to start at zero; calls that overlap
 *    on the GPU (other streams, other host threads) race on the buffer and
 *    must be serialised by the caller. */
#define POU_GRAM_NOALLOC_MAX_BYTES (8u << 20)
pou_status pou_gram_noalloc(int dtype, long long Ng, int N, const void* A, double dV, double* S, void* stream);

/* Cholesky factor and triangular inverse (Sec. 3.2): S = R^T R with R upper
 * triangular and positive diagonal, Rinv = R^-1 (N*N device doubles,
 * row-major, lower part zero), N <= POU_MAX_N.  *info (device int) is 0 on
 * success or k+1 if the k-th pivot is not positive (then Rinv is
 * unspecified).  For N > 128 Rinv also serves as the working matrix and the
 * call is a sequence of kernels on the stream. */
pou_status pou_cholinv(int N, const double* S, double* Rinv, int* info, void* stream);

/* Rotation and density (Sec. 3.2 Orth, last step; Sec. 2.1 density):
 * B = A Rinv (columns), i.e. B_j = sum_{i<=j} Rinv[i][j] A_i, and
 * rho = f sum_j B_j^2 (FP64).  A, B: [N][Ng] dtype; Rinv: N*N doubles, upper
 * triangular; rho: Ng doubles (may be NULL).  N <= POU_MAX_N for FP32,
 * N <= POU_MAX_N_FP64 for FP64.  FP32 with N > 128 takes a stream-ordered
 * scratch of a few MB (cudaMallocAsync), released on the same stream;
 * POU_ENOMEM if it cannot be had. */
pou_status pou_rotate(int dtype, long long Ng, int N, const void* A, const double* Rinv,
                      void* B, double* rho, void* stream);

/* Hartree potential of rho by the FFT Poisson solve (-Lap V_H = 4 pi (rho -
 * mean rho), V_H_hat(0) = 0): n = {nx, ny, nz}, L = box; rho, vh: Ng device
 * doubles.  workspace: pou_hartree_workspace_bytes(n) bytes of device memory. */
size_t pou_hartree_workspace_bytes(const int n[3]);
pou_status pou_hartree(const int n[3], const double L[3], const double* rho, double* vh,
                       void* workspace, size_t workspace_bytes, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* POU_H */
