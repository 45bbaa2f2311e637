// Internal declarations shared by the translation units of libpou.so.
// Not part of the public C-ABI (see include/pou.h).
#pragma once

#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>

namespace pou {

typedef long long i64;

// Per-orbital raw sums (no dV factor) produced by the H-apply pass for the
// block W it reads, against the current iterate W' (prev) and its HW', with
// sigma' = <hw', w'> of that iterate (0 when there is none):
//   z' = hw - sigma' w                 -> <w,z'>, <z',z'>
//   s = w - w',  b = (hw - hw') - sigma' s  (so that Y = Z - Z' = b - (sigma - sigma') w)
// Sums of z' rather than of hw keep ||z||^2 and the Gram diagonal free of
// cancellation when tau * sigma is large.  Slot P_SIGP (written by the
// controller) records the sigma' the sums refer to.
// The kinetic sums are kept per axis without the 1/h^2 (and 1/12) factors,
// which are applied in FP64 when the energy is assembled.
enum { P_WW = 0, P_HW, P_ZW, P_ZZ, P_KX, P_KY, P_KZ, P_SS, P_SB, P_SW, P_BB, P_BW, NPT, P_SIGP = NPT, NP };
// Energy sums of the potential pass: sum rho*Vext, sum rho*V_H, sum eps_x(rho)*rho
enum { E_EXT = 0, E_H, E_X, NE };

constexpr int HIST_MAX = 16384;
constexpr double F_OCC = 2.0;

// Iteration state, resident in device memory and updated only by the
// controller kernel, so that a whole iteration (including the backtracking
// decision and the buffer swap) runs without a host round trip.
struct State {
  double tau_bb;     // Barzilai-Borwein step of the current step l
  double tau_trial;  // step of the pending trial, tau_bb * delta^s
  double C, Q;       // nonmonotone reference value and weight (Eq. ene-de)
  double E_cur;      // E(W^l)
  double znorm2;     // ||Z^l||_F^2
  double last_tau;   // step of the last accepted trial
  double terms_cur[4];
  double terms_trial[4];
  double df[3];      // relative energy changes, newest first (Sec. 4.2)
  double gram_off_trial, gram_off_acc;
  double e_tol;
  int cur;           // pair (0/1) holding W^l, HW^l, V^l, rho^l
  int l;             // accepted steps since the orbitals were set
  int s;             // step reductions so far in step l
  int target_l;      // stop once l reaches this
  int done;          // 1: every kernel of the pass returns at once
  int status;        // 0, or a pou_status breakdown code
  int converged;
  int passes, backtracks, forced, n_df;
  int chol_info;
  int reorth;        // 1: the trial needs a second Cholesky-QR pass (FP32 form)
  int reorth_count;  // second passes taken since the orbitals were set
  int diag_now;      // 1: subspace diagonalisation due before the next trial (Algorithm M)
  int diag_count;
  int orth_now;      // 1: the next trial is orthonormalised (Algorithm M: every n_org steps)
  int chol_fail;     // 1: the pending trial's Gram matrix was not positive definite (rejected)
};

// Gate of the optional kernels of a pass: 0 always run, 1 second Cholesky-QR
// pass (State::reorth), 2 subspace diagonalisation (State::diag_now), 3 the
// trial is orthonormalised (State::orth_now; Algorithm M with n_org > 1), 4
// first trial of a step (State::s == 0; the OptM-QR direction).
__device__ __forceinline__ bool gate_open(const State* st, int gate) {
  if (gate == 0) return true;
  if (gate == 1) return st->reorth != 0;
  if (gate == 2) return st->diag_now != 0;
  if (gate == 4) return st->s == 0;
  return st->orth_now != 0;
}

// ---------------------------------------------------------------- stencil
template <typename T>
struct ApplyArgs {
  const State* st;      // nullptr: explicit mode
  const T* W[2];
  T* HW[2];
  const T* V[2];
  const T* dV;          // history: V - V' of the trial vs the current pair, formed in FP64
  const double* sigma[2];
  int mode;             // 0: trial vs current, 1: trial without history, 2: explicit W[0],V[0]->HW[0],
                        // 3: refresh of the current pair after a subspace rotation, 4: the block
                        // W[cur] with V[cur], sums only, on the first pass of a step (conjugate-gradient
                        // directions: <d, H d>)
  double* tilepart;     // [N][ntile][NPT] or nullptr
  T out_scale;
  int N, nx, ny, nz, nzc;
  T ihx2, ihy2, ihz2;
  int cubic;            // 1: the three stencil scales are equal (FP64), so one kinetic sum serves
  const T* nl;          // nonlocal part of H applied to the block (same layout), added to H w; nullptr: none
  const T* nls;         // ... applied to the step s = w - w' (mode 0), added to H s; nullptr: none
};
template <typename T>
void launch_apply_h(const ApplyArgs<T>& a, int order, cudaStream_t s, int* ntile_out);
// Tiles of the H-apply launch (the partial-sum layout).  align: 2 when the
// blocks read are 16-byte aligned and the output 8-byte aligned (the library's
// own buffers), 1 when only the output is aligned to two elements, 0 otherwise;
// each level selects the kernel (and tile shape) that its accesses allow.
int apply_h_ntile(int nx, int ny, int nz, int N, int elem_bytes, int* nzc_out, int align = 2);

// ---------------------------------------------------------------- gram / rotation
template <typename T>
struct GramArgs {
  const State* st;      // iteration mode (trial == 1): source W[cur], HW[cur], sigma[cur], tau_trial
  const T* W[2];
  const T* HW[2];
  const double* sigma[2];
  const T* A;           // plain mode: A (and B for the general product)
  const T* B;           // general product A^T B (all blocks) when non-null
  int trial;
  int src_trial_slot;   // plain mode: source is W[1-cur] (second Cholesky-QR pass)
  int src_cur_pair;     // general mode: A = W[cur], B = HW[cur] (Sigma of Algorithm M)
  int gate;             // see gate_open
  i64 ng;
  int N;
  double* split;        // [nsplit][npair][ST*ST]
  const double* tfac;   // trial mode: orbital i steps tau_trial * tfac[i] (nullptr: 1 for all)
  int tf32_single;      // FP32 tensor-core Gram: one TF32 product (hi hi) instead of the three split ones
};
template <typename T>
int gram_supertile();
template <typename T>
void gram_layout(i64 ng, int N, bool general, int* nsplit, int* npair, i64* chunk);
template <typename T>
void launch_gram(const GramArgs<T>& a, cudaStream_t s);
// Same kernel with an explicit number of splits (each split writes one
// npair * ST * ST block of FP64 partial sums).
template <typename T>
void launch_gram_nsplit(const GramArgs<T>& a, int nsplit, cudaStream_t s);

// FP32 Gram on the tensor cores (TF32 split products), N <= 128, symmetric
// modes only; writes the same [nsplit][128 * 128] split layout (transposed
// and unsymmetrised: the reduction takes the symmetric part).
bool gram_tc_eligible(const GramArgs<float>& a);
// CTAs of a tensor-core Gram launch with nsplit splits over nsup 128-row blocks
int gram_tc_ctas(int nsplit, int nsup);
// Bounded-wait self-test (a barrier nothing arrives at): 0 on success with
// *timed_out = 1 when the wait gave up and recorded it; nonzero on a CUDA error.
int wait_selftest(double limit_s, int* timed_out);
void launch_gram_tc(const GramArgs<float>& a, int nsplit, cudaStream_t s);
void configure_gram_tc();

struct GramReduceArgs {
  const State* st;
  const double* split;
  int nsplit, npair, ST, N;
  int general;          // 1: all blocks computed (A^T B); 0: upper super-tiles, symmetric
  double dV;
  double* S;            // N*N
  // diagonal replacement for the trial Gram (iteration mode): 1 from the
  // H-apply sums (Opt-Par), 2 from the sums of a materialised direction (dpart)
  int trial;
  const double* dpart;  // [N][3]: <w,w>, <w,z>, <z,z> of a materialised direction z
  const double* sigma[2];
  const double* part[2];
  int gate;             // see gate_open
  const double* tfac;   // per-orbital step factors (nullptr: 1)
};
void launch_gram_reduce(const GramReduceArgs& a, cudaStream_t s);

template <typename T>
struct RotArgs {
  const State* st;      // iteration mode: A = W~ from W[cur], HW[cur]; out W[1-cur], rho[1-cur]
  const T* W[2];
  const T* HW[2];
  const double* sigma[2];
  T* Wout[2];
  double* rho[2];
  const T* A;           // explicit mode source
  T* B;                 // explicit mode destination
  double* rho_out;      // explicit mode density (nullable)
  const double* Rinv;   // N*N FP64 (upper)
  int trial;
  int src_trial_slot;   // plain mode with state: source W[1-cur], written in place
  int src_cur_slot;     // plain mode with state: source W[cur], written in place (W <- W P)
  int gate;             // see gate_open
  int sr_salt;          // distinguishes the rotations of one pass in the rounding counter
  i64 ng;
  int N;
  int general;          // 1: full matrix (no triangular skip)
  float* rimg;          // FP32 tensor-core rotation with N > 128: scratch of rotate_rimg_bytes(N)
  const double* tfac;   // trial mode: orbital i steps tau_trial * tfac[i] (nullptr: 1 for all)
};
int rotate_grid(i64 ng, int elem_bytes);
// bytes of the split R^-1 image the FP32 tensor-core rotation needs for N > 128
size_t rotate_rimg_bytes(int N);
// FP32 rotation on the tensor cores (TF32 split products for the
// off-diagonal part), N <= 128; one CTA per SM.
int rotate_tc_grid(i64 ng);
void launch_rotate_tc(const RotArgs<float>& a, cudaStream_t s);
void configure_rotate_tc();
template <typename T>
void launch_rotate(const RotArgs<T>& a, cudaStream_t s);

template <typename T>
void launch_density(const T* U, i64 ng, int N, double* rho, cudaStream_t s);
// ||HW - W Sigma||_F^2 / dV partials (Eq. gra), one per CTA; returns the CTA count.
template <typename T>
int launch_residual(const T* W, const T* HW, const double* Sig, int N, i64 ng, double* part, int max_blocks,
                    cudaStream_t s);
void launch_convert_f64_f32(const double* in, float* out, i64 n, cudaStream_t s);
void launch_convert_f32_f64(const float* in, double* out, i64 n, cudaStream_t s);
template <typename T>
void launch_scale_copy(const T* in, T* out, T scale, i64 n, cudaStream_t s);

// ---------------------------------------------------------------- OptM-QR direction
constexpr int POU_DIR_MAX_N = 512;
constexpr int POU_DIR_MAX_N_FP64 = 128;
template <typename T>
struct DirArgs {
  State* st;
  const T* W[2];
  const T* HW[2];
  T* Z[2];              // Z[cur] written, Z[1-cur] the previous step's
  const double* Sig;    // N*N, Sig[i][j] = <w_i, hw_j> of the current pair
  double* opart;        // [grid][N][3]
  double* bpart;        // [grid][3]
  i64 ng;
  int N;
};
struct DirCtrlArgs {
  State* st;
  const double* opart;
  const double* bpart;
  double* dpart;        // [N][3]
  int nblk, N;
  double dV, tau0, tau_min, tau_max;
  int bb_variant;
};
int direction_grid(i64 ng);
void configure_direction();
template <typename T>
void launch_direction(const DirArgs<T>& a, cudaStream_t s);
void launch_direction_control(const DirCtrlArgs& a, cudaStream_t s);

// ---------------------------------------------------------------- conjugate-gradient direction
template <typename T>
struct CgArgs {
  State* st;
  const T* W[2];
  const T* HW[2];
  T* D[2];              // directions: D[cur] written, D[1-cur] the previous step's
  T* Zs[2];             // z = hw - sigma w: Zs[cur] written, Zs[1-cur] the previous step's
  const double* sigma[2];
  const double* coef;   // [N][2]: beta_i, gamma_i (form pass)
  double* opart;        // [N][nch][CG_NS]
  i64 ng;
  int N, nch;
};
constexpr int CG_NS = 6;
struct CgCtrlArgs {
  State* st;
  const double* opart;  // [N][nch][CG_NS]
  int nch, N;
  double* coef;         // [N][2]
  const double* sigma[2];
  const double* tilepart;  // <d,d>, <d,H d> of the H-apply on D (mode 4)
  int ntile;
  double* tfac;
  double* dpart;        // [N][3]
  double dV, tau0, tau_min, tau_max;
};
int cg_chunks(i64 ng);
template <typename T>
void launch_cg_dots(const CgArgs<T>& a, cudaStream_t s);
template <typename T>
void launch_cg_form(const CgArgs<T>& a, cudaStream_t s);
void launch_cg_beta(const CgCtrlArgs& a, cudaStream_t s);
void launch_cg_step(const CgCtrlArgs& a, cudaStream_t s);

// ---------------------------------------------------------------- nonlocal projectors
constexpr int kMaxProj = 256;  // = POU_MAX_PROJ of pou.h
struct NlTables {
  int P, nx, ny, nz;
  const double* gx;     // [P][nx], amplitude folded in
  const double* gy;     // [P][ny]
  const double* gz;     // [P][nz]
  const float* gxf;     // FP32 copies for the FP32 form
  const float* gyf;
  const float* gzf;
  const int* win;       // [P][6]: start and length of the x, y and z windows (they wrap)
};
template <typename T>
struct NlArgs {
  const State* st;      // nullptr: explicit block X[0]
  NlTables tab;
  const T* X[2];
  int sel;              // 0: X[0] -> C[0]; 1: trial slot 1-cur; 2: current slot cur
  double* C[2];         // [N][P] projections C_ip = <xi_p, x_i>
  T* nl;                // [N][ng]: sum_p xi_p C_ip
  T* nls;               // trial only: sum_p xi_p (C_ip - C'_ip), C' = C[cur]; nullptr otherwise
  int gate;             // see gate_open
  int N;
  double dV;
};
constexpr int kMaxProjGrid = 512;  // largest nx the projection kernel stages (fits shared memory)
// part: scratch of nl_part_bytes(N, P, n) bytes (per-plane partial sums)
size_t nl_part_bytes(int N, int P, const int n[3]);
template <typename T>
void launch_nl_project(const NlArgs<T>& a, double* part, cudaStream_t s);
template <typename T>
void launch_nl_apply(const NlArgs<T>& a, cudaStream_t s);
void configure_nonlocal();

// ---------------------------------------------------------------- cholesky
// reorth_thr > 0: first pass, sets st->reorth when max|S - I| > reorth_thr;
// reorth_thr < 0: second pass, gated on st->reorth; 0: neither.
// soft_limit >= 0 (trials of the iteration): a failing pivot rejects the
// trial (State::chol_fail) while State::s < soft_limit; otherwise, and with
// soft_limit < 0, it is a breakdown (POU_ENOTSPD).
void launch_cholinv(const State* st, const double* S, double* Rinv, int N, int* info,
                    State* st_rw, double piv_rel, double reorth_thr, cudaStream_t s, bool orth_gated = false,
                    int soft_limit = -1);
size_t cholinv_smem_bytes(int N);

// ---------------------------------------------------------------- fft / potential
struct FftPlan {
  int n[3];
  int nst[3];
  int radix[3][8];
  double2* tw[3];       // device, n[a] entries exp(-2 pi i k / n)
  double* g2[3];        // device, (2 pi m / L)^2, m in FFT order
  int lb[3];            // lines per block
  double* mem;          // one allocation holding all tables
};
bool fft_supported(int n);
int fft_plan_create(FftPlan* p, const int n[3], const double L[3]);
void fft_plan_destroy(FftPlan* p);

template <typename T>
struct PotArgs {
  const State* st;      // iteration mode: rho[1-cur] -> V[1-cur]
  const double* rho[2];
  double* V64[2];
  T* V[2];
  const double* rho_x;  // explicit mode
  double* V64_x;
  T* V_x;
  double* vh_out;       // stand-alone Hartree: write V_H only
  const double* vext;
  double2* work;
  double* epart;        // [nblk][NE]
  T* dv_out;            // iteration mode: V_new - V64[cur], rounded to T (nullable)
  int hartree, exchange;
};
template <typename T>
int launch_potential(const FftPlan& p, const PotArgs<T>& a, cudaStream_t s);  // returns nblk

// ---------------------------------------------------------------- atoms
struct AtomTables {
  double* gx; double* gy; double* gz;      // [M][n]
  double* dgx; double* dgy; double* dgz;   // [M][n]
  int* win;                                // [M][3][2] window start, length
};
void launch_atom_tables(const double* R, const double* Z, int M, double width, const int n[3],
                        const double L[3], const AtomTables& t, cudaStream_t s);
void launch_vext(const double* Z, int M, const int n[3], const AtomTables& t, double* vext,
                 cudaStream_t s);
int launch_forces(const double* rho, const double* Z, int M, const int n[3], const AtomTables& t,
                  double* fpart, cudaStream_t s);  // returns z splits; fpart [M][split][4]

// ---------------------------------------------------------------- controller
struct CtrlArgs {
  State* st;
  double* hist_E;
  double* hist_tau;
  double* sigma[2];
  double* part[2];
  const double* tilepart;
  int ntile;
  const double* epart;
  int neblk;
  int N;
  int init;
  double dV, rho1, delta, eta, tau0, tau_min, tau_max;
  int bb_variant, max_backtrack;
  double* tfac;         // per-orbital Barzilai-Borwein steps: tau_i = tau * tfac[i] (nullptr: one tau)
  const double* nlC[2]; // projections C_ip of each pair (nullptr: no projectors); the nonlocal energy
  int P;                // f sum C_ip^2 of the trial joins the external term
  int n_diag;           // subspace diagonalisation period (0: off)
  int n_org;            // Algorithm M: orthonormalise every n_org steps (1: every step)
  int refresh;          // 1: re-reduce the sums of the rotated current pair only
  int fp32;             // the H-apply formed z' = hw - sigma' w with sigma' rounded to FP32
  double kc[3];         // kinetic coefficient per axis: -1/2 * (1 or 1/12) / h_a^2
};
void launch_control(const CtrlArgs& a, cudaStream_t s);

// true if p is CUDA device (or managed) memory of this process; the entry
// points that take device pointers check them, so that a host pointer gives
// POU_EINVAL instead of reaching a kernel
bool device_accessible(const void* p);

// Shared-memory opt-ins of the kernels that need more than 48 KB; called
// once per process before any launch (and before any graph capture).
void configure_rotate();
void configure_cholinv();
void configure_fft();
void configure_eigh();
void configure_apply_h();
void configure_kernels();
void launch_eigh(const State* st, const double* Sig, double* P, double* VT, double* ev0, double* ev1, int N,
                 cudaStream_t s);

// Profiler names of the Gram and rotation launches by source: the trial
// block (2 blocks read by the Gram, 2 read + 1 written by the rotation), the
// second Cholesky-QR pass on the block just written (1; 1 + 1), the subspace
// pair of Algorithm M, or a caller's block.
inline const char* gram_prof_name(int trial, int src_trial_slot, int src_cur_pair) {
  return trial ? "gram" : src_trial_slot ? "gram_reorth" : src_cur_pair ? "gram_sigma" : "gram_plain";
}
inline const char* rotate_prof_name(int trial, int src_trial_slot, int src_cur_slot) {
  return trial ? "rotate_density" : src_trial_slot ? "rotate_reorth" : src_cur_slot ? "rotate_subspace"
                                                                                    : "rotate_plain";
}

// Streaming multiprocessors of the current device, queried once per device;
// launch shapes are sized in multiples of it.
int num_sms();

// Counts every kernel launched by the library (host side).
extern long long g_launches;

// Per-kernel CUDA-event timing.  When a context enables profiling it installs
// a recorder for the calling thread; every launch site brackets its kernel
// with prof_begin / prof_end, which record events on the launch stream.
struct ProfRecorder {
  virtual void begin(const char* name, cudaStream_t s) = 0;
  virtual void end(cudaStream_t s) = 0;
  virtual ~ProfRecorder() {}
};
extern thread_local ProfRecorder* g_prof;
inline void prof_begin(const char* name, cudaStream_t s) {
  if (g_prof) g_prof->begin(name, s);
}
inline void prof_end(cudaStream_t s) {
  ++g_launches;
  if (g_prof) g_prof->end(s);
}

}  // namespace pou
