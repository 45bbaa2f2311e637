// Host side of libpou.so: the C-ABI of include/pou.h.
//
// The context owns two buffer pairs (W, HW, V, rho) on the device.  One
// pass of the iteration is a fixed kernel sequence that reads the device
// State to find the current pair, builds the trial point in the other pair,
// evaluates it and lets the controller kernel accept it (swap) or shrink the
// step; so a pass needs no host decision and is captured once into a CUDA
// graph and replayed.  The host only sets the stopping target and reads the
// State back between batches of passes.
#include "pou.h"
#include "pou_internal.cuh"

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

using namespace pou;

namespace {

// CUDA-event recorder of one context: every bracketed launch gets a start and
// an end event on its stream; elapsed times are summed per kernel name when
// the profile is read.
struct CtxProfiler : ProfRecorder {
  std::vector<std::string> names;
  std::map<std::string, int> index;
  std::vector<long long> launches;
  std::vector<double> ms;
  std::vector<cudaEvent_t> pool;
  size_t used = 0;
  struct Rec {
    int id;
    cudaEvent_t a, b;
  };
  std::vector<Rec> recs;
  int pending_id = -1;
  cudaEvent_t pending_a = nullptr;

  cudaEvent_t next_event() {
    if (used == pool.size()) {
      cudaEvent_t e;
      cudaEventCreate(&e);
      pool.push_back(e);
    }
    return pool[used++];
  }
  void begin(const char* name, cudaStream_t s) override {
    auto it = index.find(name);
    int id;
    if (it == index.end()) {
      id = (int)names.size();
      index[name] = id;
      names.push_back(name);
      launches.push_back(0);
      ms.push_back(0.0);
    } else {
      id = it->second;
    }
    pending_id = id;
    pending_a = next_event();
    cudaEventRecord(pending_a, s);
  }
  void end(cudaStream_t s) override {
    cudaEvent_t b = next_event();
    cudaEventRecord(b, s);
    recs.push_back({pending_id, pending_a, b});
  }
  void collect() {
    for (const Rec& r : recs) {
      cudaEventSynchronize(r.b);
      float t = 0.f;
      cudaEventElapsedTime(&t, r.a, r.b);
      ms[r.id] += t;
      launches[r.id] += 1;
    }
    recs.clear();
    used = 0;
  }
  ~CtxProfiler() override {
    for (cudaEvent_t e : pool) cudaEventDestroy(e);
  }
};

}  // namespace

struct pou_ctx {
  pou_config cfg;
  int dt;       // 0 double, 1 float
  int tf32_single;  // POU_FP32_TF32: the tensor-core Gram takes one TF32 product
  size_t esz;   // bytes per orbital element
  int nx, ny, nz, N;
  i64 ng;
  double h[3], dV, tau0;
  cudaStream_t stream;
  bool own_stream;
  std::string err;

  void* W[2];
  void* HW[2];
  void* V[2];       // working potential (element type of the bulk)
  double* V64[2];   // FP64 potential (aliases V when dt == 0)
  double* rho[2];
  double* vext;
  double2* work;
  double* sigma[2];
  double* part[2];
  double* tilepart;
  int ntile;
  double* epart;
  int neblk_max;
  double* S;
  double* Rinv;
  double* split;
  size_t split_elems;
  double* evec;      // eigenvector scratch of the subspace diagonalisation
  float* rimg;       // split R^-1 image of the FP32 tensor-core rotation (N > 128)
  void* dv;          // V(trial) - V(current), working type (written by the potential pass)
  // OptM-QR direction (config direction = 1): Z = HW - W Sigma per pair, the
  // direction kernel's partials, the per-orbital sums of the trial diagonal,
  // and a zero sigma (the trial kernels then form W - tau Z)
  void* Z[2];
  double* dir_opart;
  double* dir_bpart;
  double* dir_dpart;
  double* zero_sigma;
  // per-orbital step factors (tau_mode = 1, solver = 1); conjugate-gradient
  // directions and the z of the previous step, their partial sums and
  // coefficients (solver = 1)
  double* tfac;
  void* D[2];
  void* Zs[2];
  double* cg_opart;
  double* cg_coef;
  // nonlocal projectors (pou_set_projectors): per-axis tables and windows,
  // projections of each pair and of an explicit block, the nonlocal parts of
  // H w and of H s
  int P;
  void* nl_mem;
  NlTables nlt;
  double* nlC[2];
  double* nlCe;
  void* nl;
  void* nls;
  double* nl_part;  // per-plane partial projections
  State* st;
  double* hist_E;
  double* hist_tau;
  int* info;
  FftPlan fft;

  // atoms
  int M;
  double width;
  double* dR;
  double* dZ;
  AtomTables tabs;
  double* fpart;
  std::vector<double> hR, hZ;

  // evaluation scratch (allocated on first use)
  void* ublock;
  void* gblock;
  double* rho_e;
  void* V_e;
  double* V64_e;

  cudaGraphExec_t graph;
  int kernels_per_pass;
  CtxProfiler* prof;
  bool have_orbitals;
  long long launches0;
};

namespace {

// Installs the context's recorder for the duration of one API call.
struct ProfScope {
  explicit ProfScope(pou_ctx* c) { g_prof = (c && c->prof) ? c->prof : nullptr; }
  ~ProfScope() { g_prof = nullptr; }
};

pou_status fail(pou_ctx* c, pou_status s, const char* fmt, ...) {
  if (c) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    c->err = buf;
  }
  return s;
}

#define CK(call)                                                                              \
  do {                                                                                        \
    cudaError_t e_ = (call);                                                                  \
    if (e_ != cudaSuccess) return fail(c, POU_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

pou_status dalloc(pou_ctx* c, void** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) return POU_OK;
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return fail(c, POU_ENOMEM, "cudaMalloc(%zu bytes): %s", bytes, cudaGetErrorString(e));
  }
  return POU_OK;
}

#define DALLOC(ptr, bytes)                                                   \
  do {                                                                       \
    pou_status s_ = dalloc(c, reinterpret_cast<void**>(&(ptr)), (bytes));    \
    if (s_ != POU_OK) return s_;                                             \
  } while (0)

pou_status check_launch(pou_ctx* c, const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(c, POU_ECUDA, "%s: %s", what, cudaGetErrorString(e));
  return POU_OK;
}

pou_status read_state(pou_ctx* c, State* hs) {
  CK(cudaMemcpyAsync(hs, c->st, sizeof(State), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return POU_OK;
}

template <typename Fld>
pou_status write_field(pou_ctx* c, size_t off, const Fld& v) {
  // the value is copied from pageable memory, which completes before return
  CK(cudaMemcpyAsync(reinterpret_cast<char*>(c->st) + off, &v, sizeof(Fld), cudaMemcpyHostToDevice,
                     c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return POU_OK;
}

template <typename T>
T* tp(void* p) {
  return reinterpret_cast<T*>(p);
}

// Relative pivot below which the Gram matrix counts as singular: a few
// hundred ulps of the Gram's own precision.
double pivot_tol(const pou_ctx* c) { return c->dt == 0 ? 1e-13 : 1e-6; }

// FP32 form: a trial Gram matrix further than this from the identity is
// orthonormalised a second time (its Cholesky-QR loses about
// cond(S) * (FP32 Gram error) of orthogonality).  The FP64 form keeps the
// single Cholesky-QR of the method.
constexpr double kReorthThreshold = 0.02;
double reorth_thr(const pou_ctx* c) { return c->dt == 1 ? kReorthThreshold : 0.0; }

// Stencil scale applied in the working type, and the FP64 per-axis kinetic
// coefficients: -1/2 Lap_h = -1/2 sum_a e_a / (h_a^2 [12 for order 4]).
double stencil_scale(const pou_ctx* c, int a) {
  const double h2 = c->h[a] * c->h[a];
  return c->cfg.stencil_order == 2 ? 1.0 / h2 : 1.0 / (12.0 * h2);
}

// Projections of the block the next H-apply reads and its nonlocal part
// (sel 1: the trial slot, with the step's part against the current pair when
// step is set; sel 2: the current slot; sel 0: an explicit block).  No-op
// without projectors.
template <typename T>
void enqueue_nonlocal(pou_ctx* c, int sel, const T* explicit_block, int gate, ApplyArgs<T>* aa, bool step) {
  if (c->P == 0) return;
  NlArgs<T> n{};
  n.st = sel == 0 ? nullptr : c->st;
  n.tab = c->nlt;
  for (int k = 0; k < 2; ++k) {
    n.X[k] = sel == 0 ? explicit_block : tp<T>(c->W[k]);
    n.C[k] = sel == 0 ? c->nlCe : c->nlC[k];
  }
  n.sel = sel;
  n.nl = tp<T>(c->nl);
  n.nls = (sel == 1 && step) ? tp<T>(c->nls) : nullptr;
  n.gate = gate;
  n.N = c->N;
  n.dV = c->dV;
  launch_nl_project<T>(n, c->nl_part, c->stream);
  launch_nl_apply<T>(n, c->stream);
  aa->nl = tp<T>(c->nl);
  aa->nls = n.nls;
}

// 1 when the three per-axis stencil scales are equal, so that the H-apply may
// keep one kinetic sum for all axes (the FP64 coefficients are then equal).
int cubic_scales(const pou_ctx* c) {
  return stencil_scale(c, 0) == stencil_scale(c, 1) && stencil_scale(c, 1) == stencil_scale(c, 2) ? 1 : 0;
}

// Second Cholesky-QR pass on the block just written to W[1-cur], gated on
// st->reorth (FP32 form only).
template <typename T>
void enqueue_second_orth(pou_ctx* c, int soft_limit) {
  if (c->dt != 1) return;
  cudaStream_t s = c->stream;
  GramArgs<T> g{};
  g.st = c->st;
  for (int k = 0; k < 2; ++k) g.W[k] = tp<T>(c->W[k]);
  g.src_trial_slot = 1;
  g.gate = 1;
  g.ng = c->ng;
  g.N = c->N;
  g.split = c->split;
  g.tf32_single = c->tf32_single;
  launch_gram<T>(g, s);
  int nsplit, npair;
  i64 chunk;
  gram_layout<T>(c->ng, c->N, false, &nsplit, &npair, &chunk);
  GramReduceArgs r{};
  r.st = c->st;
  r.split = c->split;
  r.nsplit = nsplit;
  r.npair = npair;
  r.ST = gram_supertile<T>();
  r.N = c->N;
  r.dV = c->dV;
  r.S = c->S;
  r.gate = 1;
  launch_gram_reduce(r, s);
  launch_cholinv(c->st, c->S, c->Rinv, c->N, nullptr, c->st, pivot_tol(c), -1.0, s, false, soft_limit);
  RotArgs<T> ra{};
  ra.rimg = c->rimg;
  ra.st = c->st;
  for (int k = 0; k < 2; ++k) {
    ra.Wout[k] = tp<T>(c->W[k]);
    ra.rho[k] = c->rho[k];
  }
  ra.Rinv = c->Rinv;
  ra.src_trial_slot = 1;
  ra.gate = 1;
  ra.sr_salt = 1;
  ra.ng = c->ng;
  ra.N = c->N;
  launch_rotate<T>(ra, s);
}

// Algorithm M, Sec. 3.3: when the controller has flagged it (State::diag_now),
// Sigma = <W^T H W> of the current pair, P^T Sigma P = Gamma, W <- W P, and
// HW and the per-orbital sums of the rotated pair are rebuilt.  Every kernel
// is gated on the flag, so the sequence costs nothing on other steps.
template <typename T>
void enqueue_diag(pou_ctx* c) {
  cudaStream_t s = c->stream;
  GramArgs<T> g{};
  g.st = c->st;
  for (int k = 0; k < 2; ++k) {
    g.W[k] = tp<T>(c->W[k]);
    g.HW[k] = tp<T>(c->HW[k]);
  }
  g.src_cur_pair = 1;
  g.gate = 2;
  g.ng = c->ng;
  g.N = c->N;
  g.split = c->split;
  g.tf32_single = c->tf32_single;
  launch_gram<T>(g, s);
  int nsplit, npair;
  i64 chunk;
  gram_layout<T>(c->ng, c->N, true, &nsplit, &npair, &chunk);
  GramReduceArgs r{};
  r.st = c->st;
  r.split = c->split;
  r.nsplit = nsplit;
  r.npair = npair;
  r.ST = gram_supertile<T>();
  r.N = c->N;
  r.general = 1;
  r.dV = c->dV;
  r.S = c->S;
  r.gate = 2;
  launch_gram_reduce(r, s);
  launch_eigh(c->st, c->S, c->Rinv, c->evec, c->sigma[0], c->sigma[1], c->N, s);
  RotArgs<T> ra{};
  ra.rimg = c->rimg;
  ra.st = c->st;
  for (int k = 0; k < 2; ++k) ra.Wout[k] = tp<T>(c->W[k]);
  ra.Rinv = c->Rinv;
  ra.src_cur_slot = 1;
  ra.gate = 2;
  ra.sr_salt = 2;
  ra.general = 1;
  ra.ng = c->ng;
  ra.N = c->N;
  launch_rotate<T>(ra, s);
  ApplyArgs<T> aa{};
  aa.st = c->st;
  for (int k = 0; k < 2; ++k) {
    aa.W[k] = tp<T>(c->W[k]);
    aa.HW[k] = tp<T>(c->HW[k]);
    aa.V[k] = tp<T>(c->V[k]);
    aa.sigma[k] = c->sigma[k];
  }
  aa.mode = 3;
  enqueue_nonlocal<T>(c, 2, nullptr, 2, &aa, false);
  aa.tilepart = c->tilepart;
  aa.out_scale = T(1);
  aa.N = c->N;
  aa.nx = c->nx;
  aa.ny = c->ny;
  aa.nz = c->nz;
  aa.ihx2 = (T)stencil_scale(c, 0);
  aa.ihy2 = (T)stencil_scale(c, 1);
  aa.ihz2 = (T)stencil_scale(c, 2);
  aa.cubic = cubic_scales(c);
  int ntile = 0;
  launch_apply_h<T>(aa, c->cfg.stencil_order, s, &ntile);
  CtrlArgs k{};
  k.st = c->st;
  k.fp32 = c->dt == 1 ? 1 : 0;
  for (int q = 0; q < 2; ++q) {
    k.sigma[q] = c->sigma[q];
    k.part[q] = c->part[q];
  }
  k.tilepart = c->tilepart;
  k.ntile = ntile;
  k.epart = c->epart;
  k.neblk = 0;
  k.N = c->N;
  k.refresh = 1;
  k.dV = c->dV;
  for (int q = 0; q < 3; ++q) k.kc[q] = -0.5 * stencil_scale(c, q);
  for (int q = 0; q < 2; ++q) k.nlC[q] = c->P ? c->nlC[q] : nullptr;
  k.P = c->P;
  launch_control(k, s);
}

// ------------------------------------------------------------- one pass
// OptM-QR (Sec. 3.1): on the first pass of a step, Sigma = <W^T HW> of the
// current pair, Z = HW - W Sigma with its sums, and the step's tau and ||Z||^2.
template <typename T>
void enqueue_direction_full(pou_ctx* c) {
  cudaStream_t s = c->stream;
  GramArgs<T> g{};
  g.st = c->st;
  for (int k = 0; k < 2; ++k) {
    g.W[k] = tp<T>(c->W[k]);
    g.HW[k] = tp<T>(c->HW[k]);
  }
  g.src_cur_pair = 1;
  g.gate = 4;
  g.ng = c->ng;
  g.N = c->N;
  g.split = c->split;
  g.tf32_single = c->tf32_single;
  launch_gram<T>(g, s);
  int nsplit, npair;
  i64 chunk;
  gram_layout<T>(c->ng, c->N, true, &nsplit, &npair, &chunk);
  GramReduceArgs r{};
  r.st = c->st;
  r.split = c->split;
  r.nsplit = nsplit;
  r.npair = npair;
  r.ST = gram_supertile<T>();
  r.N = c->N;
  r.general = 1;
  r.dV = c->dV;
  r.S = c->S;
  r.gate = 4;
  launch_gram_reduce(r, s);
  DirArgs<T> d{};
  d.st = c->st;
  for (int k = 0; k < 2; ++k) {
    d.W[k] = tp<T>(c->W[k]);
    d.HW[k] = tp<T>(c->HW[k]);
    d.Z[k] = tp<T>(c->Z[k]);
  }
  d.Sig = c->S;
  d.opart = c->dir_opart;
  d.bpart = c->dir_bpart;
  d.ng = c->ng;
  d.N = c->N;
  launch_direction<T>(d, s);
  DirCtrlArgs k{};
  k.st = c->st;
  k.opart = c->dir_opart;
  k.bpart = c->dir_bpart;
  k.dpart = c->dir_dpart;
  k.nblk = direction_grid(c->ng);
  k.N = c->N;
  k.dV = c->dV;
  k.tau0 = c->tau0;
  k.tau_min = c->cfg.tau_min;
  k.tau_max = c->cfg.tau_max;
  k.bb_variant = c->cfg.bb_variant;
  launch_direction_control(k, s);
}

// Conjugate-gradient solver: on the first pass of a step, the directions D,
// the H-apply of D for the Newton steps, and the per-orbital steps.
template <typename T>
void enqueue_cg(pou_ctx* c) {
  cudaStream_t s = c->stream;
  CgArgs<T> g{};
  g.st = c->st;
  for (int k = 0; k < 2; ++k) {
    g.W[k] = tp<T>(c->W[k]);
    g.HW[k] = tp<T>(c->HW[k]);
    g.D[k] = tp<T>(c->D[k]);
    g.Zs[k] = tp<T>(c->Zs[k]);
    g.sigma[k] = c->sigma[k];
  }
  g.coef = c->cg_coef;
  g.opart = c->cg_opart;
  g.ng = c->ng;
  g.N = c->N;
  g.nch = cg_chunks(c->ng);
  CgCtrlArgs k{};
  k.st = c->st;
  k.opart = c->cg_opart;
  k.nch = g.nch;
  k.N = c->N;
  k.coef = c->cg_coef;
  for (int q = 0; q < 2; ++q) k.sigma[q] = c->sigma[q];
  k.tilepart = c->tilepart;
  k.tfac = c->tfac;
  k.dpart = c->dir_dpart;
  k.dV = c->dV;
  k.tau0 = c->tau0;
  k.tau_min = c->cfg.tau_min;
  k.tau_max = c->cfg.tau_max;
  launch_cg_dots<T>(g, s);
  launch_cg_beta(k, s);
  launch_cg_form<T>(g, s);
  ApplyArgs<T> aa{};
  aa.st = c->st;
  for (int q = 0; q < 2; ++q) {
    aa.W[q] = tp<T>(c->D[q]);
    aa.HW[q] = nullptr;
    aa.V[q] = tp<T>(c->V[q]);
    aa.sigma[q] = c->sigma[q];
  }
  aa.mode = 4;
  aa.tilepart = c->tilepart;
  aa.out_scale = T(1);
  aa.N = c->N;
  aa.nx = c->nx;
  aa.ny = c->ny;
  aa.nz = c->nz;
  aa.ihx2 = (T)stencil_scale(c, 0);
  aa.ihy2 = (T)stencil_scale(c, 1);
  aa.ihz2 = (T)stencil_scale(c, 2);
  aa.cubic = cubic_scales(c);
  int ntile = 0;
  launch_apply_h<T>(aa, c->cfg.stencil_order, s, &ntile);
  k.ntile = ntile;
  launch_cg_step(k, s);
}

template <typename T>
void enqueue_pass(pou_ctx* c) {
  cudaStream_t s = c->stream;
  if (c->cfg.n_diag > 0) enqueue_diag<T>(c);
  const bool full = c->cfg.direction == 1;
  const bool cg = c->cfg.solver == 1;
  if (full) enqueue_direction_full<T>(c);
  if (cg) enqueue_cg<T>(c);
  // the trial kernels take a materialised direction (OptM-QR's Z, the CG
  // directions D) with a zero sigma, or Opt-Par's (W, HW, sigma)
  void* const* dirb = full ? c->Z : (cg ? c->D : c->HW);
  const bool mat = full || cg;
  // trial block Wt = W - tau Z from the current pair, Gram matrix
  // the trial point (1 + tau sigma_ii) w - tau hw of Opt-Par; OptM-QR hands
  // the kernels Z and a zero sigma, so that they form w - tau z
  GramArgs<T> g{};
  g.st = c->st;
  for (int k = 0; k < 2; ++k) {
    g.W[k] = tp<T>(c->W[k]);
    g.HW[k] = tp<T>(dirb[k]);
    g.sigma[k] = mat ? c->zero_sigma : c->sigma[k];
  }
  g.tfac = c->tfac;
  g.trial = 1;
  g.gate = 3;  // skipped on the intermediate steps of Algorithm M (n_org > 1)
  g.ng = c->ng;
  g.N = c->N;
  g.split = c->split;
  g.tf32_single = c->tf32_single;
  launch_gram<T>(g, s);
  int nsplit, npair;
  i64 chunk;
  gram_layout<T>(c->ng, c->N, false, &nsplit, &npair, &chunk);
  GramReduceArgs r{};
  r.st = c->st;
  r.gate = 3;
  r.split = c->split;
  r.nsplit = nsplit;
  r.npair = npair;
  r.ST = gram_supertile<T>();
  r.N = c->N;
  r.general = 0;
  r.dV = c->dV;
  r.S = c->S;
  // Diagonal of the trial Gram matrix: the squared norm of the very column
  // the rotation scales by R_jj.  Both rotations form the trial point with
  // the FP64 coefficients (the FP32 one as a double-float, hi + lo), so the
  // diagonal is the FP64 norm of (1 + tau sigma) w - tau hw from the
  // H-apply sums.
  r.trial = mat ? 2 : 1;
  r.dpart = c->dir_dpart;
  r.tfac = c->tfac;
  for (int k = 0; k < 2; ++k) {
    r.sigma[k] = c->sigma[k];
    r.part[k] = c->part[k];
  }
  launch_gram_reduce(r, s);
  // Cholesky and R^-1 in FP64 (R^-1 = I on the intermediate steps of Algorithm M)
  launch_cholinv(c->st, c->S, c->Rinv, c->N, nullptr, c->st, pivot_tol(c), reorth_thr(c), s, true,
                 c->cfg.max_backtrack);
  // W_new = Wt R^-1 and rho into the other pair
  RotArgs<T> ra{};
  ra.rimg = c->rimg;
  ra.st = c->st;
  for (int k = 0; k < 2; ++k) {
    ra.W[k] = tp<T>(c->W[k]);
    ra.HW[k] = tp<T>(dirb[k]);
    ra.sigma[k] = mat ? c->zero_sigma : c->sigma[k];
    ra.Wout[k] = tp<T>(c->W[k]);
    ra.rho[k] = c->rho[k];
  }
  ra.Rinv = c->Rinv;
  ra.trial = 1;
  ra.tfac = c->tfac;
  ra.ng = c->ng;
  ra.N = c->N;
  launch_rotate<T>(ra, s);
  enqueue_second_orth<T>(c, c->cfg.max_backtrack);
  // Hartree potential, V and the energy sums of the trial density
  PotArgs<T> pa{};
  pa.st = c->st;
  for (int k = 0; k < 2; ++k) {
    pa.rho[k] = c->rho[k];
    pa.V64[k] = c->V64[k];
    pa.V[k] = tp<T>(c->V[k]);
  }
  pa.vext = c->vext;
  pa.work = c->work;
  pa.epart = c->epart;
  pa.dv_out = tp<T>(c->dv);
  pa.hartree = c->cfg.hartree;
  pa.exchange = c->cfg.exchange;
  const int neblk = launch_potential<T>(c->fft, pa, s);
  // H-apply of the trial with the sums against the current pair
  ApplyArgs<T> aa{};
  aa.st = c->st;
  for (int k = 0; k < 2; ++k) {
    aa.W[k] = tp<T>(c->W[k]);
    aa.HW[k] = tp<T>(c->HW[k]);
    aa.V[k] = tp<T>(c->V[k]);
    aa.sigma[k] = c->sigma[k];
  }
  aa.mode = 0;
  aa.dV = tp<T>(c->dv);
  enqueue_nonlocal<T>(c, 1, nullptr, 0, &aa, true);
  aa.tilepart = c->tilepart;
  aa.out_scale = T(1);
  aa.N = c->N;
  aa.nx = c->nx;
  aa.ny = c->ny;
  aa.nz = c->nz;
  aa.ihx2 = (T)stencil_scale(c, 0);
  aa.ihy2 = (T)stencil_scale(c, 1);
  aa.ihz2 = (T)stencil_scale(c, 2);
  aa.cubic = cubic_scales(c);
  int ntile = 0;
  launch_apply_h<T>(aa, c->cfg.stencil_order, s, &ntile);
  // accept / reject
  CtrlArgs k{};
  k.st = c->st;
  k.fp32 = c->dt == 1 ? 1 : 0;
  k.hist_E = c->hist_E;
  k.hist_tau = c->hist_tau;
  for (int q = 0; q < 2; ++q) {
    k.sigma[q] = c->sigma[q];
    k.part[q] = c->part[q];
  }
  k.tilepart = c->tilepart;
  k.ntile = ntile;
  k.epart = c->epart;
  k.neblk = neblk;
  k.N = c->N;
  k.init = 0;
  k.dV = c->dV;
  k.rho1 = c->cfg.rho1;
  k.delta = c->cfg.delta;
  k.eta = c->cfg.eta;
  k.tau0 = c->tau0;
  k.tau_min = c->cfg.tau_min;
  k.tau_max = c->cfg.tau_max;
  k.bb_variant = c->cfg.bb_variant;
  k.max_backtrack = c->cfg.max_backtrack;
  k.tfac = c->cfg.tau_mode == 1 ? c->tfac : nullptr;
  k.n_diag = c->cfg.n_diag;
  k.n_org = c->cfg.n_org;
  for (int q = 0; q < 3; ++q) k.kc[q] = -0.5 * stencil_scale(c, q);
  for (int q = 0; q < 2; ++q) k.nlC[q] = c->P ? c->nlC[q] : nullptr;
  k.P = c->P;
  launch_control(k, s);
}

// Orthonormalise the block staged in W[0], build rho, V, HW, E (the initialisation of Algorithm B).
template <typename T>
pou_status init_from_staged(pou_ctx* c) {
  cudaStream_t s = c->stream;
  State hs{};
  hs.cur = 0;
  hs.done = 0;
  CK(cudaMemcpyAsync(c->st, &hs, sizeof(State), cudaMemcpyHostToDevice, s));
  GramArgs<T> g{};
  g.A = tp<T>(c->W[0]);
  g.trial = 0;
  g.ng = c->ng;
  g.N = c->N;
  g.split = c->split;
  g.tf32_single = c->tf32_single;
  launch_gram<T>(g, s);
  int nsplit, npair;
  i64 chunk;
  gram_layout<T>(c->ng, c->N, false, &nsplit, &npair, &chunk);
  GramReduceArgs r{};
  r.split = c->split;
  r.nsplit = nsplit;
  r.npair = npair;
  r.ST = gram_supertile<T>();
  r.N = c->N;
  r.dV = c->dV;
  r.S = c->S;
  launch_gram_reduce(r, s);
  launch_cholinv(c->st, c->S, c->Rinv, c->N, c->info, c->st, pivot_tol(c), reorth_thr(c), s);
  RotArgs<T> ra{};
  ra.rimg = c->rimg;
  ra.st = c->st;
  for (int k = 0; k < 2; ++k) {
    ra.Wout[k] = tp<T>(c->W[k]);
    ra.rho[k] = c->rho[k];
  }
  ra.A = tp<T>(c->W[0]);
  ra.Rinv = c->Rinv;
  ra.trial = 0;
  ra.ng = c->ng;
  ra.N = c->N;
  launch_rotate<T>(ra, s);
  enqueue_second_orth<T>(c, -1);
  PotArgs<T> pa{};
  pa.st = c->st;
  for (int k = 0; k < 2; ++k) {
    pa.rho[k] = c->rho[k];
    pa.V64[k] = c->V64[k];
    pa.V[k] = tp<T>(c->V[k]);
  }
  pa.vext = c->vext;
  pa.work = c->work;
  pa.epart = c->epart;
  pa.hartree = c->cfg.hartree;
  pa.exchange = c->cfg.exchange;
  const int neblk = launch_potential<T>(c->fft, pa, s);
  ApplyArgs<T> aa{};
  aa.st = c->st;
  for (int k = 0; k < 2; ++k) {
    aa.W[k] = tp<T>(c->W[k]);
    aa.HW[k] = tp<T>(c->HW[k]);
    aa.V[k] = tp<T>(c->V[k]);
    aa.sigma[k] = c->sigma[k];
  }
  aa.mode = 1;
  enqueue_nonlocal<T>(c, 1, nullptr, 0, &aa, false);
  aa.tilepart = c->tilepart;
  aa.out_scale = T(1);
  aa.N = c->N;
  aa.nx = c->nx;
  aa.ny = c->ny;
  aa.nz = c->nz;
  aa.ihx2 = (T)stencil_scale(c, 0);
  aa.ihy2 = (T)stencil_scale(c, 1);
  aa.ihz2 = (T)stencil_scale(c, 2);
  aa.cubic = cubic_scales(c);
  int ntile = 0;
  launch_apply_h<T>(aa, c->cfg.stencil_order, s, &ntile);
  CtrlArgs k{};
  k.st = c->st;
  k.fp32 = c->dt == 1 ? 1 : 0;
  k.hist_E = c->hist_E;
  k.hist_tau = c->hist_tau;
  for (int q = 0; q < 2; ++q) {
    k.sigma[q] = c->sigma[q];
    k.part[q] = c->part[q];
  }
  k.tilepart = c->tilepart;
  k.ntile = ntile;
  k.epart = c->epart;
  k.neblk = neblk;
  k.N = c->N;
  k.init = 1;
  k.dV = c->dV;
  k.tau0 = c->tau0;
  k.tfac = c->cfg.tau_mode == 1 ? c->tfac : nullptr;
  for (int q = 0; q < 3; ++q) k.kc[q] = -0.5 * stencil_scale(c, q);
  for (int q = 0; q < 2; ++q) k.nlC[q] = c->P ? c->nlC[q] : nullptr;
  k.P = c->P;
  launch_control(k, s);
  pou_status e = check_launch(c, "initialisation kernels");
  if (e != POU_OK) return e;
  State out;
  e = read_state(c, &out);
  if (e != POU_OK) return e;
  if (out.status == POU_ENOTSPD)
    return fail(c, POU_ENOTSPD, "initial orbitals are rank deficient (pivot %d)", out.chol_info);
  if (out.status == POU_ENAN) return fail(c, POU_ENAN, "initial energy is not finite");
  c->have_orbitals = true;
  return POU_OK;
}

pou_status stage_block(pou_ctx* c, const void* U, int dtype, int on_device, void* dst) {
  const size_t n = (size_t)c->N * (size_t)c->ng;
  if (on_device && !device_accessible(U)) return fail(c, POU_EINVAL, "on_device = 1 but not device memory");
  if (dtype == c->dt) {
    CK(cudaMemcpyAsync(dst, U, n * c->esz, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                       c->stream));
    return POU_OK;
  }
  if (on_device) {
    if (dtype == POU_DT_F64)
      launch_convert_f64_f32(static_cast<const double*>(U), static_cast<float*>(dst), (i64)n, c->stream);
    else
      launch_convert_f32_f64(static_cast<const float*>(U), static_cast<double*>(dst), (i64)n, c->stream);
    return check_launch(c, "convert");
  }
  // host data of the other type: one orbital at a time through the FFT work buffer
  const size_t in_esz = dtype == POU_DT_F64 ? 8 : 4;
  for (int i = 0; i < c->N; ++i) {
    const char* src = static_cast<const char*>(U) + (size_t)i * c->ng * in_esz;
    CK(cudaMemcpyAsync(c->work, src, c->ng * in_esz, cudaMemcpyHostToDevice, c->stream));
    char* d = static_cast<char*>(dst) + (size_t)i * c->ng * c->esz;
    if (dtype == POU_DT_F64)
      launch_convert_f64_f32(reinterpret_cast<const double*>(c->work), reinterpret_cast<float*>(d), c->ng,
                             c->stream);
    else
      launch_convert_f32_f64(reinterpret_cast<const float*>(c->work), reinterpret_cast<double*>(d), c->ng,
                             c->stream);
  }
  return check_launch(c, "convert");
}

pou_status unstage_block(pou_ctx* c, const void* src, void* U, int dtype, int on_device) {
  const size_t n = (size_t)c->N * (size_t)c->ng;
  if (on_device && !device_accessible(U)) return fail(c, POU_EINVAL, "on_device = 1 but not device memory");
  if (dtype == c->dt) {
    CK(cudaMemcpyAsync(U, src, n * c->esz, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                       c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return POU_OK;
  }
  if (on_device) {
    if (c->dt == 0)
      launch_convert_f64_f32(static_cast<const double*>(src), static_cast<float*>(U), (i64)n, c->stream);
    else
      launch_convert_f32_f64(static_cast<const float*>(src), static_cast<double*>(U), (i64)n, c->stream);
    pou_status e = check_launch(c, "convert");
    if (e != POU_OK) return e;
    CK(cudaStreamSynchronize(c->stream));
    return POU_OK;
  }
  const size_t out_esz = dtype == POU_DT_F64 ? 8 : 4;
  for (int i = 0; i < c->N; ++i) {
    const char* sp = static_cast<const char*>(src) + (size_t)i * c->ng * c->esz;
    if (c->dt == 0)
      launch_convert_f64_f32(reinterpret_cast<const double*>(sp), reinterpret_cast<float*>(c->work), c->ng,
                             c->stream);
    else
      launch_convert_f32_f64(reinterpret_cast<const float*>(sp), reinterpret_cast<double*>(c->work), c->ng,
                             c->stream);
    char* d = static_cast<char*>(U) + (size_t)i * c->ng * out_esz;
    CK(cudaMemcpyAsync(d, c->work, c->ng * out_esz, cudaMemcpyDeviceToHost, c->stream));
  }
  CK(cudaStreamSynchronize(c->stream));
  return check_launch(c, "convert");
}

pou_status ensure_eval_buffers(pou_ctx* c) {
  if (c->rho_e) return POU_OK;
  const size_t blk = (size_t)c->N * c->ng * c->esz;
  DALLOC(c->ublock, blk);
  DALLOC(c->gblock, blk);
  DALLOC(c->rho_e, c->ng * sizeof(double));
  DALLOC(c->V64_e, c->ng * sizeof(double));
  if (c->dt == 1)
    DALLOC(c->V_e, c->ng * sizeof(float));
  else
    c->V_e = c->V64_e;
  return POU_OK;
}

// rho(U), V(rho) and the energy sums of an arbitrary block on the device
template <typename T>
pou_status eval_block(pou_ctx* c, const T* U, T* HUout, T scale, pou_energy_terms* terms) {
  cudaStream_t s = c->stream;
  launch_density<T>(U, c->ng, c->N, c->rho_e, s);
  PotArgs<T> pa{};
  pa.rho_x = c->rho_e;
  pa.V64_x = c->V64_e;
  pa.V_x = tp<T>(c->V_e);
  pa.vext = c->vext;
  pa.work = c->work;
  pa.epart = c->epart;
  pa.hartree = c->cfg.hartree;
  pa.exchange = c->cfg.exchange;
  const int neblk = launch_potential<T>(c->fft, pa, s);
  ApplyArgs<T> aa{};
  aa.W[0] = U;
  aa.HW[0] = HUout;
  aa.V[0] = tp<T>(c->V_e);
  aa.mode = 2;
  enqueue_nonlocal<T>(c, 0, U, 0, &aa, false);
  aa.tilepart = c->tilepart;
  aa.out_scale = scale;
  aa.N = c->N;
  aa.nx = c->nx;
  aa.ny = c->ny;
  aa.nz = c->nz;
  aa.ihx2 = (T)stencil_scale(c, 0);
  aa.ihy2 = (T)stencil_scale(c, 1);
  aa.ihz2 = (T)stencil_scale(c, 2);
  aa.cubic = cubic_scales(c);
  int ntile = 0;
  launch_apply_h<T>(aa, c->cfg.stencil_order, s, &ntile);
  pou_status e = check_launch(c, "evaluation kernels");
  if (e != POU_OK) return e;
  if (terms) {
    std::vector<double> tpart((size_t)c->N * ntile * NPT), ep((size_t)neblk * NE);
    CK(cudaMemcpyAsync(tpart.data(), c->tilepart, tpart.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(ep.data(), c->epart, ep.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    double kin = 0.0;
    for (int i = 0; i < c->N; ++i) {
      double si[3] = {0.0, 0.0, 0.0};
      for (int j = 0; j < ntile; ++j)
        for (int q = 0; q < 3; ++q) si[q] += tpart[((size_t)i * ntile + j) * NPT + P_KX + q];
      for (int q = 0; q < 3; ++q) kin += -0.5 * stencil_scale(c, q) * si[q];
    }
    double se[NE] = {0, 0, 0};
    for (int b = 0; b < neblk; ++b)
      for (int q = 0; q < NE; ++q) se[q] += ep[(size_t)b * NE + q];
    double enl = 0.0;
    if (c->P) {
      std::vector<double> Ce((size_t)c->N * c->P);
      CK(cudaMemcpy(Ce.data(), c->nlCe, Ce.size() * sizeof(double), cudaMemcpyDeviceToHost));
      for (double v : Ce) enl += v * v;
    }
    terms->kinetic = F_OCC * c->dV * kin;
    terms->external = c->dV * se[E_EXT] + F_OCC * enl;
    terms->hartree = 0.5 * c->dV * se[E_H];
    terms->exchange = c->dV * se[E_X];
    terms->total = terms->kinetic + terms->external + terms->hartree + terms->exchange;
  }
  return POU_OK;
}

pou_status cur_index(pou_ctx* c, int* cur) {
  State hs;
  pou_status e = read_state(c, &hs);
  if (e != POU_OK) return e;
  *cur = hs.cur;
  return POU_OK;
}

pou_status build_graph(pou_ctx* c) {
  if (c->graph) return POU_OK;
  cudaGraph_t g;
  CK(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
  const long long before = g_launches;
  if (c->dt == 0)
    enqueue_pass<double>(c);
  else
    enqueue_pass<float>(c);
  cudaError_t e = cudaStreamEndCapture(c->stream, &g);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(c, POU_ECUDA, "graph capture: %s", cudaGetErrorString(e));
  }
  c->kernels_per_pass = (int)(g_launches - before);
  g_launches = before;  // captured launches are counted when replayed
  e = cudaGraphInstantiate(&c->graph, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    c->graph = nullptr;
    return fail(c, POU_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
  }
  return POU_OK;
}

pou_status run_passes(pou_ctx* c, int npass) {
  if (c->prof) {
    // profiled passes are launched one kernel at a time between events
    for (int i = 0; i < npass; ++i) {
      if (c->dt == 0)
        enqueue_pass<double>(c);
      else
        enqueue_pass<float>(c);
      if (c->prof->used > 60000) c->prof->collect();
    }
    return check_launch(c, "pass");
  }
  pou_status e = build_graph(c);
  if (e != POU_OK) return e;
  for (int i = 0; i < npass; ++i) {
    CK(cudaGraphLaunch(c->graph, c->stream));
    g_launches += c->kernels_per_pass;
  }
  return POU_OK;
}

}  // namespace

void pou::configure_kernels() {
  static bool done = false;
  if (done) return;
  configure_rotate();
  configure_cholinv();
  configure_fft();
  configure_eigh();
  configure_apply_h();
  configure_gram_tc();
  configure_direction();
  configure_nonlocal();
  configure_rotate_tc();
  done = true;
}

// ===================================================================== C-ABI
extern "C" {

void pou_config_default(pou_config* cfg) {
  if (!cfg) return;
  std::memset(cfg, 0, sizeof(*cfg));
  cfg->n[0] = cfg->n[1] = cfg->n[2] = 32;
  cfg->L[0] = cfg->L[1] = cfg->L[2] = 10.0;
  cfg->stencil_order = 2;
  cfg->N = 4;
  cfg->precision = POU_FP64;
  cfg->hartree = 1;
  cfg->exchange = 1;
  cfg->bb_variant = 3;
  cfg->rho1 = 1e-4;
  cfg->delta = 0.1;
  cfg->eta = 0.85;
  cfg->max_backtrack = 10;
  cfg->tau0 = 0.0;
  cfg->tau_min = 1e-12;
  cfg->tau_max = 1e3;
  cfg->n_org = 1;
  cfg->n_diag = 0;
  cfg->stream = nullptr;
  cfg->direction = 0;
  cfg->tau_mode = 0;
  cfg->solver = 0;
}

static pou_status create_buffers(pou_ctx* c);

pou_status pou_create(const pou_config* cfg, pou_ctx** out) {
  if (!out) return POU_EINVAL;
  *out = nullptr;
  if (!cfg) return POU_EINVAL;
  for (int a = 0; a < 3; ++a) {
    if (cfg->n[a] < 2 || !fft_supported(cfg->n[a])) return POU_EINVAL;
    if (!(cfg->L[a] > 0.0) || !std::isfinite(cfg->L[a])) return POU_EINVAL;
  }
  if (cfg->stencil_order != 2 && cfg->stencil_order != 4) return POU_EINVAL;
  if (cfg->N < 1 || cfg->N > POU_MAX_N) return POU_EINVAL;
  if (cfg->precision != POU_FP64 && cfg->precision != POU_FP32 && cfg->precision != POU_FP32_TF32)
    return POU_EINVAL;
  if (cfg->bb_variant < 1 || cfg->bb_variant > 3) return POU_EINVAL;
  if (!(cfg->delta > 0.0 && cfg->delta < 1.0) || !(cfg->eta >= 0.0 && cfg->eta <= 1.0)) return POU_EINVAL;
  if (!(cfg->rho1 >= 0.0) || cfg->max_backtrack < 0 || cfg->max_backtrack > 60) return POU_EINVAL;
  if (!(cfg->tau_min > 0.0) || !(cfg->tau_max >= cfg->tau_min)) return POU_EINVAL;
  if (cfg->n_org < 1 || cfg->n_diag < 0) return POU_EINVAL;
  // OptM-QR direction: Algorithm E only (no n_org, no subspace diagonalisation)
  if (cfg->direction != 0 && cfg->direction != 1) return POU_EINVAL;
  if (cfg->direction == 1 && (cfg->n_org != 1 || cfg->n_diag != 0)) return POU_EINVAL;
  // per-orbital steps and the conjugate-gradient solver: Opt-Par directions, Algorithm E
  if (cfg->tau_mode != 0 && cfg->tau_mode != 1) return POU_EINVAL;
  if (cfg->solver != 0 && cfg->solver != 1) return POU_EINVAL;
  if ((cfg->tau_mode == 1 || cfg->solver == 1) &&
      (cfg->direction != 0 || cfg->n_org != 1 || cfg->n_diag != 0))
    return POU_EINVAL;
  if (cfg->tau_mode == 1 && cfg->solver == 1) return POU_EINVAL;  // CG takes its own per-orbital steps
  // N > 128: the FP32 forms only (split or single TF32 Gram), without the subspace diagonalisation
  if (cfg->N > POU_MAX_N_FP64 && (cfg->precision == POU_FP64 || cfg->n_diag > 0)) return POU_EINVAL;
  const long long ng = (long long)cfg->n[0] * cfg->n[1] * cfg->n[2];
  if ((long long)cfg->N > ng) return POU_EINVAL;

  pou_ctx* c = new pou_ctx();  // value-initialised: every pointer starts null
  c->cfg = *cfg;
  c->dt = cfg->precision == POU_FP64 ? 0 : 1;
  c->tf32_single = cfg->precision == POU_FP32_TF32 ? 1 : 0;
  c->esz = c->dt == 0 ? 8 : 4;
  c->nx = cfg->n[0];
  c->ny = cfg->n[1];
  c->nz = cfg->n[2];
  c->N = cfg->N;
  c->ng = ng;
  for (int a = 0; a < 3; ++a) c->h[a] = cfg->L[a] / cfg->n[a];
  c->dV = c->h[0] * c->h[1] * c->h[2];
  {
    const double cc = cfg->stencil_order == 2 ? 4.0 : 16.0 / 3.0;
    double lm = 0.0;
    for (int a = 0; a < 3; ++a) lm += 0.5 * cc / (c->h[a] * c->h[a]);
    c->tau0 = cfg->tau0 > 0.0 ? cfg->tau0 : 1.0 / lm;
  }
  c->launches0 = g_launches;
  pou_status st = create_buffers(c);
  if (st != POU_OK) {
    pou_destroy(c);
    return st;
  }
  *out = c;
  return POU_OK;
}

static pou_status create_buffers(pou_ctx* c) {
  const pou_config* cfg = &c->cfg;
  configure_kernels();
  CK(cudaGetLastError());
  if (cfg->stream) {
    c->stream = static_cast<cudaStream_t>(cfg->stream);
    c->own_stream = false;
  } else {
    CK(cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking));
    c->own_stream = true;
  }
  const size_t blk = (size_t)c->N * c->ng * c->esz;
  for (int k = 0; k < 2; ++k) {
    DALLOC(c->W[k], blk);
    DALLOC(c->HW[k], blk);
    DALLOC(c->V[k], c->ng * c->esz);
    if (c->dt == 0)
      c->V64[k] = tp<double>(c->V[k]);
    else
      DALLOC(c->V64[k], c->ng * sizeof(double));
    DALLOC(c->rho[k], c->ng * sizeof(double));
    DALLOC(c->sigma[k], c->N * sizeof(double));
    DALLOC(c->part[k], (size_t)c->N * NP * sizeof(double));
  }
  DALLOC(c->vext, c->ng * sizeof(double));
  CK(cudaMemsetAsync(c->vext, 0, c->ng * sizeof(double), c->stream));
  DALLOC(c->work, c->ng * sizeof(double2));
  // a caller's block that is not aligned takes a kernel with narrower
  // accesses and another tile shape: room for every layout
  c->ntile = 0;
  for (int align = 0; align <= 2; ++align)
    c->ntile = std::max(c->ntile, apply_h_ntile(c->nx, c->ny, c->nz, c->N, (int)c->esz, nullptr, align));
  DALLOC(c->tilepart, (size_t)c->N * c->ntile * NPT * sizeof(double));
  c->neblk_max = (int)std::max<long long>((long long)num_sms() * 4, (long long)c->nz * c->ny);
  DALLOC(c->epart, (size_t)c->neblk_max * NE * sizeof(double));
  DALLOC(c->S, (size_t)c->N * c->N * sizeof(double));
  DALLOC(c->Rinv, (size_t)c->N * c->N * sizeof(double));
  {
    int nsplit, npair;
    i64 chunk;
    int ST;
    // the larger of the symmetric Gram's and the general product's (Sigma) layouts
    size_t elems = 0;
    for (int general = 0; general < 2; ++general) {
      if (c->dt == 0) {
        gram_layout<double>(c->ng, c->N, general != 0, &nsplit, &npair, &chunk);
        ST = gram_supertile<double>();
      } else {
        gram_layout<float>(c->ng, c->N, general != 0, &nsplit, &npair, &chunk);
        ST = gram_supertile<float>();
      }
      elems = std::max(elems, (size_t)nsplit * npair * ST * ST);
    }
    c->split_elems = elems;
    DALLOC(c->split, c->split_elems * sizeof(double));
  }
  if (c->dt == 1 && c->N > 128) DALLOC(c->rimg, rotate_rimg_bytes(c->N));
  DALLOC(c->evec, (size_t)c->N * c->N * sizeof(double));
  DALLOC(c->dv, c->ng * c->esz);
  if (cfg->direction == 1) {
    DALLOC(c->Z[0], blk);
    DALLOC(c->Z[1], blk);
    const int dg = direction_grid(c->ng);
    DALLOC(c->dir_opart, (size_t)dg * c->N * 3 * sizeof(double));
    DALLOC(c->dir_bpart, (size_t)dg * 3 * sizeof(double));
  }
  if (cfg->direction == 1 || cfg->solver == 1) {
    DALLOC(c->dir_dpart, (size_t)c->N * 3 * sizeof(double));
    DALLOC(c->zero_sigma, (size_t)c->N * sizeof(double));
    CK(cudaMemsetAsync(c->zero_sigma, 0, (size_t)c->N * sizeof(double), c->stream));
  }
  if (cfg->tau_mode == 1 || cfg->solver == 1) DALLOC(c->tfac, (size_t)c->N * sizeof(double));
  if (cfg->solver == 1) {
    for (int k = 0; k < 2; ++k) {
      DALLOC(c->D[k], blk);
      DALLOC(c->Zs[k], blk);
    }
    DALLOC(c->cg_opart, (size_t)c->N * cg_chunks(c->ng) * CG_NS * sizeof(double));
    DALLOC(c->cg_coef, (size_t)c->N * 2 * sizeof(double));
  }
  DALLOC(c->st, sizeof(State));
  CK(cudaMemsetAsync(c->st, 0, sizeof(State), c->stream));
  DALLOC(c->hist_E, HIST_MAX * sizeof(double));
  DALLOC(c->hist_tau, HIST_MAX * sizeof(double));
  DALLOC(c->info, sizeof(int));
  if (fft_plan_create(&c->fft, cfg->n, cfg->L) != 0)
    return fail(c, POU_ENOMEM, "FFT plan tables could not be allocated");
  CK(cudaStreamSynchronize(c->stream));
  return POU_OK;
}

void pou_destroy(pou_ctx* c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  if (c->graph) cudaGraphExecDestroy(c->graph);
  void* ptrs[] = {c->W[0], c->W[1], c->HW[0], c->HW[1], c->V[0], c->V[1], c->rho[0], c->rho[1],
                  c->sigma[0], c->sigma[1], c->part[0], c->part[1], c->vext, c->work, c->tilepart,
                  c->epart, c->S, c->Rinv, c->split, c->evec, c->dv, c->st, c->hist_E, c->hist_tau, c->info,
                  c->dR, c->dZ, c->tabs.gx, c->fpart, c->ublock, c->gblock, c->rho_e, c->V64_e, c->rimg,
                  c->Z[0], c->Z[1], c->dir_opart, c->dir_bpart, c->dir_dpart, c->zero_sigma,
                  c->tfac, c->D[0], c->D[1], c->Zs[0], c->Zs[1], c->cg_opart, c->cg_coef,
                  c->nl_mem, c->nlC[0], c->nlC[1], c->nlCe, c->nl, c->nls, c->nl_part};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (c->dt == 1) {
    if (c->V64[0]) cudaFree(c->V64[0]);
    if (c->V64[1]) cudaFree(c->V64[1]);
    if (c->V_e) cudaFree(c->V_e);
  }
  fft_plan_destroy(&c->fft);
  delete c->prof;
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  delete c;
}

const char* pou_last_error(const pou_ctx* c) { return c ? c->err.c_str() : "null context"; }

pou_status pou_set_vext(pou_ctx* c, const double* vext, int on_device) {
  if (!c || !vext) return fail(c, POU_EINVAL, "null argument");
  if (on_device && !device_accessible(vext)) return fail(c, POU_EINVAL, "on_device = 1 but not device memory");
  CK(cudaMemcpyAsync(c->vext, vext, c->ng * sizeof(double),
                     on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  c->have_orbitals = false;  // V and E of the current orbitals are stale
  return POU_OK;
}

pou_status pou_set_atoms(pou_ctx* c, int M, const double* R, const double* Z, double width) {
  ProfScope prof_scope(c);
  if (!c) return POU_EINVAL;
  if (M < 1 || !R || !Z || !(width > 0.0)) return fail(c, POU_EINVAL, "need M >= 1 atoms and width > 0");
  for (int i = 0; i < 3 * M; ++i)
    if (!std::isfinite(R[i])) return fail(c, POU_EINVAL, "non-finite atom position");
  for (int i = 0; i < M; ++i)
    if (!std::isfinite(Z[i])) return fail(c, POU_EINVAL, "non-finite atom charge");
  if (M != c->M) {
    if (c->dR) cudaFree(c->dR);
    if (c->dZ) cudaFree(c->dZ);
    if (c->tabs.gx) cudaFree(c->tabs.gx);
    if (c->fpart) cudaFree(c->fpart);
    c->dR = c->dZ = c->fpart = nullptr;
    c->tabs = AtomTables{};
    DALLOC(c->dR, (size_t)M * 3 * sizeof(double));
    DALLOC(c->dZ, (size_t)M * sizeof(double));
    const size_t nt = (size_t)M * (c->nx + c->ny + c->nz);
    // one allocation: 6 tables of doubles followed by the int windows
    char* base = nullptr;
    DALLOC(base, 2 * nt * sizeof(double) + (size_t)M * 6 * sizeof(int));
    double* d = reinterpret_cast<double*>(base);
    c->tabs.gx = d;
    c->tabs.gy = d + (size_t)M * c->nx;
    c->tabs.gz = c->tabs.gy + (size_t)M * c->ny;
    c->tabs.dgx = c->tabs.gz + (size_t)M * c->nz;
    c->tabs.dgy = c->tabs.dgx + (size_t)M * c->nx;
    c->tabs.dgz = c->tabs.dgy + (size_t)M * c->ny;
    c->tabs.win = reinterpret_cast<int*>(c->tabs.dgz + (size_t)M * c->nz);
    DALLOC(c->fpart, (size_t)M * 8 * 4 * sizeof(double));
    c->M = M;
  }
  c->hR.assign(R, R + 3 * M);
  c->hZ.assign(Z, Z + M);
  c->width = width;
  CK(cudaMemcpyAsync(c->dR, R, (size_t)M * 3 * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  CK(cudaMemcpyAsync(c->dZ, Z, (size_t)M * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  launch_atom_tables(c->dR, c->dZ, M, width, c->cfg.n, c->cfg.L, c->tabs, c->stream);
  launch_vext(c->dZ, M, c->cfg.n, c->tabs, c->vext, c->stream);
  pou_status e = check_launch(c, "atom kernels");
  if (e != POU_OK) return e;
  CK(cudaStreamSynchronize(c->stream));
  c->have_orbitals = false;
  return POU_OK;
}

static_assert(POU_MAX_PROJ == kMaxProj, "projector limit of the header and the kernels");

pou_status pou_set_projectors(pou_ctx* c, int P, const double* centres, const double* widths, const double* amps) {
  if (!c) return POU_EINVAL;
  if (P < 0 || P > POU_MAX_PROJ) return fail(c, POU_EINVAL, "need 0 <= P <= %d projectors", POU_MAX_PROJ);
  if (P > 0 && (!centres || !widths || !amps)) return fail(c, POU_EINVAL, "null projector arrays");
  if (P > 0 && c->nx > kMaxProjGrid)
    return fail(c, POU_EINVAL, "projectors need nx <= %d", kMaxProjGrid);
  if (P > 0 && c->cfg.solver == 1)
    return fail(c, POU_EINVAL, "projectors are not combined with the conjugate-gradient solver");
  for (int p = 0; p < P; ++p) {
    if (!(widths[p] > 0.0) || !std::isfinite(widths[p]) || !std::isfinite(amps[p]))
      return fail(c, POU_EINVAL, "projector %d: width must be > 0 and values finite", p);
    for (int a = 0; a < 3; ++a)
      if (!std::isfinite(centres[3 * p + a])) return fail(c, POU_EINVAL, "non-finite projector centre");
  }
  CK(cudaStreamSynchronize(c->stream));
  // the pass changes: the next iterate captures a new graph
  if (c->graph) {
    cudaGraphExecDestroy(c->graph);
    c->graph = nullptr;
  }
  void* old[] = {c->nl_mem, c->nlC[0], c->nlC[1], c->nlCe, c->nl, c->nls, c->nl_part};
  for (void* q : old)
    if (q) cudaFree(q);
  c->nl_mem = c->nl = c->nls = nullptr;
  c->nl_part = nullptr;
  c->nlC[0] = c->nlC[1] = c->nlCe = nullptr;
  c->P = 0;
  c->nlt = NlTables{};
  c->have_orbitals = false;  // E and H of the current orbitals change
  if (P == 0) return POU_OK;
  const int n[3] = {c->nx, c->ny, c->nz};
  std::vector<double> tab[3];
  std::vector<int> win((size_t)P * 6);
  for (int a = 0; a < 3; ++a) tab[a].assign((size_t)P * n[a], 0.0);
  for (int p = 0; p < P; ++p) {
    const double two_s2 = 2.0 * widths[p] * widths[p];
    for (int a = 0; a < 3; ++a) {
      const double L = c->cfg.L[a], h = c->h[a];
      double cp = centres[3 * p + a];
      cp -= L * std::floor(cp / L);  // folded into [0, L)
      double* g = tab[a].data() + (size_t)p * n[a];
      double gmax = 0.0;
      int kmax = 0;
      for (int k = 0; k < n[a]; ++k) {
        double v = 0.0;
        for (int m = -1; m <= 1; ++m) {
          const double d = k * h - cp - m * L;
          v += std::exp(-d * d / two_s2);
        }
        g[k] = v;
        if (v > gmax) {
          gmax = v;
          kmax = k;
        }
      }
      // window: the circular run around the peak where the table is >= 1e-14 of its peak
      const double thr = 1e-14 * gmax;
      int lo = 0, hi = 0;
      while (lo < n[a] - 1 && g[(kmax - lo - 1 + n[a]) % n[a]] >= thr) ++lo;
      while (hi < n[a] - 1 - lo && g[(kmax + hi + 1) % n[a]] >= thr) ++hi;
      const int len = lo + hi + 1;
      win[(size_t)p * 6 + 2 * a] = len >= n[a] ? 0 : (kmax - lo + n[a]) % n[a];
      win[(size_t)p * 6 + 2 * a + 1] = std::min(len, n[a]);
      if (a == 0)
        for (int k = 0; k < n[a]; ++k) g[k] *= amps[p];
    }
  }
  const size_t nt = (size_t)P * (n[0] + n[1] + n[2]);
  const size_t bytes = nt * sizeof(double) + nt * sizeof(float) + win.size() * sizeof(int);
  DALLOC(c->nl_mem, bytes);
  double* d = static_cast<double*>(c->nl_mem);
  float* f = reinterpret_cast<float*>(d + nt);
  int* w = reinterpret_cast<int*>(f + nt);
  size_t off = 0;
  const double* dt[3];
  const float* ft[3];
  for (int a = 0; a < 3; ++a) {
    std::vector<float> tf(tab[a].begin(), tab[a].end());
    CK(cudaMemcpy(d + off, tab[a].data(), tab[a].size() * sizeof(double), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(f + off, tf.data(), tf.size() * sizeof(float), cudaMemcpyHostToDevice));
    dt[a] = d + off;
    ft[a] = f + off;
    off += tab[a].size();
  }
  CK(cudaMemcpy(w, win.data(), win.size() * sizeof(int), cudaMemcpyHostToDevice));
  const size_t blk = (size_t)c->N * c->ng * c->esz;
  DALLOC(c->nlC[0], (size_t)c->N * P * sizeof(double));
  DALLOC(c->nlC[1], (size_t)c->N * P * sizeof(double));
  DALLOC(c->nlCe, (size_t)c->N * P * sizeof(double));
  DALLOC(c->nl, blk);
  DALLOC(c->nls, blk);
  DALLOC(c->nl_part, nl_part_bytes(c->N, P, n));
  c->nlt.P = P;
  c->nlt.nx = c->nx;
  c->nlt.ny = c->ny;
  c->nlt.nz = c->nz;
  c->nlt.gx = dt[0];
  c->nlt.gy = dt[1];
  c->nlt.gz = dt[2];
  c->nlt.gxf = ft[0];
  c->nlt.gyf = ft[1];
  c->nlt.gzf = ft[2];
  c->nlt.win = w;
  c->P = P;
  return POU_OK;
}

pou_status pou_set_orbitals(pou_ctx* c, const void* U, int dtype, int on_device) {
  ProfScope prof_scope(c);
  if (!c) return POU_EINVAL;
  if (!U || (dtype != POU_DT_F64 && dtype != POU_DT_F32)) return fail(c, POU_EINVAL, "bad orbitals argument");
  const long long before = g_launches;
  pou_status e = stage_block(c, U, dtype, on_device, c->W[0]);
  if (e != POU_OK) return e;
  e = c->dt == 0 ? init_from_staged<double>(c) : init_from_staged<float>(c);
  (void)before;
  return e;
}

pou_status pou_iterate(pou_ctx* c, int max_iter, double e_tol, double grad_tol, pou_report* rep) {
  ProfScope prof_scope(c);
  if (!c) return POU_EINVAL;
  if (!c->have_orbitals) return fail(c, POU_EINVAL, "no orbitals: call pou_set_orbitals first");
  if (max_iter < 0) return fail(c, POU_EINVAL, "max_iter < 0");
  State hs;
  pou_status e = read_state(c, &hs);
  if (e != POU_OK) return e;
  if (hs.status) return fail(c, (pou_status)hs.status, "iteration stopped earlier with status %d", hs.status);
  const State start = hs;
  const int target = hs.l + max_iter;
  double grad = -1.0;
  int conv = 0;
  if (max_iter > 0) {
    e = write_field(c, offsetof(State, target_l), target);
    if (e != POU_OK) return e;
    e = write_field(c, offsetof(State, e_tol), e_tol);
    if (e != POU_OK) return e;
    e = write_field(c, offsetof(State, converged), 0);
    if (e != POU_OK) return e;
    int l = hs.l;
    int next_grad = l + 10;
    while (true) {
      int stop_at = target;
      if (grad_tol > 0.0) stop_at = std::min(target, next_grad);
      e = write_field(c, offsetof(State, target_l), stop_at);
      if (e != POU_OK) return e;
      e = write_field(c, offsetof(State, done), 0);
      if (e != POU_OK) return e;
      // each pass accepts at most one step; rejected passes are re-issued
      while (true) {
        const int passes_before = hs.passes;
        e = run_passes(c, stop_at - l);
        if (e != POU_OK) return e;
        e = read_state(c, &hs);
        if (e != POU_OK) return e;
        l = hs.l;
        if (hs.done || l >= stop_at) break;
        if (hs.passes == passes_before) return fail(c, POU_ECUDA, "iteration made no progress");
      }
      e = check_launch(c, "iteration");
      if (e != POU_OK) return e;
      if (hs.status) break;
      if (hs.converged) {
        conv = 1;
        break;
      }
      if (grad_tol > 0.0) {
        e = pou_gradient_norm(c, &grad);
        if (e != POU_OK) return e;
        if (grad < grad_tol) {
          conv = 2;
          break;
        }
        next_grad = l + 10;
      }
      if (l >= target) break;
    }
    e = write_field(c, offsetof(State, done), 1);
    if (e != POU_OK) return e;
    e = read_state(c, &hs);
    if (e != POU_OK) return e;
  }
  if (rep) {
    rep->iterations = hs.l - start.l;
    rep->passes = hs.passes - start.passes;
    rep->backtracks = hs.backtracks - start.backtracks;
    rep->forced = hs.forced - start.forced;
    rep->total_iterations = hs.l;
    rep->converged = conv;
    rep->energy = hs.E_cur;
    rep->tau = hs.last_tau;
    rep->df_mean3 = hs.n_df >= 3 ? (hs.df[0] + hs.df[1] + hs.df[2]) / 3.0 : -1.0;
    rep->grad_norm = grad;
    rep->gram_offdiag = hs.gram_off_acc;
    rep->second_passes = hs.reorth_count - start.reorth_count;
    rep->diagonalisations = hs.diag_count - start.diag_count;
  }
  if (hs.status == POU_ENOTSPD)
    return fail(c, POU_ENOTSPD, "trial Gram matrix not positive definite (pivot %d)", hs.chol_info);
  if (hs.status == POU_ENAN) return fail(c, POU_ENAN, "non-finite trial energy");
  if ((e_tol > 0.0 || grad_tol > 0.0) && !conv) return fail(c, POU_ENOCONV, "tolerance not met in %d steps", max_iter);
  return POU_OK;
}

pou_status pou_energy(pou_ctx* c, pou_energy_terms* out) {
  if (!c || !out) return POU_EINVAL;
  if (!c->have_orbitals) return fail(c, POU_EINVAL, "no orbitals");
  State hs;
  pou_status e = read_state(c, &hs);
  if (e != POU_OK) return e;
  out->kinetic = hs.terms_cur[0];
  out->external = hs.terms_cur[1];
  out->hartree = hs.terms_cur[2];
  out->exchange = hs.terms_cur[3];
  out->total = hs.E_cur;
  return POU_OK;
}

pou_status pou_get_orbitals(pou_ctx* c, void* U, int dtype, int on_device) {
  if (!c || !U || (dtype != POU_DT_F64 && dtype != POU_DT_F32)) return fail(c, POU_EINVAL, "bad argument");
  if (!c->have_orbitals) return fail(c, POU_EINVAL, "no orbitals");
  int cur;
  pou_status e = cur_index(c, &cur);
  if (e != POU_OK) return e;
  return unstage_block(c, c->W[cur], U, dtype, on_device);
}

pou_status pou_get_density(pou_ctx* c, double* rho, int on_device) {
  if (!c || !rho) return POU_EINVAL;
  if (on_device && !device_accessible(rho)) return fail(c, POU_EINVAL, "on_device = 1 but not device memory");
  if (!c->have_orbitals) return fail(c, POU_EINVAL, "no orbitals");
  int cur;
  pou_status e = cur_index(c, &cur);
  if (e != POU_OK) return e;
  CK(cudaMemcpyAsync(rho, c->rho[cur], c->ng * sizeof(double),
                     on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return POU_OK;
}

pou_status pou_get_potential(pou_ctx* c, double* V, int on_device) {
  if (!c || !V) return POU_EINVAL;
  if (on_device && !device_accessible(V)) return fail(c, POU_EINVAL, "on_device = 1 but not device memory");
  if (!c->have_orbitals) return fail(c, POU_EINVAL, "no orbitals");
  int cur;
  pou_status e = cur_index(c, &cur);
  if (e != POU_OK) return e;
  CK(cudaMemcpyAsync(V, c->V64[cur], c->ng * sizeof(double),
                     on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return POU_OK;
}

extern "C++" {
namespace {
// Sigma = <W^T HW> of the current pair (general Gram into c->S), then the
// residual partials into c->epart.
template <typename T>
pou_status gradient_norm_impl(pou_ctx* c, int cur, double* out) {
  cudaStream_t s = c->stream;
  GramArgs<T> g{};
  g.A = tp<T>(c->W[cur]);
  g.B = tp<T>(c->HW[cur]);
  g.ng = c->ng;
  g.N = c->N;
  g.split = c->split;
  g.tf32_single = c->tf32_single;
  launch_gram<T>(g, s);
  int nsplit, npair;
  i64 chunk;
  gram_layout<T>(c->ng, c->N, true, &nsplit, &npair, &chunk);
  GramReduceArgs r{};
  r.split = c->split;
  r.nsplit = nsplit;
  r.npair = npair;
  r.ST = gram_supertile<T>();
  r.N = c->N;
  r.general = 1;
  r.dV = c->dV;
  r.S = c->S;
  launch_gram_reduce(r, s);  // S_ij = <w_i, hw_j> = Sigma_ji
  const int nb = launch_residual<T>(tp<T>(c->W[cur]), tp<T>(c->HW[cur]), c->S, c->N, c->ng, c->epart,
                                    c->neblk_max * NE, s);
  std::vector<double> h(nb);
  CK(cudaMemcpyAsync(h.data(), c->epart, nb * sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  double t = 0.0;
  for (double v : h) t += v;
  *out = std::sqrt(c->dV * t);
  return POU_OK;
}
}  // namespace
}  // extern "C++"

pou_status pou_gradient_norm(pou_ctx* c, double* out) {
  ProfScope prof_scope(c);
  if (!c || !out) return fail(c, POU_EINVAL, "bad argument");
  if (!c->have_orbitals) return fail(c, POU_EINVAL, "no orbitals set");
  int cur;
  pou_status e = cur_index(c, &cur);
  if (e != POU_OK) return e;
  return c->dt == 1 ? gradient_norm_impl<float>(c, cur, out) : gradient_norm_impl<double>(c, cur, out);
}

pou_status pou_evaluate(pou_ctx* c, const void* U, int dtype, int on_device, pou_energy_terms* out) {
  ProfScope prof_scope(c);
  if (!c || !U || !out || (dtype != POU_DT_F64 && dtype != POU_DT_F32)) return fail(c, POU_EINVAL, "bad argument");
  pou_status e = ensure_eval_buffers(c);
  if (e != POU_OK) return e;
  const void* src = U;
  if (on_device && !device_accessible(U)) return fail(c, POU_EINVAL, "on_device = 1 but not device memory");
  if (!(on_device && dtype == c->dt)) {
    e = stage_block(c, U, dtype, on_device, c->ublock);
    if (e != POU_OK) return e;
    src = c->ublock;
  }
  if (c->dt == 0) return eval_block<double>(c, static_cast<const double*>(src), nullptr, 1.0, out);
  return eval_block<float>(c, static_cast<const float*>(src), nullptr, 1.0f, out);
}

pou_status pou_backward(pou_ctx* c, const void* U, int dtype, int on_device, double g, void* dEdU,
                        double* dEdR, double* dEdZ) {
  ProfScope prof_scope(c);
  if (!c) return POU_EINVAL;
  if ((dEdR || dEdZ) && c->M == 0) return fail(c, POU_EINVAL, "atom gradients need pou_set_atoms");
  if (U && dtype != POU_DT_F64 && dtype != POU_DT_F32) return fail(c, POU_EINVAL, "bad dtype");
  pou_status e = ensure_eval_buffers(c);
  if (e != POU_OK) return e;
  const void* src;
  int out_dt = dtype;
  if (U == nullptr) {
    if (!c->have_orbitals) return fail(c, POU_EINVAL, "no orbitals");
    int cur;
    e = cur_index(c, &cur);
    if (e != POU_OK) return e;
    src = c->W[cur];
    out_dt = (dtype == POU_DT_F64 || dtype == POU_DT_F32) ? dtype : c->dt;
  } else if (on_device && dtype == c->dt) {
    if (!device_accessible(U)) return fail(c, POU_EINVAL, "on_device = 1 but not device memory");
    src = U;
  } else {
    e = stage_block(c, U, dtype, on_device, c->ublock);
    if (e != POU_OK) return e;
    src = c->ublock;
  }
  const double scale = g * 2.0 * F_OCC * c->dV;
  if (dEdU && on_device && !device_accessible(dEdU))
    return fail(c, POU_EINVAL, "on_device = 1 but dEdU is not device memory");
  const bool direct = dEdU && on_device && out_dt == c->dt;
  void* gout = dEdU ? (direct ? dEdU : c->gblock) : nullptr;
  if (c->dt == 0)
    e = eval_block<double>(c, static_cast<const double*>(src), static_cast<double*>(gout), scale, nullptr);
  else
    e = eval_block<float>(c, static_cast<const float*>(src), static_cast<float*>(gout), (float)scale, nullptr);
  if (e != POU_OK) return e;
  if (dEdU && !direct) {
    e = unstage_block(c, c->gblock, dEdU, out_dt, on_device);
    if (e != POU_OK) return e;
  }
  if (dEdR || dEdZ) {
    const int nsplit = launch_forces(c->rho_e, c->dZ, c->M, c->cfg.n, c->tabs, c->fpart, c->stream);
    e = check_launch(c, "forces");
    if (e != POU_OK) return e;
    std::vector<double> fp((size_t)c->M * nsplit * 4);
    CK(cudaMemcpyAsync(fp.data(), c->fpart, fp.size() * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    for (int I = 0; I < c->M; ++I) {
      double f[4] = {0, 0, 0, 0};
      for (int sp = 0; sp < nsplit; ++sp)
        for (int q = 0; q < 4; ++q) f[q] += fp[((size_t)I * nsplit + sp) * 4 + q];
      if (dEdR)
        for (int a = 0; a < 3; ++a) dEdR[I * 3 + a] = -g * c->dV * c->hZ[I] * f[a];
      if (dEdZ) dEdZ[I] = -g * c->dV * f[3];
    }
  } else {
    CK(cudaStreamSynchronize(c->stream));
  }
  return POU_OK;
}

pou_status pou_get_history(pou_ctx* c, double* E, double* tau, int max_entries, int* count) {
  if (!c || !count || max_entries < 0) return POU_EINVAL;
  State hs;
  pou_status e = read_state(c, &hs);
  if (e != POU_OK) return e;
  int n = std::min(std::min(hs.l, HIST_MAX), max_entries);
  if (E && n) CK(cudaMemcpyAsync(E, c->hist_E, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  if (tau && n) CK(cudaMemcpyAsync(tau, c->hist_tau, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  *count = n;
  return POU_OK;
}

// state blob: header, State, sigma/part of the current pair, history, then
// W, HW (current pair) in the bulk type, rho and V64 of the current pair
struct BlobHeader {
  char magic[8];
  int version, dt, N, nx, ny, nz;
  long long bytes;
};

pou_status pou_get_state(pou_ctx* c, void* blob, size_t* size) {
  if (!c || !size) return POU_EINVAL;
  const size_t blk = (size_t)c->N * c->ng * c->esz;
  // OptM-QR also keeps the previous iterate and its direction (its next
  // Barzilai-Borwein step differences against them)
  const size_t need = sizeof(BlobHeader) + sizeof(State) + 2 * HIST_MAX * sizeof(double) +
                      (size_t)c->N * (NP + 1) * sizeof(double) + 2 * blk + 2 * c->ng * sizeof(double) +
                      (c->cfg.direction == 1 ? 2 * blk : 0) + (c->cfg.solver == 1 ? 2 * blk : 0) +
                      (c->cfg.tau_mode == 1 ? (size_t)c->N * sizeof(double) : 0) +
                      (size_t)c->N * c->P * sizeof(double);
  if (!blob) {
    *size = need;
    return POU_OK;
  }
  if (*size < need) return fail(c, POU_EINVAL, "state buffer too small (%zu < %zu)", *size, need);
  if (!c->have_orbitals) return fail(c, POU_EINVAL, "no orbitals");
  State hs;
  pou_status e = read_state(c, &hs);
  if (e != POU_OK) return e;
  const int cur = hs.cur;
  char* p = static_cast<char*>(blob);
  BlobHeader h{};
  std::memcpy(h.magic, "POUSTATE", 8);
  h.version = 1;
  h.dt = c->dt;
  h.N = c->N;
  h.nx = c->nx;
  h.ny = c->ny;
  h.nz = c->nz;
  h.bytes = (long long)need;
  std::memcpy(p, &h, sizeof h);
  p += sizeof h;
  std::memcpy(p, &hs, sizeof hs);
  p += sizeof hs;
  CK(cudaMemcpy(p, c->hist_E, HIST_MAX * sizeof(double), cudaMemcpyDeviceToHost));
  p += HIST_MAX * sizeof(double);
  CK(cudaMemcpy(p, c->hist_tau, HIST_MAX * sizeof(double), cudaMemcpyDeviceToHost));
  p += HIST_MAX * sizeof(double);
  CK(cudaMemcpy(p, c->sigma[cur], c->N * sizeof(double), cudaMemcpyDeviceToHost));
  p += c->N * sizeof(double);
  CK(cudaMemcpy(p, c->part[cur], (size_t)c->N * NP * sizeof(double), cudaMemcpyDeviceToHost));
  p += (size_t)c->N * NP * sizeof(double);
  CK(cudaMemcpy(p, c->W[cur], blk, cudaMemcpyDeviceToHost));
  p += blk;
  CK(cudaMemcpy(p, c->HW[cur], blk, cudaMemcpyDeviceToHost));
  p += blk;
  CK(cudaMemcpy(p, c->rho[cur], c->ng * sizeof(double), cudaMemcpyDeviceToHost));
  p += c->ng * sizeof(double);
  CK(cudaMemcpy(p, c->V64[cur], c->ng * sizeof(double), cudaMemcpyDeviceToHost));
  p += c->ng * sizeof(double);
  if (c->cfg.direction == 1) {
    CK(cudaMemcpy(p, c->W[1 - cur], blk, cudaMemcpyDeviceToHost));
    p += blk;
    CK(cudaMemcpy(p, c->Z[1 - cur], blk, cudaMemcpyDeviceToHost));
    p += blk;
  }
  if (c->cfg.solver == 1) {
    CK(cudaMemcpy(p, c->D[1 - cur], blk, cudaMemcpyDeviceToHost));
    p += blk;
    CK(cudaMemcpy(p, c->Zs[1 - cur], blk, cudaMemcpyDeviceToHost));
    p += blk;
  }
  if (c->cfg.tau_mode == 1) {
    CK(cudaMemcpy(p, c->tfac, (size_t)c->N * sizeof(double), cudaMemcpyDeviceToHost));
    p += (size_t)c->N * sizeof(double);
  }
  if (c->P) CK(cudaMemcpy(p, c->nlC[cur], (size_t)c->N * c->P * sizeof(double), cudaMemcpyDeviceToHost));
  *size = need;
  return POU_OK;
}

pou_status pou_set_state(pou_ctx* c, const void* blob, size_t size) {
  if (!c || !blob) return POU_EINVAL;
  if (size < sizeof(BlobHeader)) return fail(c, POU_EINVAL, "state blob too small");
  BlobHeader h;
  std::memcpy(&h, blob, sizeof h);
  if (std::memcmp(h.magic, "POUSTATE", 8) != 0 || h.version != 1) return fail(c, POU_EINVAL, "not a state blob");
  if (h.dt != c->dt || h.N != c->N || h.nx != c->nx || h.ny != c->ny || h.nz != c->nz)
    return fail(c, POU_EINVAL, "state blob does not match this context");
  if ((long long)size < h.bytes) return fail(c, POU_EINVAL, "state blob truncated");
  const size_t blk = (size_t)c->N * c->ng * c->esz;
  const char* p = static_cast<const char*>(blob) + sizeof h;
  State hs;
  std::memcpy(&hs, p, sizeof hs);
  p += sizeof hs;
  const int cur = hs.cur;
  if (cur != 0 && cur != 1) return fail(c, POU_EINVAL, "corrupt state blob");
  hs.done = 1;
  CK(cudaMemcpy(c->hist_E, p, HIST_MAX * sizeof(double), cudaMemcpyHostToDevice));
  p += HIST_MAX * sizeof(double);
  CK(cudaMemcpy(c->hist_tau, p, HIST_MAX * sizeof(double), cudaMemcpyHostToDevice));
  p += HIST_MAX * sizeof(double);
  CK(cudaMemcpy(c->sigma[cur], p, c->N * sizeof(double), cudaMemcpyHostToDevice));
  p += c->N * sizeof(double);
  CK(cudaMemcpy(c->part[cur], p, (size_t)c->N * NP * sizeof(double), cudaMemcpyHostToDevice));
  p += (size_t)c->N * NP * sizeof(double);
  CK(cudaMemcpy(c->W[cur], p, blk, cudaMemcpyHostToDevice));
  p += blk;
  CK(cudaMemcpy(c->HW[cur], p, blk, cudaMemcpyHostToDevice));
  p += blk;
  CK(cudaMemcpy(c->rho[cur], p, c->ng * sizeof(double), cudaMemcpyHostToDevice));
  p += c->ng * sizeof(double);
  CK(cudaMemcpy(c->V64[cur], p, c->ng * sizeof(double), cudaMemcpyHostToDevice));
  p += c->ng * sizeof(double);
  {
    const size_t extra = (c->cfg.direction == 1 ? 2 * blk : 0) + (c->cfg.solver == 1 ? 2 * blk : 0) +
                         (c->cfg.tau_mode == 1 ? (size_t)c->N * sizeof(double) : 0) +
                         (size_t)c->N * c->P * sizeof(double);
    if (h.bytes != (long long)((p - static_cast<const char*>(blob)) + extra))
      return fail(c, POU_EINVAL, "state blob lacks the history of this context's direction or steps");
  }
  if (c->cfg.direction == 1) {
    CK(cudaMemcpy(c->W[1 - cur], p, blk, cudaMemcpyHostToDevice));
    p += blk;
    CK(cudaMemcpy(c->Z[1 - cur], p, blk, cudaMemcpyHostToDevice));
    p += blk;
  }
  if (c->cfg.solver == 1) {
    CK(cudaMemcpy(c->D[1 - cur], p, blk, cudaMemcpyHostToDevice));
    p += blk;
    CK(cudaMemcpy(c->Zs[1 - cur], p, blk, cudaMemcpyHostToDevice));
    p += blk;
  }
  if (c->cfg.tau_mode == 1) {
    CK(cudaMemcpy(c->tfac, p, (size_t)c->N * sizeof(double), cudaMemcpyHostToDevice));
    p += (size_t)c->N * sizeof(double);
  }
  if (c->P) CK(cudaMemcpy(c->nlC[cur], p, (size_t)c->N * c->P * sizeof(double), cudaMemcpyHostToDevice));
  if (c->dt == 1)
    launch_convert_f64_f32(c->V64[cur], static_cast<float*>(c->V[cur]), c->ng, c->stream);
  CK(cudaMemcpy(c->st, &hs, sizeof hs, cudaMemcpyHostToDevice));
  pou_status e = check_launch(c, "set_state");
  if (e != POU_OK) return e;
  CK(cudaDeviceSynchronize());
  c->have_orbitals = true;
  return POU_OK;
}

pou_status pou_selftest_wait_timeout(double limit_s, int* timed_out) {
  if (!timed_out || !(limit_s > 0.0) || limit_s > 10.0) return POU_EINVAL;
  *timed_out = 0;
  return wait_selftest(limit_s, timed_out) == 0 ? POU_OK : POU_ECUDA;
}

pou_status pou_synchronize(pou_ctx* c) {
  if (!c) return POU_EINVAL;
  CK(cudaStreamSynchronize(c->stream));
  return POU_OK;
}

long long pou_launch_count(const pou_ctx* c) { return c ? g_launches - c->launches0 : 0; }

pou_status pou_set_profiling(pou_ctx* c, int enable) {
  if (!c) return POU_EINVAL;
  if (enable && !c->prof) c->prof = new CtxProfiler();
  if (!enable && c->prof) {
    CK(cudaStreamSynchronize(c->stream));
    delete c->prof;
    c->prof = nullptr;
  }
  return POU_OK;
}

pou_status pou_get_profile(pou_ctx* c, int max_entries, char* names, long long* launches, double* ms, int* count) {
  if (!c || !count || max_entries < 0) return POU_EINVAL;
  if (!c->prof) {
    *count = 0;
    return POU_OK;
  }
  CK(cudaStreamSynchronize(c->stream));
  c->prof->collect();
  const int n = std::min<int>(max_entries, (int)c->prof->names.size());
  for (int i = 0; i < n; ++i) {
    if (names) {
      std::memset(names + 32 * i, 0, 32);
      std::strncpy(names + 32 * i, c->prof->names[i].c_str(), 31);
    }
    if (launches) launches[i] = c->prof->launches[i];
    if (ms) ms[i] = c->prof->ms[i];
  }
  *count = n;
  return POU_OK;
}

// ------------------------------------------------------------ stand-alone ops
size_t pou_gram_workspace_bytes(int dtype, long long Ng, int N) {
  int nsplit, npair;
  i64 chunk;
  if (dtype == POU_DT_F64) {
    gram_layout<double>(Ng, N, false, &nsplit, &npair, &chunk);
    return (size_t)nsplit * npair * gram_supertile<double>() * gram_supertile<double>() * sizeof(double);
  }
  gram_layout<float>(Ng, N, false, &nsplit, &npair, &chunk);
  return (size_t)nsplit * npair * gram_supertile<float>() * gram_supertile<float>() * sizeof(double);
}

pou_status pou_gram(int dtype, long long Ng, int N, const void* A, double dV, double* S, void* workspace,
                    size_t workspace_bytes, void* stream) {
  configure_kernels();
  if ((dtype != POU_DT_F64 && dtype != POU_DT_F32) || Ng < 1 || N < 1 || N > POU_MAX_N || !A || !S ||
      !workspace)
    return POU_EINVAL;
  if (workspace_bytes < pou_gram_workspace_bytes(dtype, Ng, N)) return POU_EINVAL;
  if (!device_accessible(A) || !device_accessible(S) || !device_accessible(workspace)) return POU_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int nsplit, npair;
  i64 chunk;
  GramReduceArgs r{};
  if (dtype == POU_DT_F64) {
    GramArgs<double> g{};
    g.A = static_cast<const double*>(A);
    g.ng = Ng;
    g.N = N;
    g.split = static_cast<double*>(workspace);
    launch_gram<double>(g, s);
    gram_layout<double>(Ng, N, false, &nsplit, &npair, &chunk);
    r.ST = gram_supertile<double>();
  } else {
    GramArgs<float> g{};
    g.A = static_cast<const float*>(A);
    g.ng = Ng;
    g.N = N;
    g.split = static_cast<double*>(workspace);
    launch_gram<float>(g, s);
    gram_layout<float>(Ng, N, false, &nsplit, &npair, &chunk);
    r.ST = gram_supertile<float>();
  }
  r.split = static_cast<double*>(workspace);
  r.nsplit = nsplit;
  r.npair = npair;
  r.N = N;
  r.dV = dV;
  r.S = S;
  launch_gram_reduce(r, s);
  return cudaGetLastError() == cudaSuccess ? POU_OK : POU_ECUDA;
}

pou_status pou_cholinv(int N, const double* S, double* Rinv, int* info, void* stream) {
  configure_kernels();
  if (N < 1 || N > POU_MAX_N || !S || !Rinv || !info) return POU_EINVAL;
  if (!device_accessible(S) || !device_accessible(Rinv) || !device_accessible(info)) return POU_EINVAL;
  launch_cholinv(nullptr, S, Rinv, N, info, nullptr, 0.0, 0.0, static_cast<cudaStream_t>(stream));
  return cudaGetLastError() == cudaSuccess ? POU_OK : POU_ECUDA;
}

pou_status pou_rotate(int dtype, long long Ng, int N, const void* A, const double* Rinv, void* B, double* rho,
                      void* stream) {
  configure_kernels();
  if ((dtype != POU_DT_F64 && dtype != POU_DT_F32) || Ng < 1 || N < 1 || N > POU_MAX_N || !A || !Rinv || !B)
    return POU_EINVAL;
  if (dtype == POU_DT_F64 && N > POU_MAX_N_FP64) return POU_EINVAL;
  if (!device_accessible(A) || !device_accessible(Rinv) || !device_accessible(B) ||
      (rho && !device_accessible(rho)))
    return POU_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (dtype == POU_DT_F64) {
    RotArgs<double> ra{};
    ra.A = static_cast<const double*>(A);
    ra.B = static_cast<double*>(B);
    ra.rho_out = rho;
    ra.Rinv = Rinv;
    ra.ng = Ng;
    ra.N = N;
    launch_rotate<double>(ra, s);
  } else {
    RotArgs<float> ra{};
    ra.A = static_cast<const float*>(A);
    ra.B = static_cast<float*>(B);
    ra.rho_out = rho;
    ra.Rinv = Rinv;
    ra.ng = Ng;
    ra.N = N;
    // N > 128: stream-ordered scratch for the split R^-1 image, freed after the launch
    if (N > 128 && cudaMallocAsync(reinterpret_cast<void**>(&ra.rimg), rotate_rimg_bytes(N), s) != cudaSuccess) {
      cudaGetLastError();
      return POU_ENOMEM;
    }
    launch_rotate<float>(ra, s);
    if (ra.rimg) cudaFreeAsync(ra.rimg, s);
  }
  return cudaGetLastError() == cudaSuccess ? POU_OK : POU_ECUDA;
}

size_t pou_hartree_workspace_bytes(const int n[3]) {
  if (!n) return 0;
  return (size_t)n[0] * n[1] * n[2] * sizeof(double2);
}

pou_status pou_hartree(const int n[3], const double L[3], const double* rho, double* vh, void* workspace,
                       size_t workspace_bytes, void* stream) {
  configure_kernels();
  if (!n || !L || !rho || !vh || !workspace) return POU_EINVAL;
  for (int a = 0; a < 3; ++a)
    if (n[a] < 1 || !fft_supported(n[a]) || !(L[a] > 0.0)) return POU_EINVAL;
  if (workspace_bytes < pou_hartree_workspace_bytes(n)) return POU_EINVAL;
  if (!device_accessible(rho) || !device_accessible(vh) || !device_accessible(workspace)) return POU_EINVAL;
  FftPlan p{};
  if (fft_plan_create(&p, n, L) != 0) {
    fft_plan_destroy(&p);
    return POU_ENOMEM;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  PotArgs<double> pa{};
  pa.rho_x = rho;
  pa.vh_out = vh;
  pa.work = static_cast<double2*>(workspace);
  pa.hartree = 1;
  launch_potential<double>(p, pa, s);
  cudaError_t e = cudaGetLastError();
  cudaStreamSynchronize(s);
  fft_plan_destroy(&p);
  return e == cudaSuccess ? POU_OK : POU_ECUDA;
}

}  // extern "C"

namespace pou {
bool device_accessible(const void* p) {
  if (!p) return false;
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}
}  // namespace pou
