// Cholesky-QR contractions of Sec. 3.2 on CUDA cores:
//   * Gram S = <Wt^T Wt> of the trial block Wt = W - tau Z
//     = (1 + tau sigma_i) w_i - tau hw_i, formed on the fly from W and HW
//     (so Z is never stored), split over the grid dimension with one FP64
//     partial per split and a deterministic reduction (FP64 form, and the
//     general product A^T B of either form; the symmetric FP32 Gram runs on
//     the tensor cores, k_gram_tc.cu);
//   * the reduction of the split partials, with the exact FP64 diagonal of
//     the trial Gram from the H-apply sums;
//   * rotation W_new = Wt R^-1 (R^-1 upper triangular) fused with the
//     density rho = f sum_j w_new_j^2 (FP64 form; the FP32 form runs on the
//     tensor cores, k_rotate_tc.cu).
#include "pou_internal.cuh"

#include <algorithm>

namespace pou {

namespace {

template <typename T>
struct GT;
template <>
struct GT<float> {
  static constexpr int RT = 8, ST = 128, BK = 16;
};
template <>
struct GT<double> {
  static constexpr int RT = 4, ST = 64, BK = 16;
};

constexpr int GNT = 256;

// Double-float accumulation in FP32 for sums of squares: (s, c) carries the
// running sum s and its rounding error c.  x*x is split exactly into
// p + e (FMA), and each addition s + p is split exactly into t + err
// (TwoSum), so s + c is the sum to about 2^-44 relative.
struct F2 {
  float s, c;
};
__device__ __forceinline__ void two_sum_add(F2& a, float b, float extra) {
  const float t = a.s + b;
  const float bp = t - a.s;
  const float err = (a.s - (t - bp)) + (b - bp);
  a.c += err + extra;
  a.s = t;
}
__device__ __forceinline__ void add_square(F2& a, float x) {
  const float p = x * x;
  two_sum_add(a, p, fmaf(x, x, -p));
}
__device__ __forceinline__ void add_f2(F2& a, const F2& b) { two_sum_add(a, b.s, b.c); }

// Gram of a block over the grid dimension.  Work unit: a tile of BK
// consecutive grid points; CTA b of G takes tiles b, b + G, b + 2G, ...
// spread over the whole grid, so that its running sums of off-diagonal
// products stay incoherent (small) instead of accumulating one region's
// overlap.  Sums are two-level: a per-tile partial (lo) is added into a
// per-CTA total (hi).  The next tile is prefetched into registers while the
// current one is multiplied out of shared memory (double buffer, one barrier
// per tile).  Every thread owns an RT x RT block of the ST x ST super-tile.
template <typename T>
__global__ void __launch_bounds__(GNT, 1) k_gram(GramArgs<T> a, i64 ntiles, int nsup, int npair) {
  constexpr int RT = GT<T>::RT, ST = GT<T>::ST, BK = GT<T>::BK;
  constexpr int PER = ST * BK / GNT;  // tile elements loaded per thread
  __shared__ __align__(16) T As[2][BK][ST + 4];
  __shared__ __align__(16) T Bs[2][BK][ST + 4];
  __shared__ T coefs[ST], coefs2[ST], taus[ST], taus2[ST];

  if (a.st && a.st->done) return;
  if (!gate_open(a.st, a.gate)) return;
  const bool general = (a.B != nullptr) || a.src_cur_pair;
  const int p = blockIdx.y;
  int I, J;
  if (general) {
    I = p / nsup;
    J = p % nsup;
  } else {
    int r = 0, rem = p;
    while (rem >= nsup - r) {
      rem -= nsup - r;
      ++r;
    }
    I = r;
    J = r + rem;
  }
  const bool diag = (!general) && (I == J);
  const int tid = threadIdx.x;
  const int ti = tid / 16, tj = tid % 16;
  const i64 ng = a.ng;
  const int N = a.N;

  const T* Wa;
  const T* Ha = nullptr;
  const T* Bsrc;
  if (a.trial) {
    const int cur = a.st->cur;
    Wa = a.W[cur];
    Ha = a.HW[cur];
    Bsrc = Wa;
    const double tau = a.st->tau_trial;
    for (int r = tid; r < ST; r += GNT) {
      const int gi = I * ST + r, gj = J * ST + r;
      const double ti = (gi < N && a.tfac) ? tau * a.tfac[gi] : tau;
      const double tj = (gj < N && a.tfac) ? tau * a.tfac[gj] : tau;
      coefs[r] = gi < N ? (T)(1.0 + ti * a.sigma[cur][gi]) : T(0);
      coefs2[r] = gj < N ? (T)(1.0 + tj * a.sigma[cur][gj]) : T(0);
      taus[r] = (T)ti;
      taus2[r] = (T)tj;
    }
  } else if (a.src_trial_slot) {
    Wa = a.W[1 - a.st->cur];
    Bsrc = Wa;
  } else if (a.src_cur_pair) {
    Wa = a.W[a.st->cur];
    Bsrc = a.HW[a.st->cur];
  } else {
    Wa = a.A;
    Bsrc = general ? a.B : a.A;
  }
  __syncthreads();

  // element e of a tile: row r = e / BK (orbital within the super-tile), k = e % BK
  T pa[PER], pah[PER], pb[PER], pbh[PER];
  auto fetch = [&](i64 tile) {
    const i64 k0 = tile * BK;
#pragma unroll
    for (int q = 0; q < PER; ++q) {
      const int e = tid + q * GNT;
      const int r = e / BK, k = e % BK;
      const int gi = I * ST + r, gj = J * ST + r;
      const i64 gk = k0 + k;
      const bool okA = gi < N && gk < ng, okB = gj < N && gk < ng;
      pa[q] = okA ? Wa[(i64)gi * ng + gk] : T(0);
      if (a.trial) pah[q] = okA ? Ha[(i64)gi * ng + gk] : T(0);
      if (!diag) {
        pb[q] = okB ? Bsrc[(i64)gj * ng + gk] : T(0);
        if (a.trial) pbh[q] = okB ? Ha[(i64)gj * ng + gk] : T(0);
      }
    }
  };
  auto stash = [&](int buf) {
#pragma unroll
    for (int q = 0; q < PER; ++q) {
      const int e = tid + q * GNT;
      const int r = e / BK, k = e % BK;
      As[buf][k][r] = a.trial ? coefs[r] * pa[q] - taus[r] * pah[q] : pa[q];
      if (!diag) Bs[buf][k][r] = a.trial ? coefs2[r] * pb[q] - taus2[r] * pbh[q] : pb[q];
    }
  };

  T hi[RT][RT], lo[RT][RT];
#pragma unroll
  for (int r = 0; r < RT; ++r)
#pragma unroll
    for (int c = 0; c < RT; ++c) hi[r][c] = T(0);

  const i64 G = gridDim.x;
  i64 t = blockIdx.x;
  int buf = 0;
  if (t < ntiles) {
    fetch(t);
    stash(0);
  }
  __syncthreads();
  for (; t < ntiles; t += G) {
    const i64 tn = t + G;
    if (tn < ntiles) fetch(tn);
    const T(*At)[ST + 4] = As[buf];
    const T(*Bt)[ST + 4] = diag ? As[buf] : Bs[buf];
#pragma unroll
    for (int r = 0; r < RT; ++r)
#pragma unroll
      for (int c = 0; c < RT; ++c) lo[r][c] = T(0);
#pragma unroll 4
    for (int k = 0; k < BK; ++k) {
      T av[RT], bv[RT];
#pragma unroll
      for (int r = 0; r < RT; ++r) av[r] = At[k][ti * RT + r];
#pragma unroll
      for (int c = 0; c < RT; ++c) bv[c] = Bt[k][tj * RT + c];
#pragma unroll
      for (int r = 0; r < RT; ++r)
#pragma unroll
        for (int c = 0; c < RT; ++c) lo[r][c] = fma(av[r], bv[c], lo[r][c]);
    }
#pragma unroll
    for (int r = 0; r < RT; ++r)
#pragma unroll
      for (int c = 0; c < RT; ++c) hi[r][c] += lo[r][c];
    if (tn < ntiles) stash(buf ^ 1);
    __syncthreads();
    buf ^= 1;
  }

  double* out = a.split + ((i64)blockIdx.x * npair + p) * (i64)(ST * ST);
#pragma unroll
  for (int r = 0; r < RT; ++r)
#pragma unroll
    for (int c = 0; c < RT; ++c) out[(ti * RT + r) * ST + tj * RT + c] = (double)hi[r][c];
}

__global__ void k_gram_reduce(GramReduceArgs a) {
  if (a.st && a.st->done) return;
  if (!gate_open(a.st, a.gate)) return;
  const int r = blockIdx.y * blockDim.y + threadIdx.y;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const int N = a.N;
  if (r >= N || c >= N) return;
  if (!a.general && r > c) return;
  const int ST = a.ST;
  const int nsup = (N + ST - 1) / ST;
  const int I = r / ST, J = c / ST;
  int p;
  if (a.general) {
    p = I * nsup + J;
  } else {
    p = I * nsup - I * (I - 1) / 2 + (J - I);
  }
  const i64 off = (i64)p * ST * ST + (r % ST) * ST + (c % ST);
  const i64 stride = (i64)a.npair * ST * ST;
  double s = 0.0;
  if (!a.general && I == J) {
    // diagonal super-tile: symmetric part (the tensor-core kernel stores an
    // unsymmetrised product; for the others both halves are equal)
    const i64 offt = (i64)p * ST * ST + (c % ST) * ST + (r % ST);
    for (int k = 0; k < a.nsplit; ++k) s += 0.5 * (a.split[off + k * stride] + a.split[offt + k * stride]);
  } else {
    for (int k = 0; k < a.nsplit; ++k) s += a.split[off + k * stride];
  }
  s *= a.dV;
  if (a.trial == 2 && r == c) {
    // a materialised direction (OptM-QR, conjugate gradient): the trial
    // column w - t z, z the direction block; FP64 sums of the kernel that
    // formed z
    const double tau = a.st->tau_trial * (a.tfac ? a.tfac[r] : 1.0);
    const double* dp = a.dpart + (i64)r * 3;
    s = a.dV * (dp[0] - 2.0 * tau * dp[1] + tau * tau * dp[2]);
  } else if (a.trial && r == c) {
    // FP64 norm of the trial column a w - t hw (FP64 coefficients, as both
    // rotations form the trial point) from the H-apply sums of W[cur]:
    //   a w - t hw = w - t z_e,  z_e = hw - s_e w,  s_e = (a - 1) / t,
    //   z_e = z' - d w with z' = hw - sigma' w, d = s_e - sigma',
    //   ||w - t z_e||^2 = <w,w> - 2 t <w,z_e> + t^2 <z_e,z_e>.
    const int cur = a.st->cur;
    const double tau = a.st->tau_trial * (a.tfac ? a.tfac[r] : 1.0);
    const double coef = 1.0 + tau * a.sigma[cur][r];
    const double t = tau;
    const double* pp = a.part[cur] + (i64)r * NP;
    const double d = (coef - 1.0) / t - pp[P_SIGP];
    const double wz = pp[P_ZW] - d * pp[P_WW];
    const double zz = pp[P_ZZ] - 2.0 * d * pp[P_ZW] + d * d * pp[P_WW];
    s = a.dV * (pp[P_WW] - 2.0 * t * wz + t * t * zz);
  }
  a.S[(i64)r * N + c] = s;
  if (!a.general) a.S[(i64)c * N + r] = s;
}

// --------------------------------------------------------------- rotation
// FP64 form (the FP32 form runs on the tensor cores, k_rotate_tc.cu):
// W_new = X R^-1 with X = Wt (trial) or the block itself, fused with the
// density.  A chunk of RP points of all N orbitals is staged in shared
// memory; each thread forms 8 outputs x 4 points.  For the upper-triangular
// R^-1 only i <= j contributes.
constexpr int RNT = 256;
constexpr int RP = 64;  // points per chunk

__global__ void __launch_bounds__(RNT) k_rotate(RotArgs<double> a, int nchunks) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int N = a.N;
  const int NPAD = 128;
  double* Rs = reinterpret_cast<double*>(smem_raw);  // [NPAD][NPAD]
  double* Xs = Rs + NPAD * NPAD;                      // [NPAD][RP + 4]
  double* coefs = Xs + NPAD * (RP + 4);               // [NPAD]
  double* taus = coefs + NPAD;                        // [NPAD] per-orbital trial step
  constexpr int XS = RP + 4;

  if (a.st && a.st->done) return;
  if (!gate_open(a.st, a.gate)) return;
  const int tid = threadIdx.x;
  const double* Wsrc;
  const double* Hsrc = nullptr;
  double* out;
  double* rho;
  double tau = 0.0;
  if (a.trial) {
    const int cur = a.st->cur;
    Wsrc = a.W[cur];
    Hsrc = a.HW[cur];
    out = a.Wout[1 - cur];
    rho = a.rho[1 - cur];
    tau = a.st->tau_trial;
    for (int i = tid; i < NPAD; i += RNT) {
      const double t = (i < N && a.tfac) ? tau * a.tfac[i] : tau;
      coefs[i] = i < N ? 1.0 + t * a.sigma[cur][i] : 0.0;
      taus[i] = t;
    }
  } else if (a.st) {
    const int cur = a.st->cur;
    // in-place passes read the block they overwrite: every chunk is staged in
    // shared memory before any of its outputs is stored
    if (a.src_cur_slot) {
      Wsrc = a.Wout[cur];
      out = a.Wout[cur];
      rho = nullptr;  // a rotation within the span leaves rho unchanged
    } else {
      Wsrc = a.src_trial_slot ? a.Wout[1 - cur] : a.A;
      out = a.Wout[1 - cur];
      rho = a.rho[1 - cur];
    }
  } else {
    Wsrc = a.A;
    out = a.B;
    rho = a.rho_out;
  }
  for (int idx = tid; idx < NPAD * NPAD; idx += RNT) {
    const int i = idx / NPAD, j = idx % NPAD;
    Rs[idx] = (i < N && j < N) ? a.Rinv[(i64)i * N + j] : 0.0;
  }
  __syncthreads();

  const int lane = tid & 31, warp = tid >> 5;
  const int jw = warp & 3, pw = warp >> 2;
  const int jg = lane & 3, pg = lane >> 2;
  const int j0 = jw * 32 + jg * 8;  // 8 output orbitals
  const int pl0 = pw * 32 + pg * 4; // 4 points within the chunk
  const int imax = a.general ? N : min(N, j0 + 8);
  const i64 ng = a.ng;

  for (int ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
    const i64 p0 = (i64)ch * RP;
    for (int idx = tid; idx < N * RP; idx += RNT) {
      const int i = idx / RP, pp = idx % RP;
      const i64 gp = p0 + pp;
      double v = 0.0;
      if (gp < ng) {
        const i64 off = (i64)i * ng + gp;
        v = a.trial ? coefs[i] * Wsrc[off] - taus[i] * Hsrc[off] : Wsrc[off];
      }
      Xs[i * XS + pp] = v;
    }
    __syncthreads();

    double acc[8][4];
#pragma unroll
    for (int jj = 0; jj < 8; ++jj)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[jj][q] = 0.0;
    for (int i = 0; i < imax; ++i) {
      double rv[8], xv[4];
#pragma unroll
      for (int jj = 0; jj < 8; ++jj) rv[jj] = Rs[i * NPAD + j0 + jj];
#pragma unroll
      for (int q = 0; q < 4; ++q) xv[q] = Xs[i * XS + pl0 + q];
#pragma unroll
      for (int jj = 0; jj < 8; ++jj)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[jj][q] = fma(rv[jj], xv[q], acc[jj][q]);
    }
    double sqd[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
    for (int jj = 0; jj < 8; ++jj) {
      const int j = j0 + jj;
      if (j < N) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const i64 gp = p0 + pl0 + q;
          if (gp < ng) out[(i64)j * ng + gp] = acc[jj][q];
          sqd[q] = fma(acc[jj][q], acc[jj][q], sqd[q]);
        }
      }
    }
    if (rho != nullptr) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        sqd[q] += __shfl_xor_sync(0xffffffffu, sqd[q], 1);
        sqd[q] += __shfl_xor_sync(0xffffffffu, sqd[q], 2);
      }
    }
    __syncthreads();  // Xs no longer read; reuse a region for the density
    if (rho != nullptr) {
      double* dsum = Xs;  // [4][RP]
      if (jg == 0) {
#pragma unroll
        for (int q = 0; q < 4; ++q) dsum[jw * RP + pl0 + q] = sqd[q];
      }
      __syncthreads();
      if (tid < RP) {
        const i64 gp = p0 + tid;
        if (gp < ng) rho[gp] = F_OCC * (dsum[tid] + dsum[RP + tid] + dsum[2 * RP + tid] + dsum[3 * RP + tid]);
      }
      __syncthreads();
    }
  }
}

// FP32 form, general rotation W <- W P of Algorithm M (P dense, far from the
// identity) on the CUDA cores.  There every output is an O(1) mixture of the
// inputs, and the tensor-core path (TF32 split products, truncating FP32
// accumulation) would leave errors of a few 1e-7 relative in the rotated
// orbitals; here every product is an exact FP32 FMA with round-to-nearest
// accumulation, and the self term P_jj w_j is added with double-float
// coefficients and stored with unbiased (dithered) rounding like the
// tensor-core rotation.  Runs once every n_diag steps.
__device__ __forceinline__ unsigned mix32(unsigned x) {
  // lowbias32 integer mixer (C. Wellons, hash-prospector)
  x ^= x >> 16;
  x *= 0x7feb352dU;
  x ^= x >> 15;
  x *= 0x846ca68bU;
  x ^= x >> 16;
  return x;
}
__device__ __forceinline__ float dither(float x, unsigned byte) {
  const float ulp = __uint_as_float(__float_as_uint(x) & 0x7f800000u) * 1.1920928955078125e-7f;
  return ((float)byte * (1.0f / 256.0f) - 0.498046875f) * ulp;
}

__global__ void __launch_bounds__(RNT) k_rotate_f32_cc(RotArgs<float> a, int nchunks) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int N = a.N;
  const int NPAD = 128;
  float* Rs = reinterpret_cast<float*>(smem_raw);  // [NPAD][NPAD], zero diagonal
  float* Xs = Rs + NPAD * NPAD;                     // [NPAD][RP + 4]
  float* self = Xs + NPAD * (RP + 4);               // [2][NPAD]: P_jj hi, lo
  constexpr int XS = RP + 4;

  if (a.st && a.st->done) return;
  if (!gate_open(a.st, a.gate)) return;
  const int tid = threadIdx.x;
  const float* Wsrc;
  float* out;
  double* rho;
  if (a.st) {
    const int cur = a.st->cur;
    if (a.src_cur_slot) {
      Wsrc = a.Wout[cur];
      out = a.Wout[cur];
      rho = nullptr;  // a rotation within the span leaves rho unchanged
    } else {
      Wsrc = a.src_trial_slot ? a.Wout[1 - cur] : a.A;
      out = a.Wout[1 - cur];
      rho = a.rho[1 - cur];
    }
  } else {
    Wsrc = a.A;
    out = a.B;
    rho = a.rho_out;
  }
  for (int idx = tid; idx < NPAD * NPAD; idx += RNT) {
    const int i = idx / NPAD, j = idx % NPAD;
    const double v = (i < N && j < N && (a.general || i <= j)) ? a.Rinv[(i64)i * N + j] : 0.0;
    Rs[idx] = (i == j) ? 0.f : (float)v;
    if (i == j) {
      self[i] = (float)v;
      self[NPAD + i] = (float)(v - (double)(float)v);
    }
  }
  __syncthreads();
  const unsigned seed32 = mix32((unsigned)(a.st ? a.st->passes : 0) * 4u + (unsigned)a.sr_salt + 0x85ebca6bu);

  const int lane = tid & 31, warp = tid >> 5;
  const int jw = warp & 3, pw = warp >> 2;
  const int jg = lane & 3, pg = lane >> 2;
  const int j0 = jw * 32 + jg * 8;  // 8 output orbitals
  const int pl0 = pw * 32 + pg * 4; // 4 points within the chunk
  const int imax = a.general ? N : min(N, j0 + 8);
  const i64 ng = a.ng;

  for (int ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
    const i64 p0 = (i64)ch * RP;
    for (int idx = tid; idx < N * RP; idx += RNT) {
      const int i = idx / RP, pp = idx % RP;
      const i64 gp = p0 + pp;
      Xs[i * XS + pp] = gp < ng ? Wsrc[(i64)i * ng + gp] : 0.f;
    }
    __syncthreads();

    float acc[8][4];
#pragma unroll
    for (int jj = 0; jj < 8; ++jj)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[jj][q] = 0.f;
    for (int i = 0; i < imax; ++i) {
      float rv[8], xv[4];
#pragma unroll
      for (int jj = 0; jj < 8; ++jj) rv[jj] = Rs[i * NPAD + j0 + jj];
#pragma unroll
      for (int q = 0; q < 4; ++q) xv[q] = Xs[i * XS + pl0 + q];
#pragma unroll
      for (int jj = 0; jj < 8; ++jj)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[jj][q] = fmaf(rv[jj], xv[q], acc[jj][q]);
    }
    // self term with double-float P_jj, unbiased rounding; density in double-float
    float ds[4] = {0.f, 0.f, 0.f, 0.f}, dc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int jj = 0; jj < 8; ++jj) {
      const int j = j0 + jj;
      if (j >= N) continue;
      const float ph = self[j], plo = self[NPAD + j];
      const unsigned bits = mix32(seed32 ^ mix32((unsigned)j * 0x9e3779b1u ^ (unsigned)(p0 + pl0)));
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float wv = Xs[j * XS + pl0 + q];
        const float d = dither(wv, (bits >> (8 * q)) & 0xffu);
        const float o = fmaf(ph, wv, fmaf(plo, wv, acc[jj][q] + d));
        const i64 gp = p0 + pl0 + q;
        if (gp < ng) out[(i64)j * ng + gp] = o;
        const float sq = o * o;
        F2 f{ds[q], dc[q]};
        two_sum_add(f, sq, fmaf(o, o, -sq));
        ds[q] = f.s;
        dc[q] = f.c;
      }
    }
    if (rho != nullptr) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        for (int o = 1; o <= 2; o <<= 1) {
          F2 f{ds[q], dc[q]};
          two_sum_add(f, __shfl_xor_sync(0xffffffffu, ds[q], o), __shfl_xor_sync(0xffffffffu, dc[q], o));
          ds[q] = f.s;
          dc[q] = f.c;
        }
      }
    }
    __syncthreads();  // Xs no longer read; reuse a region for the density
    if (rho != nullptr) {
      double* dsum = reinterpret_cast<double*>(Xs);  // [4][RP]
      if (jg == 0) {
#pragma unroll
        for (int q = 0; q < 4; ++q) dsum[jw * RP + pl0 + q] = (double)ds[q] + (double)dc[q];
      }
      __syncthreads();
      if (tid < RP) {
        const i64 gp = p0 + tid;
        if (gp < ng) rho[gp] = F_OCC * (dsum[tid] + dsum[RP + tid] + dsum[2 * RP + tid] + dsum[3 * RP + tid]);
      }
      __syncthreads();
    }
  }
}

// Residual of the Kohn-Sham equations, the convergence report of Sec. 4.2
// (Eq. gra): G = HW - W Sigma with Sigma_ij = <hw_i, w_j>, so that
// g_i = hw_i - sum_j Sigma_ji w_j, and ||G||_F^2 = dV sum_i sum_p g_i(p)^2.
// Sig is the general Gram S_ij = <w_i, hw_j> = Sigma_ji.
// G is formed point by point (a chunk of RP points staged in shared memory,
// 8 orbitals x 4 points per thread, working-type FMAs): near convergence g
// is a small difference of O(1) terms, which the trace identity
// tr(HW^T HW) - |Sigma|^2 would lose to cancellation.  Orbitals are taken in
// blocks of 128 (Sigma one 128 x 128 tile at a time for N > 128).  Each CTA
// writes one FP64 partial of sum g^2.
template <typename T>
__global__ void __launch_bounds__(RNT) k_residual(const T* W, const T* HW, const double* Sig, int N, i64 ng,
                                                   int nchunks, double* part) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int NPAD = 128;
  T* Ss = reinterpret_cast<T*>(smem_raw);  // [NPAD][NPAD]: Ss[j][i] = S_(ib+i)(jb+j) = Sigma_ji
  T* Xs = Ss + NPAD * NPAD;                // [NPAD][RP + 4] chunk of W, rows jb ..
  constexpr int XS = RP + 4;
  __shared__ double red[RNT / 32];
  const int tid = threadIdx.x;
  const int nb = (N + NPAD - 1) / NPAD;
  auto load_sig = [&](int ib, int jb) {
    for (int idx = tid; idx < NPAD * NPAD; idx += RNT) {
      const int j = idx / NPAD, i = idx % NPAD;
      const int gi = ib * NPAD + i, gj = jb * NPAD + j;
      Ss[idx] = (gi < N && gj < N) ? (T)Sig[(i64)gi * N + gj] : T(0);
    }
  };
  if (nb == 1) load_sig(0, 0);
  const int lane = tid & 31, warp = tid >> 5;
  const int iw = warp & 3, pw = warp >> 2;
  const int ig = lane & 3, pg = lane >> 2;
  const int i0 = iw * 32 + ig * 8;   // 8 orbitals of the block
  const int pl0 = pw * 32 + pg * 4;  // 4 points within the chunk
  double total = 0.0;
  for (int ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
    const i64 p0 = (i64)ch * RP;
    for (int ib = 0; ib < nb; ++ib) {
      T acc[8][4];
#pragma unroll
      for (int ii = 0; ii < 8; ++ii)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[ii][q] = T(0);
      for (int jb = 0; jb < nb; ++jb) {
        const int nj = min(NPAD, N - jb * NPAD);
        __syncthreads();
        if (nb > 1) load_sig(ib, jb);
        for (int idx = tid; idx < nj * RP; idx += RNT) {
          const int j = idx / RP, pp = idx % RP;
          const i64 gp = p0 + pp;
          Xs[j * XS + pp] = gp < ng ? W[(i64)(jb * NPAD + j) * ng + gp] : T(0);
        }
        __syncthreads();
        for (int j = 0; j < nj; ++j) {
          T sv[8], xv[4];
#pragma unroll
          for (int ii = 0; ii < 8; ++ii) sv[ii] = Ss[j * NPAD + i0 + ii];
#pragma unroll
          for (int q = 0; q < 4; ++q) xv[q] = Xs[j * XS + pl0 + q];
#pragma unroll
          for (int ii = 0; ii < 8; ++ii)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[ii][q] = fma(sv[ii], xv[q], acc[ii][q]);
        }
      }
      double part_sum = 0.0;
#pragma unroll
      for (int ii = 0; ii < 8; ++ii) {
        const int i = ib * NPAD + i0 + ii;
        if (i >= N) continue;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const i64 gp = p0 + pl0 + q;
          if (gp >= ng) continue;
          const T g = HW[(i64)i * ng + gp] - acc[ii][q];
          part_sum += (double)g * (double)g;
        }
      }
      total += part_sum;
    }
  }
  for (int o = 16; o > 0; o >>= 1) total += __shfl_xor_sync(0xffffffffu, total, o);
  if (lane == 0) red[warp] = total;
  __syncthreads();
  if (tid == 0) {
    double v = 0.0;
    for (int w = 0; w < RNT / 32; ++w) v += red[w];
    part[blockIdx.x] = v;
  }
}

template <typename T>
__global__ void k_density(const T* U, i64 ng, int N, double* rho) {
  const i64 p = (i64)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= ng) return;
  if (sizeof(T) == 8) {
    double s = 0.0;
    for (int i = 0; i < N; ++i) {
      const double v = (double)U[(i64)i * ng + p];
      s = fma(v, v, s);
    }
    rho[p] = F_OCC * s;
  } else {
    F2 s{0.f, 0.f};
    for (int i = 0; i < N; ++i) add_square(s, (float)U[(i64)i * ng + p]);
    rho[p] = F_OCC * ((double)s.s + (double)s.c);
  }
}

__global__ void k_f64_to_f32(const double* in, float* out, i64 n) {
  for (i64 i = (i64)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (i64)gridDim.x * blockDim.x)
    out[i] = (float)in[i];
}
__global__ void k_f32_to_f64(const float* in, double* out, i64 n) {
  for (i64 i = (i64)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (i64)gridDim.x * blockDim.x)
    out[i] = (double)in[i];
}
template <typename T>
__global__ void k_scale_copy(const T* in, T* out, T scale, i64 n) {
  for (i64 i = (i64)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (i64)gridDim.x * blockDim.x)
    out[i] = scale * in[i];
}

int grid_for(i64 n) {
  i64 b = (n + 255) / 256;
  if (b > num_sms() * 16) b = num_sms() * 16;
  if (b < 1) b = 1;
  return (int)b;
}

}  // namespace

template <typename T>
int gram_supertile() {
  return GT<T>::ST;
}
template int gram_supertile<float>();
template int gram_supertile<double>();

template <typename T>
void gram_layout(i64 ng, int N, bool general, int* nsplit, int* npair, i64* chunk) {
  const int ST = GT<T>::ST, BK = GT<T>::BK;
  const int nsup = (N + ST - 1) / ST;
  const int np = general ? nsup * nsup : nsup * (nsup + 1) / 2;
  const i64 ntiles = (ng + BK - 1) / BK;
  // one CTA per SM in total (one wave), at least 32 tiles per CTA; the
  // tensor-core Gram of the FP32 form (symmetric, N > 128) runs a diagonal
  // pair's two splits in one CTA
  i64 g = std::max(1, num_sms() / np);
  if (sizeof(T) == 4 && !general && nsup > 1)
    while (gram_tc_ctas((int)g + 1, nsup) <= num_sms()) ++g;
  g = std::max<i64>(1, std::min<i64>(g, ntiles / 32));
  *npair = np;
  *chunk = ntiles;  // tiles over the whole grid
  *nsplit = (int)g;
}
template void gram_layout<float>(i64, int, bool, int*, int*, i64*);
template void gram_layout<double>(i64, int, bool, int*, int*, i64*);

template <typename T>
static bool use_tc(const GramArgs<T>& a) {
  if constexpr (sizeof(T) == 4) {
    return gram_tc_eligible(a);
  } else {
    return false;
  }
}

template <typename T>
void launch_gram(const GramArgs<T>& a, cudaStream_t s) {
  int nsplit, npair;
  i64 ntiles;
  gram_layout<T>(a.ng, a.N, a.B != nullptr || a.src_cur_pair, &nsplit, &npair, &ntiles);
  if constexpr (sizeof(T) == 4) {
    if (use_tc(a)) {
      launch_gram_tc(a, nsplit, s);
      return;
    }
  }
  const int nsup = (a.N + GT<T>::ST - 1) / GT<T>::ST;
  dim3 grid(nsplit, npair);
  prof_begin(gram_prof_name(a.trial, a.src_trial_slot, a.src_cur_pair), s);
  k_gram<T><<<grid, GNT, 0, s>>>(a, ntiles, nsup, npair);
  prof_end(s);
}
template void launch_gram<float>(const GramArgs<float>&, cudaStream_t);
template void launch_gram<double>(const GramArgs<double>&, cudaStream_t);

template <typename T>
void launch_gram_nsplit(const GramArgs<T>& a, int nsplit, cudaStream_t s) {
  int ns, npair;
  i64 ntiles;
  gram_layout<T>(a.ng, a.N, a.B != nullptr || a.src_cur_pair, &ns, &npair, &ntiles);
  if constexpr (sizeof(T) == 4) {
    if (use_tc(a)) {
      launch_gram_tc(a, nsplit, s);
      return;
    }
  }
  const int nsup = (a.N + GT<T>::ST - 1) / GT<T>::ST;
  dim3 grid(nsplit, npair);
  prof_begin(gram_prof_name(a.trial, a.src_trial_slot, a.src_cur_pair), s);
  k_gram<T><<<grid, GNT, 0, s>>>(a, ntiles, nsup, npair);
  prof_end(s);
}
template void launch_gram_nsplit<float>(const GramArgs<float>&, int, cudaStream_t);
template void launch_gram_nsplit<double>(const GramArgs<double>&, int, cudaStream_t);

void launch_gram_reduce(const GramReduceArgs& a, cudaStream_t s) {
  dim3 block(32, 8);
  dim3 grid((a.N + 31) / 32, (a.N + 7) / 8);
  prof_begin("gram_reduce", s);
  k_gram_reduce<<<grid, block, 0, s>>>(a);
  prof_end(s);
}

static size_t rotate_smem() {
  const int NPAD = 128;
  return sizeof(double) * ((size_t)NPAD * NPAD + (size_t)NPAD * (RP + 4) + 2 * NPAD);
}
static size_t rotate_f32_smem() {
  const int NPAD = 128;
  return sizeof(float) * ((size_t)NPAD * NPAD + (size_t)NPAD * (RP + 4) + 2 * NPAD);
}

template <typename T>
static size_t residual_smem() {
  const int NPAD = 128;
  return sizeof(T) * ((size_t)NPAD * NPAD + (size_t)NPAD * (RP + 4));
}

void configure_rotate() {
  cudaFuncSetAttribute(k_rotate, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rotate_smem());
  cudaFuncSetAttribute(k_rotate_f32_cc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rotate_f32_smem());
  cudaFuncSetAttribute(k_residual<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)residual_smem<float>());
  cudaFuncSetAttribute(k_residual<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)residual_smem<double>());
}

template <typename T>
int launch_residual(const T* W, const T* HW, const double* Sig, int N, i64 ng, double* part, int max_blocks,
                    cudaStream_t s) {
  const int nchunks = (int)((ng + RP - 1) / RP);
  const int grid = std::max(1, std::min(nchunks, max_blocks));
  prof_begin("residual", s);
  k_residual<T><<<grid, RNT, residual_smem<T>(), s>>>(W, HW, Sig, N, ng, nchunks, part);
  prof_end(s);
  return grid;
}
template int launch_residual<float>(const float*, const float*, const double*, int, i64, double*, int, cudaStream_t);
template int launch_residual<double>(const double*, const double*, const double*, int, i64, double*, int,
                                     cudaStream_t);

int rotate_grid(i64 ng, int elem_bytes) {
  if (elem_bytes == 4) return rotate_tc_grid(ng);
  const int nchunks = (int)((ng + RP - 1) / RP);
  return std::min(nchunks, num_sms());
}

template <typename T>
void launch_rotate(const RotArgs<T>& a, cudaStream_t s) {
  if constexpr (sizeof(T) == 4) {
    if (a.general) {
      // dense P of Algorithm M: CUDA cores, exact FP32 products (the
      // tensor-core rotation takes upper triangular R^-1 only)
      const int nchunks = (int)((a.ng + RP - 1) / RP);
      prof_begin(rotate_prof_name(a.trial, a.src_trial_slot, a.src_cur_slot), s);
      k_rotate_f32_cc<<<std::min(nchunks, 2 * num_sms()), RNT, rotate_f32_smem(), s>>>(a, nchunks);
      prof_end(s);
    } else {
      launch_rotate_tc(a, s);
    }
  } else {
    const int nchunks = (int)((a.ng + RP - 1) / RP);
    prof_begin(rotate_prof_name(a.trial, a.src_trial_slot, a.src_cur_slot), s);
    k_rotate<<<rotate_grid(a.ng, 8), RNT, rotate_smem(), s>>>(a, nchunks);
    prof_end(s);
  }
}
template void launch_rotate<float>(const RotArgs<float>&, cudaStream_t);
template void launch_rotate<double>(const RotArgs<double>&, cudaStream_t);

template <typename T>
void launch_density(const T* U, i64 ng, int N, double* rho, cudaStream_t s) {
  prof_begin("density", s);
  k_density<T><<<(unsigned)((ng + 255) / 256), 256, 0, s>>>(U, ng, N, rho);
  prof_end(s);
}
template void launch_density<float>(const float*, i64, int, double*, cudaStream_t);
template void launch_density<double>(const double*, i64, int, double*, cudaStream_t);

void launch_convert_f64_f32(const double* in, float* out, i64 n, cudaStream_t s) {
  prof_begin("convert", s);
  k_f64_to_f32<<<grid_for(n), 256, 0, s>>>(in, out, n);
  prof_end(s);
}
void launch_convert_f32_f64(const float* in, double* out, i64 n, cudaStream_t s) {
  prof_begin("convert", s);
  k_f32_to_f64<<<grid_for(n), 256, 0, s>>>(in, out, n);
  prof_end(s);
}
template <typename T>
void launch_scale_copy(const T* in, T* out, T scale, i64 n, cudaStream_t s) {
  prof_begin("scale_copy", s);
  k_scale_copy<T><<<grid_for(n), 256, 0, s>>>(in, out, scale, n);
  prof_end(s);
}
template void launch_scale_copy<float>(const float*, float*, float, i64, cudaStream_t);
template void launch_scale_copy<double>(const double*, double*, double, i64, cudaStream_t);

}  // namespace pou
