// Cholesky-QR, middle step (Sec. 3.2): S = R^T R with R upper triangular and
// positive diagonal, then R^-1, in FP64; for N <= 128 in one CTA's shared
// memory, for larger N in global memory over many CTAs (further below).
// A non-positive pivot is reported through *info and the iteration state
// (status POU_ENOTSPD, done = 1); no trap, no wait.
// The same kernel records max |S - I| of the trial Gram matrix, the
// near-identity diagnostic of Fig. 2.
//
// Blocked, 32-wide panels.  Factorisation (right-looking): the diagonal
// block is factored by one warp with warp-level synchronisation only, the
// panel row is solved column by column in parallel, and the trailing matrix
// is updated with 4 x 4 register tiles (two FP64 FMAs per shared-memory
// load).  Inverse X = R^-1: the diagonal blocks are inverted by one warp
// each (one column per lane), then the off-diagonal blocks level by level,
// X_pq = -X_pp sum_{r=p+1..q} R_pr X_rq, all blocks of a level at once.
// X^T is kept in the (unused) lower triangle of the working matrix.
#include "pou_internal.cuh"

#include <algorithm>

namespace pou {

namespace {

constexpr int CNT = 512;
constexpr int NB = 32;       // panel width
constexpr int MAXB = 4;      // panels for N <= 128

__global__ void __launch_bounds__(CNT) k_cholinv(const State* st_ro, State* st, const double* S,
                                                  double* Rinv, int N, int* info, double piv_rel,
                                                  double reorth_thr, int orth_gated, int soft_limit) {
  extern __shared__ double A[];  // [N][N+1]: upper = R, strictly lower = X^T
  __shared__ double rdiag[128];  // 1 / R_ii
  __shared__ double T[MAXB - 1][NB][NB + 1];  // sums of one level of the inverse
  __shared__ volatile int fail;
  __shared__ double offmax[CNT / 32];
  __shared__ double dmax;
  if (st_ro && st_ro->done) return;
  if (reorth_thr < 0.0 && !(st_ro && st_ro->reorth)) return;  // gated second pass
  if (orth_gated && st_ro && !st_ro->orth_now) {
    // Algorithm M, intermediate step: no orthonormalisation, R^-1 = I
    for (int idx = threadIdx.x; idx < N * N; idx += CNT) Rinv[idx] = (idx / N == idx % N) ? 1.0 : 0.0;
    if (threadIdx.x == 0 && st) {
      st->reorth = 0;
      st->gram_off_trial = 0.0;
      st->chol_info = 0;
    }
    return;
  }
  const int ld = N + 1;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  double om = 0.0;
  for (int idx = tid; idx < N * N; idx += CNT) {
    const int i = idx / N, j = idx % N;
    const double v = S[idx];
    A[i * ld + j] = v;
    om = fmax(om, fabs(v - (i == j ? 1.0 : 0.0)));
  }
  for (int o = 16; o > 0; o >>= 1) om = fmax(om, __shfl_xor_sync(0xffffffffu, om, o));
  if (lane == 0) offmax[warp] = om;
  __syncthreads();
  if (tid == 0) {
    fail = 0;
    double m = 0.0;
    for (int k = 0; k < N; ++k) m = fmax(m, fabs(A[k * ld + k]));
    dmax = m;
    if (st && reorth_thr >= 0.0) {
      double o = 0.0;
      for (int w = 0; w < CNT / 32; ++w) o = fmax(o, offmax[w]);
      st->gram_off_trial = o;
      // an ill-conditioned trial block loses orthogonality in the FP32 form:
      // ask for a second Cholesky-QR pass
      st->reorth = (reorth_thr > 0.0 && o > reorth_thr) ? 1 : 0;
    }
    if (st && reorth_thr < 0.0) st->reorth_count += 1;
  }
  __syncthreads();

  const int np = (N + NB - 1) / NB;
  // ------------------------------------------------------------ factorisation
  for (int p = 0; p < np; ++p) {
    const int c0 = p * NB, c1 = min(N, c0 + NB);
    if (warp == 0) {
      // diagonal block, right-looking, lane = column c0 + lane
      const int j = c0 + lane;
      for (int k = c0; k < c1; ++k) {
        if (lane == 0) {
          const double d = A[k * ld + k];
          // a pivot at rounding level of the largest diagonal entry means the
          // columns are numerically dependent
          if (!(d > piv_rel * dmax) || !isfinite(d)) {
            fail = k + 1;
          } else {
            const double r = sqrt(d);
            A[k * ld + k] = r;
            rdiag[k] = 1.0 / r;
          }
        }
        __syncwarp();
        if (fail) break;
        const double rk = rdiag[k];
        if (j > k && j < c1) A[k * ld + j] *= rk;
        __syncwarp();
        if (j > k && j < c1) {
          const double akj = A[k * ld + j];
          for (int i = k + 1; i <= j; ++i) A[i * ld + j] -= A[k * ld + i] * akj;
        }
        __syncwarp();
      }
    }
    __syncthreads();
    if (fail) break;
    // panel row: R[c0:c1, j] = R_pp^-T A[c0:c1, j] for j >= c1, one column per thread
    for (int j = c1 + tid; j < N; j += CNT) {
      for (int i = c0; i < c1; ++i) {
        const double x = A[i * ld + j] * rdiag[i];
        A[i * ld + j] = x;
        for (int k = i + 1; k < c1; ++k) A[k * ld + j] -= A[i * ld + k] * x;
      }
    }
    __syncthreads();
    // trailing update of the upper triangle: A[i][j] -= sum_k R[k][i] R[k][j]
    const int m = N - c1;
    if (m > 0) {
      const int mt = (m + 3) / 4;
      const int npairs = mt * (mt + 1) / 2;
      for (int t = tid; t < npairs; t += CNT) {
        // unrank t -> (ti <= tj)
        int ti = 0, rem = t;
        while (rem >= mt - ti) {
          rem -= mt - ti;
          ++ti;
        }
        const int tj = ti + rem;
        const int i0 = c1 + 4 * ti, j0 = c1 + 4 * tj;
        double acc[4][4];
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
          for (int c = 0; c < 4; ++c) acc[r][c] = 0.0;
        for (int k = c0; k < c1; ++k) {
          double a[4], b[4];
#pragma unroll
          for (int r = 0; r < 4; ++r) a[r] = (i0 + r < N) ? A[k * ld + i0 + r] : 0.0;
#pragma unroll
          for (int c = 0; c < 4; ++c) b[c] = (j0 + c < N) ? A[k * ld + j0 + c] : 0.0;
#pragma unroll
          for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[r][c] = fma(a[r], b[c], acc[r][c]);
        }
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            const int i = i0 + r, j = j0 + c;
            if (i < N && j < N && j >= i) A[i * ld + j] -= acc[r][c];
          }
      }
    }
    __syncthreads();
  }
  if (fail) {
    if (tid == 0) {
      if (info) *info = fail;
      if (st) {
        st->chol_info = fail;
        if (soft_limit >= 0 && st->s < soft_limit) {
          st->chol_fail = 1;  // the controller rejects the trial and shrinks the step
        } else {
          st->status = 4;  // POU_ENOTSPD
          st->done = 1;
        }
      }
    }
    return;
  }

  // ------------------------------------------------------------ inverse
  // X[i][j] (i <= j) is stored at A[j][i] for i < j and in rdiag for i == j.
  auto X = [&](int i, int j) -> double { return i == j ? rdiag[i] : A[j * ld + i]; };
  // diagonal blocks: warp p, lane = column, back substitution upward
  if (warp < np) {
    const int c0 = warp * NB, c1 = min(N, c0 + NB);
    const int j = c0 + lane;
    if (j < c1) {
      for (int i = j - 1; i >= c0; --i) {
        double s = 0.0;
        for (int k = i + 1; k <= j; ++k) s = fma(A[i * ld + k], X(k, j), s);
        A[j * ld + i] = -s * rdiag[i];
      }
    }
  }
  __syncthreads();
  // off-diagonal blocks, level d = q - p
  for (int d = 1; d < np; ++d) {
    const int nblk = np - d;  // blocks (p, p + d), p = 0 .. nblk-1
    // T_p = sum_{r=p+1..p+d} R_pr X_r,p+d
    for (int idx = tid; idx < nblk * NB * NB; idx += CNT) {
      const int b = idx / (NB * NB), e = idx % (NB * NB);
      const int r0 = e / NB, cc = e % NB;
      const int p = b, q = b + d;
      const int i = p * NB + r0, j = q * NB + cc;
      double s = 0.0;
      if (i < N && j < N) {
        for (int k = (p + 1) * NB; k <= j; ++k) s = fma(A[i * ld + k], X(k, j), s);
      }
      T[b][r0][cc] = s;
    }
    __syncthreads();
    // X_pq = -X_pp T_p (X_pp upper triangular)
    for (int idx = tid; idx < nblk * NB * NB; idx += CNT) {
      const int b = idx / (NB * NB), e = idx % (NB * NB);
      const int r0 = e / NB, cc = e % NB;
      const int p = b, q = b + d;
      const int i = p * NB + r0, j = q * NB + cc;
      if (i < N && j < N) {
        double s = 0.0;
        const int kend = min(N, (p + 1) * NB);
        for (int k = i; k < kend; ++k) s = fma(X(i, k), T[b][k - p * NB][cc], s);
        A[j * ld + i] = -s;
      }
    }
    __syncthreads();
  }
  for (int idx = tid; idx < N * N; idx += CNT) {
    const int i = idx / N, j = idx % N;
    Rinv[idx] = (j > i) ? A[j * ld + i] : (j == i ? rdiag[i] : 0.0);
  }
  if (tid == 0) {
    if (info) *info = 0;
    if (st) st->chol_info = 0;
  }
}


// ---------------------------------------------------------------------------
// N > 128 (up to 512): the same blocked algorithm on the N x N matrix in
// global memory (it stays in L2), one short kernel per step so that every
// panel's work is spread over many SMs (one SM does about two FP64 FMAs per
// cycle): per 32-wide panel p, (1) factor the diagonal block in shared
// memory, (2) solve the panel row, one column per thread, (3) update the
// trailing upper triangle in 32 x 32 tiles; then invert the diagonal blocks
// and the off-diagonal blocks level by level, and move X = R^-1 into place.
// The working matrix is the output buffer: upper triangle R (1 / R_kk on the
// diagonal, which is also X_kk), strictly lower triangle X^T.
struct BigArgs {
  const State* st;  // gating (done, second pass)
  State* st_rw;     // diagnostics and breakdown status (may be null)
  const double* S;
  double* A;        // N x N working matrix = Rinv
  int N;
  int* flag;        // 0, or 1 + the failing pivot
  double piv_rel, reorth_thr;
  int orth_gated;   // trial pass: skipped (R^-1 = I) on the intermediate steps of Algorithm M
  int soft_limit;   // >= 0: a failing pivot rejects the trial while State::s < soft_limit
};

__device__ __forceinline__ bool big_intermediate(const BigArgs& a) {
  return a.orth_gated && a.st && !a.st->orth_now;
}

__device__ __forceinline__ bool big_gated(const BigArgs& a) {
  if (a.st && a.st->done) return true;
  if (big_intermediate(a)) return true;
  return a.reorth_thr < 0.0 && !(a.st && a.st->reorth);
}

constexpr int BT = 32;  // panel / tile width

// copy S into the working matrix; trial diagnostics as in the small kernel
__global__ void __launch_bounds__(1024) k_big_init(BigArgs a) {
  __shared__ double offmax[32];
  const int N = a.N, tid = threadIdx.x;
  if (a.st && a.st->done) return;
  if (big_intermediate(a)) {
    // Algorithm M, intermediate step: no orthonormalisation, R^-1 = I
    for (i64 idx = tid; idx < (i64)N * N; idx += 1024) a.A[idx] = (idx / N == idx % N) ? 1.0 : 0.0;
    if (tid == 0 && a.st_rw) {
      a.st_rw->reorth = 0;
      a.st_rw->gram_off_trial = 0.0;
      a.st_rw->chol_info = 0;
    }
    return;
  }
  if (big_gated(a)) return;
  double om = 0.0;
  for (i64 idx = tid; idx < (i64)N * N; idx += 1024) {
    const int i = (int)(idx / N), j = (int)(idx % N);
    const double v = a.S[idx];
    a.A[idx] = v;
    om = fmax(om, fabs(v - (i == j ? 1.0 : 0.0)));
  }
  for (int o = 16; o > 0; o >>= 1) om = fmax(om, __shfl_xor_sync(0xffffffffu, om, o));
  if ((tid & 31) == 0) offmax[tid >> 5] = om;
  __syncthreads();
  if (tid == 0) {
    *a.flag = 0;
    if (a.st_rw && a.reorth_thr >= 0.0) {
      double o = 0.0;
      for (int w = 0; w < 32; ++w) o = fmax(o, offmax[w]);
      a.st_rw->gram_off_trial = o;
      a.st_rw->reorth = (a.reorth_thr > 0.0 && o > a.reorth_thr) ? 1 : 0;
    }
    if (a.st_rw && a.reorth_thr < 0.0) a.st_rw->reorth_count += 1;
  }
}

// (1) diagonal block of panel p, one warp, in shared memory
__global__ void __launch_bounds__(32) k_big_diag(BigArgs a, int p) {
  __shared__ double T[BT][BT + 1];
  __shared__ double rd[BT];
  __shared__ volatile int fail;
  if (big_gated(a) || *a.flag) return;
  const int N = a.N, lane = threadIdx.x;
  const int c0 = p * BT, nb = min(BT, N - c0);
  double dm = 0.0;
  for (int k = lane; k < N; k += 32) dm = fmax(dm, fabs(a.S[(i64)k * N + k]));
  for (int o = 16; o > 0; o >>= 1) dm = fmax(dm, __shfl_xor_sync(0xffffffffu, dm, o));
  for (int r = 0; r < nb; ++r)
    if (lane < nb) T[r][lane] = a.A[(i64)(c0 + r) * N + c0 + lane];
  if (lane == 0) fail = 0;
  __syncwarp();
  const int j = lane;
  for (int k = 0; k < nb; ++k) {
    if (lane == 0) {
      const double d = T[k][k];
      if (!(d > a.piv_rel * dm) || !isfinite(d)) {
        fail = c0 + k + 1;
      } else {
        const double r = sqrt(d);
        T[k][k] = r;
        rd[k] = 1.0 / r;
      }
    }
    __syncwarp();
    if (fail) break;
    const double rk = rd[k];
    if (j > k && j < nb) T[k][j] *= rk;
    __syncwarp();
    if (j > k && j < nb) {
      const double akj = T[k][j];
      for (int i = k + 1; i <= j; ++i) T[i][j] -= T[k][i] * akj;
    }
    __syncwarp();
  }
  if (fail) {
    if (lane == 0) {
      *a.flag = fail;
      if (a.st_rw) {
        a.st_rw->chol_info = fail;
        if (a.soft_limit >= 0 && a.st_rw->s < a.soft_limit) {
          a.st_rw->chol_fail = 1;
        } else {
          a.st_rw->status = 4;  // POU_ENOTSPD
          a.st_rw->done = 1;
        }
      }
    }
    return;
  }
  // upper part with 1 / R_kk on the diagonal
  for (int r = 0; r < nb; ++r)
    if (lane < nb && lane >= r) a.A[(i64)(c0 + r) * N + c0 + lane] = lane == r ? rd[r] : T[r][lane];
}

// (2) panel row R[c0:c1, j] = R_pp^-T A[c0:c1, j], j >= c1, one column per thread
__global__ void __launch_bounds__(128) k_big_row(BigArgs a, int p) {
  __shared__ double R[BT][BT + 1];
  if (big_gated(a) || *a.flag) return;
  const int N = a.N, c0 = p * BT, c1 = min(N, c0 + BT), nb = c1 - c0;
  for (int idx = threadIdx.x; idx < BT * BT; idx += 128) {
    const int r = idx / BT, c = idx % BT;
    R[r][c] = (r < nb && c < nb && c >= r) ? a.A[(i64)(c0 + r) * N + c0 + c] : 0.0;
  }
  __syncthreads();
  const int j = c1 + blockIdx.x * 128 + threadIdx.x;
  if (j >= N) return;
  double x[BT];
#pragma unroll
  for (int r = 0; r < BT; ++r) x[r] = r < nb ? a.A[(i64)(c0 + r) * N + j] : 0.0;
#pragma unroll
  for (int i = 0; i < BT; ++i) {
    x[i] *= R[i][i];  // 1 / R_ii
#pragma unroll
    for (int k = i + 1; k < BT; ++k) x[k] -= R[i][k] * x[i];
  }
#pragma unroll
  for (int r = 0; r < BT; ++r)
    if (r < nb) a.A[(i64)(c0 + r) * N + j] = x[r];
}

// (3) trailing update A[i][j] -= sum_k R[k][i] R[k][j] over the panel, tiles bi <= bj
__global__ void __launch_bounds__(256) k_big_update(BigArgs a, int p) {
  __shared__ double Pi[BT][BT + 1], Pj[BT][BT + 1];
  if (big_gated(a) || *a.flag) return;
  const int N = a.N, c0 = p * BT, c1 = min(N, c0 + BT), nb = c1 - c0;
  const int mt = (N - c1 + BT - 1) / BT;
  int bi = 0, rem = blockIdx.x;
  while (rem >= mt - bi) {
    rem -= mt - bi;
    ++bi;
  }
  const int bj = bi + rem;
  const int i0 = c1 + bi * BT, j0 = c1 + bj * BT;
  for (int idx = threadIdx.x; idx < BT * BT; idx += 256) {
    const int k = idx / BT, c = idx % BT;
    Pi[k][c] = (k < nb && i0 + c < N) ? a.A[(i64)(c0 + k) * N + i0 + c] : 0.0;
    Pj[k][c] = (k < nb && j0 + c < N) ? a.A[(i64)(c0 + k) * N + j0 + c] : 0.0;
  }
  __syncthreads();
  // thread: row ii = tid / 8, columns 4 (tid % 8) .. + 3
  const int ii = threadIdx.x >> 3, jj = (threadIdx.x & 7) * 4;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int k = 0; k < nb; ++k) {
    const double u = Pi[k][ii];
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[c] = fma(u, Pj[k][jj + c], acc[c]);
  }
  const int i = i0 + ii;
  if (i >= N) return;
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const int jc = j0 + jj + c;
    if (jc < N) a.A[(i64)i * N + jc] -= acc[c];
  }
}

// inverse of the diagonal blocks: X_pp = R_pp^-1, X^T into the lower triangle
__global__ void __launch_bounds__(32) k_big_invdiag(BigArgs a) {
  __shared__ double T[BT][BT + 1];
  if (big_gated(a) || *a.flag) return;
  const int N = a.N, c0 = blockIdx.x * BT, nb = min(BT, N - c0), lane = threadIdx.x;
  for (int r = 0; r < nb; ++r)
    if (lane < nb) T[r][lane] = lane >= r ? a.A[(i64)(c0 + r) * N + c0 + lane] : 0.0;
  __syncwarp();
  // column j = lane: back substitution upward; X kept in T's lower part as X^T
  const int j = lane;
  if (j < nb) {
    for (int i = j - 1; i >= 0; --i) {
      double s = 0.0;
      for (int k = i + 1; k <= j; ++k) s = fma(T[i][k], k == j ? T[j][j] : T[j][k], s);
      T[j][i] = -s * T[i][i];
    }
  }
  __syncwarp();
  for (int r = 0; r < nb; ++r)
    if (lane < r) a.A[(i64)(c0 + r) * N + c0 + lane] = T[r][lane];
}

// one level of the inverse: blocks (p, p + d), X_pq = -X_pp sum_{r=p+1..q} R_pr X_rq
__global__ void __launch_bounds__(256) k_big_invlevel(BigArgs a, int d) {
  __shared__ double Tq[BT][BT + 1];
  if (big_gated(a) || *a.flag) return;
  const int N = a.N, pb = blockIdx.x, qb = pb + d;
  const int pi0 = pb * BT, qj0 = qb * BT;
  const int ii = threadIdx.x >> 3, jj = (threadIdx.x & 7) * 4;
  const int i = pi0 + ii;
  auto X = [&](int k, int jc) -> double {  // X[k][jc], k <= jc
    return k == jc ? a.A[(i64)k * N + k] : (k < jc ? a.A[(i64)jc * N + k] : 0.0);
  };
  double t[4] = {0.0, 0.0, 0.0, 0.0};
  if (i < N) {
    const int kend = min(N, qj0 + BT);
    for (int k = pi0 + BT; k < kend; ++k) {
      const double r = a.A[(i64)i * N + k];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int jc = qj0 + jj + c;
        if (jc < N) t[c] = fma(r, X(k, jc), t[c]);
      }
    }
  }
#pragma unroll
  for (int c = 0; c < 4; ++c) Tq[ii][jj + c] = t[c];
  __syncthreads();
  if (i >= N) return;
  const int kend = min(N, pi0 + BT);
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const int jc = qj0 + jj + c;
    if (jc >= N) continue;
    double s = 0.0;
    for (int k = i; k < kend; ++k) s = fma(X(i, k), Tq[k - pi0][jj + c], s);
    a.A[(i64)jc * N + i] = -s;
  }
}

// X^T (lower) to X (upper), zero lower; status
__global__ void __launch_bounds__(256) k_big_final(BigArgs a, int* info) {
  if (big_gated(a) || *a.flag) return;
  const int N = a.N;
  const i64 np = (i64)N * (N - 1) / 2;
  for (i64 t = blockIdx.x * 256 + threadIdx.x; t < np; t += (i64)gridDim.x * 256) {
    // unrank t -> (i < j), row-major over the strict upper triangle
    int i = (int)((2.0 * N - 1.0 - sqrt((2.0 * N - 1.0) * (2.0 * N - 1.0) - 8.0 * (double)t)) / 2.0);
    i = max(0, min(i, N - 2));
    while (i > 0 && (i64)i * (2 * N - i - 1) / 2 > t) --i;
    while ((i64)(i + 1) * (2 * N - i - 2) / 2 <= t) ++i;
    const int j = (int)(t - (i64)i * (2 * N - i - 1) / 2) + i + 1;
    a.A[(i64)i * N + j] = a.A[(i64)j * N + i];
    a.A[(i64)j * N + i] = 0.0;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    if (info) *info = 0;
    if (a.st_rw) a.st_rw->chol_info = 0;
  }
}

void launch_cholinv_big(const State* st, const double* S, double* Rinv, int N, int* info, State* st_rw,
                        double piv_rel, double reorth_thr, cudaStream_t s, bool orth_gated, int soft_limit) {
  // the failing-pivot flag: the caller's info, else the iteration state's chol_info
  if (!info && !st_rw) return;
  BigArgs a{st,       st_rw,      S, Rinv, N, info ? info : &st_rw->chol_info, piv_rel, reorth_thr,
            orth_gated ? 1 : 0, soft_limit};
  const int np = (N + BT - 1) / BT;
  k_big_init<<<1, 1024, 0, s>>>(a);
  for (int p = 0; p < np; ++p) {
    k_big_diag<<<1, 32, 0, s>>>(a, p);
    const int c1 = std::min(N, (p + 1) * BT);
    if (c1 < N) {
      k_big_row<<<(N - c1 + 127) / 128, 128, 0, s>>>(a, p);
      const int mt = (N - c1 + BT - 1) / BT;
      k_big_update<<<mt * (mt + 1) / 2, 256, 0, s>>>(a, p);
    }
  }
  k_big_invdiag<<<np, 32, 0, s>>>(a);
  for (int d = 1; d < np; ++d) k_big_invlevel<<<np - d, 256, 0, s>>>(a, d);
  k_big_final<<<std::max(1, std::min(num_sms(), (N * (N - 1) / 2 + 255) / 256)), 256, 0, s>>>(a, info);
}
}  // namespace

size_t cholinv_smem_bytes(int N) { return sizeof(double) * (size_t)N * (N + 1); }

void configure_cholinv() {
  cudaFuncSetAttribute(k_cholinv, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cholinv_smem_bytes(128));
}

void launch_cholinv(const State* st, const double* S, double* Rinv, int N, int* info, State* st_rw,
                    double piv_rel, double reorth_thr, cudaStream_t s, bool orth_gated, int soft_limit) {
  prof_begin("cholinv", s);
  if (N <= 128) {  // one CTA is faster here than the multi-kernel path (0.34 vs 0.38 ms)
    k_cholinv<<<1, CNT, cholinv_smem_bytes(N), s>>>(st, st_rw, S, Rinv, N, info, piv_rel, reorth_thr,
                                                     orth_gated ? 1 : 0, soft_limit);
  } else {
    launch_cholinv_big(st, S, Rinv, N, info, st_rw, piv_rel, reorth_thr, s, orth_gated, soft_limit);
  }
  prof_end(s);
}

}  // namespace pou
