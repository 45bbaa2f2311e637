// Cholesky-QR, middle step (Sec. 3.2): S = R^T R with R upper triangular and
// positive diagonal, then R^-1, in FP64 in one CTA's shared memory.
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

namespace pou {

namespace {

constexpr int CNT = 512;
constexpr int NB = 32;       // panel width
constexpr int MAXB = 4;      // panels for N <= 128

__global__ void __launch_bounds__(CNT) k_cholinv(const State* st_ro, State* st, const double* S,
                                                  double* Rinv, int N, int* info, double piv_rel,
                                                  double reorth_thr) {
  extern __shared__ double A[];  // [N][N+1]: upper = R, strictly lower = X^T
  __shared__ double rdiag[128];  // 1 / R_ii
  __shared__ double T[MAXB - 1][NB][NB + 1];  // sums of one level of the inverse
  __shared__ volatile int fail;
  __shared__ double offmax[CNT / 32];
  __shared__ double dmax;
  if (st_ro && st_ro->done) return;
  if (reorth_thr < 0.0 && !(st_ro && st_ro->reorth)) return;  // gated second pass
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
        st->status = 4;  // POU_ENOTSPD
        st->done = 1;
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

}  // namespace

size_t cholinv_smem_bytes(int N) { return sizeof(double) * (size_t)N * (N + 1); }

void configure_cholinv() {
  cudaFuncSetAttribute(k_cholinv, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cholinv_smem_bytes(128));
}

void launch_cholinv(const State* st, const double* S, double* Rinv, int N, int* info, State* st_rw,
                    double piv_rel, double reorth_thr, cudaStream_t s) {
  const size_t smem = cholinv_smem_bytes(N);
  prof_begin("cholinv", s);
  k_cholinv<<<1, CNT, smem, s>>>(st, st_rw, S, Rinv, N, info, piv_rel, reorth_thr);
  prof_end(s);
}

}  // namespace pou
