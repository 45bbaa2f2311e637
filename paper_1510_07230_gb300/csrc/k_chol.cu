// Cholesky-QR, middle step (Sec. 3.2): S = R^T R with R upper triangular and
// positive diagonal, then R^-1, in FP64 in one CTA's shared memory.
// A non-positive pivot is reported through *info and the iteration state
// (status POU_ENOTSPD, done = 1); no trap, no wait.
// The same kernel records max |S - I| of the trial Gram matrix, the
// near-identity diagnostic of Fig. 2.
#include "pou_internal.cuh"

namespace pou {

namespace {

constexpr int CNT = 512;

__global__ void __launch_bounds__(CNT) k_cholinv(const State* st_ro, State* st, const double* S,
                                                  double* Rinv, int N, int* info, double piv_rel,
                                                  double reorth_thr) {
  extern __shared__ double A[];  // [N][N+1]
  __shared__ int fail;
  __shared__ double offmax[CNT / 32];
  __shared__ double dmax;
  if (st_ro && st_ro->done) return;
  if (reorth_thr < 0.0 && !(st_ro && st_ro->reorth)) return;  // gated second pass
  const int ld = N + 1;
  const int tid = threadIdx.x;
  double om = 0.0;
  for (int idx = tid; idx < N * N; idx += CNT) {
    const int i = idx / N, j = idx % N;
    const double v = S[idx];
    A[i * ld + j] = v;
    om = fmax(om, fabs(v - (i == j ? 1.0 : 0.0)));
  }
  for (int o = 16; o > 0; o >>= 1) om = fmax(om, __shfl_xor_sync(0xffffffffu, om, o));
  if ((tid & 31) == 0) offmax[tid >> 5] = om;
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

  // right-looking factorisation, upper triangle holds R
  for (int k = 0; k < N; ++k) {
    if (tid == 0) {
      const double d = A[k * ld + k];
      // a pivot at rounding level of the largest diagonal entry means the
      // columns are numerically dependent
      if (!(d > piv_rel * dmax) || !isfinite(d)) {
        fail = k + 1;
      } else {
        A[k * ld + k] = sqrt(d);
      }
    }
    __syncthreads();
    if (fail) break;
    const double rkk = A[k * ld + k];
    for (int j = k + 1 + tid; j < N; j += CNT) A[k * ld + j] /= rkk;
    __syncthreads();
    const int m = N - k - 1;
    for (int idx = tid; idx < m * m; idx += CNT) {
      const int i = k + 1 + idx / m, j = k + 1 + idx % m;
      if (j >= i) A[i * ld + j] -= A[k * ld + i] * A[k * ld + j];
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

  // in-place inverse of the upper triangular R, bottom row first:
  // X[i][j] = -(sum_{k=i+1..j} R[i][k] X[k][j]) / R[i][i],  X[i][i] = 1 / R[i][i]
  for (int i = N - 1; i >= 0; --i) {
    const double rii = A[i * ld + i];
    double v[(128 + CNT - 1) / CNT + 1];
    int cnt = 0;
    for (int j = i + tid; j < N; j += CNT) {
      double s;
      if (j == i) {
        s = 1.0 / rii;
      } else {
        s = 0.0;
        for (int k = i + 1; k <= j; ++k) s += A[i * ld + k] * A[k * ld + j];
        s = -s / rii;
      }
      v[cnt++] = s;
    }
    __syncthreads();
    cnt = 0;
    for (int j = i + tid; j < N; j += CNT) A[i * ld + j] = v[cnt++];
    __syncthreads();
  }
  for (int idx = tid; idx < N * N; idx += CNT) {
    const int i = idx / N, j = idx % N;
    Rinv[idx] = (j >= i) ? A[i * ld + j] : 0.0;
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
