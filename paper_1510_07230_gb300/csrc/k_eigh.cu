// Subspace diagonalisation of Algorithm M (Sec. 3.3): the symmetric N x N
// matrix Sigma = <W^T H W> is diagonalised, P^T Sigma P = Gamma, by cyclic
// Jacobi rotations in FP64 in one CTA.  Each sweep visits every (p, q) pair
// once in a round-robin schedule of N-1 rounds of N/2 disjoint pairs, so the
// rotations of one round are applied in parallel: first to the rows, then
// to the columns of A (shared memory), then to the eigenvector rows of
// V^T (global memory).  The sweeps stop when the off-diagonal mass is below
// 1e-30 of the diagonal mass (or after 30 sweeps).
// Output: P (row-major, column j = eigenvector j) and Gamma.
#include "pou_internal.cuh"

namespace pou {

namespace {

constexpr int ENT = 512;

__global__ void __launch_bounds__(ENT) k_eigh(const State* st, const double* Sig, double* P, double* VT,
                                               double* evals_sel0, double* evals_sel1, int N) {
  extern __shared__ double A[];  // [N][N+1]
  __shared__ double cs[64 + 1], sn[64 + 1];
  __shared__ int pp[64 + 1], qq[64 + 1];
  __shared__ double red[ENT / 32][2];
  __shared__ int stop;
  if (st) {
    if (st->done || !st->diag_now) return;
  }
  const int tid = threadIdx.x;
  const int ld = N + 1;
  for (int idx = tid; idx < N * N; idx += ENT) {
    const int i = idx / N, j = idx % N;
    A[i * ld + j] = 0.5 * (Sig[(i64)i * N + j] + Sig[(i64)j * N + i]);
    VT[idx] = (i == j) ? 1.0 : 0.0;
  }
  __syncthreads();
  const int n2 = N + (N & 1);  // an odd N pairs one index with a dummy each round
  const int npairs = n2 / 2;
  for (int sweep = 0; sweep < 30; ++sweep) {
    // convergence: off-diagonal vs diagonal mass
    double off = 0.0, dia = 0.0;
    for (int idx = tid; idx < N * N; idx += ENT) {
      const int i = idx / N, j = idx % N;
      const double v = A[i * ld + j];
      if (i == j)
        dia += v * v;
      else
        off += v * v;
    }
    for (int o = 16; o > 0; o >>= 1) {
      off += __shfl_xor_sync(0xffffffffu, off, o);
      dia += __shfl_xor_sync(0xffffffffu, dia, o);
    }
    if ((tid & 31) == 0) {
      red[tid >> 5][0] = off;
      red[tid >> 5][1] = dia;
    }
    __syncthreads();
    if (tid == 0) {
      double o = 0.0, d = 0.0;
      for (int w = 0; w < ENT / 32; ++w) {
        o += red[w][0];
        d += red[w][1];
      }
      stop = (o <= 1e-30 * d) || (o == 0.0);
    }
    __syncthreads();
    if (stop) break;
    for (int round = 0; round < n2 - 1; ++round) {
      // pairs of the round-robin schedule: position 0 fixed, others rotate
      if (tid < npairs) {
        const int k = tid;
        auto pos = [&](int i) { return i == 0 ? 0 : 1 + (i - 1 + round) % (n2 - 1); };
        int p = pos(k), q = pos(n2 - 1 - k);
        if (p > q) {
          const int t = p;
          p = q;
          q = t;
        }
        double c = 1.0, s = 0.0;
        if (q < N) {
          const double apq = A[p * ld + q];
          if (apq != 0.0) {
            const double app = A[p * ld + p], aqq = A[q * ld + q];
            const double theta = (aqq - app) / (2.0 * apq);
            const double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(1.0 + theta * theta));
            c = 1.0 / sqrt(1.0 + t * t);
            s = t * c;
          }
        }
        cs[k] = c;
        sn[k] = s;
        pp[k] = p;
        qq[k] = q;
      }
      __syncthreads();
      // rows: A <- J^T A
      for (int idx = tid; idx < npairs * N; idx += ENT) {
        const int k = idx / N, j = idx % N;
        const int p = pp[k], q = qq[k];
        if (q >= N || sn[k] == 0.0) continue;
        const double c = cs[k], s = sn[k];
        const double ap = A[p * ld + j], aq = A[q * ld + j];
        A[p * ld + j] = c * ap - s * aq;
        A[q * ld + j] = s * ap + c * aq;
      }
      __syncthreads();
      // columns: A <- A J
      for (int idx = tid; idx < npairs * N; idx += ENT) {
        const int k = idx / N, i = idx % N;
        const int p = pp[k], q = qq[k];
        if (q >= N || sn[k] == 0.0) continue;
        const double c = cs[k], s = sn[k];
        const double ap = A[i * ld + p], aq = A[i * ld + q];
        A[i * ld + p] = c * ap - s * aq;
        A[i * ld + q] = s * ap + c * aq;
      }
      // eigenvectors: V <- V J, stored as rows of V^T
      for (int idx = tid; idx < npairs * N; idx += ENT) {
        const int k = idx / N, i = idx % N;
        const int p = pp[k], q = qq[k];
        if (q >= N || sn[k] == 0.0) continue;
        const double c = cs[k], s = sn[k];
        const double vp = VT[(i64)p * N + i], vq = VT[(i64)q * N + i];
        VT[(i64)p * N + i] = c * vp - s * vq;
        VT[(i64)q * N + i] = s * vp + c * vq;
      }
      __syncthreads();
    }
  }
  __syncthreads();
  // ascending eigenvalues (the order of the columns of P fixes the order in
  // which the next Cholesky-QR orthonormalises the orbitals)
  __shared__ int order[128];
  if (tid == 0) {
    for (int i = 0; i < N; ++i) order[i] = i;
    for (int i = 1; i < N; ++i) {  // insertion sort, stable
      const int k = order[i];
      const double v = A[k * ld + k];
      int j = i - 1;
      while (j >= 0 && A[order[j] * ld + order[j]] > v) {
        order[j + 1] = order[j];
        --j;
      }
      order[j + 1] = k;
    }
  }
  __syncthreads();
  double* evals = evals_sel0;
  if (st) evals = (st->cur == 0) ? evals_sel0 : evals_sel1;
  for (int idx = tid; idx < N * N; idx += ENT) {
    const int i = idx / N, j = idx % N;
    P[idx] = VT[(i64)order[j] * N + i];
  }
  for (int i = tid; i < N; i += ENT) evals[i] = A[order[i] * ld + order[i]];
}

}  // namespace

void configure_eigh() {
  cudaFuncSetAttribute(k_eigh, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)(sizeof(double) * 128 * 129));
}

void launch_eigh(const State* st, const double* Sig, double* P, double* VT, double* ev0, double* ev1, int N,
                 cudaStream_t s) {
  const size_t smem = sizeof(double) * (size_t)N * (N + 1);
  prof_begin("eigh", s);
  k_eigh<<<1, ENT, smem, s>>>(st, Sig, P, VT, ev0, ev1, N);
  prof_end(s);
}

}  // namespace pou
