// OptM-QR direction (Sec. 3.1, the comparison method of Table 1): the search
// direction of every orbital uses the full Lagrange-multiplier matrix,
//   Z = HW - W Sigma,   Sigma = <W^T HW>   (z_i = hw_i - sum_j Sigma_ji w_j),
// instead of Opt-Par's z_i = hw_i - sigma_ii w_i.  It is also the gradient of
// Eq. (gra).  The Barzilai-Borwein step uses S = W - W', Y = Z - Z' of the
// previous iterate (its own Z', not Opt-Par's).
//
// k_direction, per chunk of RP grid points and every orbital block:
//   * z_i = hw_i - sum_j S_ij w_j with S = <W^T HW> of the current pair
//     (S_ij = <w_i, hw_j> = Sigma_ji), the W chunk staged in shared memory
//     like the residual kernel; Z is written to Z[cur];
//   * per orbital, the raw sums <w,w>, <w,z>, <z,z> (no dV), from which the
//     controller takes ||Z||_F^2 and the Gram kernels' reduction the trial
//     column norms ||w - tau z||^2;
//   * with a previous iterate (step l > 0): tr S^T S, tr S^T Y, tr Y^T Y from
//     W' = W[1-cur] and Z' = Z[1-cur].
// k_direction_control (one CTA) reduces the partials and sets the step's
// tau (tau^1 or tau^2 as in Opt-Par, tau_0 at l = 0) and ||Z||_F^2.  Both run
// on the first pass of a step only (State::s == 0); a backtracking pass keeps
// Z and shrinks tau.
#include "pou_internal.cuh"

namespace pou {

namespace {

constexpr int DNT = 256;
constexpr int DP = 64;     // grid points per chunk
constexpr int NPAD = 128;  // orbital block
constexpr int XS = DP + 4;

template <typename T>
__global__ void __launch_bounds__(DNT) k_direction(DirArgs<T> a, int nchunks) {
  if (a.st->done || a.st->s != 0) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* Ss = reinterpret_cast<T*>(smem_raw);        // [NPAD][NPAD]: Ss[j][i] = S_(ib+i)(jb+j)
  T* Xs = Ss + NPAD * NPAD;                       // [NPAD][XS]: chunk of W, orbitals jb ..
  double* acc = reinterpret_cast<double*>(Xs + NPAD * XS);  // [2][N][3] per-orbital sums, one set per point half
  __shared__ double red[DNT / 32][3];
  const int N = a.N;
  const i64 ng = a.ng;
  const int cur = a.st->cur;
  const bool hist = a.st->l > 0;
  const T* W = a.W[cur];
  const T* HW = a.HW[cur];
  const T* Wp = a.W[1 - cur];
  const T* Zp = a.Z[1 - cur];
  T* Z = a.Z[cur];
  const int tid = threadIdx.x;
  for (int idx = tid; idx < 2 * N * 3; idx += DNT) acc[idx] = 0.0;
  const int nb = (N + NPAD - 1) / NPAD;
  auto load_sig = [&](int ib, int jb) {
    for (int idx = tid; idx < NPAD * NPAD; idx += DNT) {
      const int j = idx / NPAD, i = idx % NPAD;
      const int gi = ib * NPAD + i, gj = jb * NPAD + j;
      Ss[idx] = (gi < N && gj < N) ? (T)a.Sig[(i64)gi * N + gj] : T(0);
    }
  };
  if (nb == 1) load_sig(0, 0);
  const int lane = tid & 31, warp = tid >> 5;
  const int iw = warp & 3, pw = warp >> 2;
  const int ig = lane & 3, pg = lane >> 2;
  const int i0 = iw * 32 + ig * 8;   // 8 orbitals of the block
  const int pl0 = pw * 32 + pg * 4;  // 4 points of the chunk
  double bss = 0.0, bsy = 0.0, byy = 0.0;
  for (int ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
    const i64 p0 = (i64)ch * DP;
    for (int ib = 0; ib < nb; ++ib) {
      T sum[8][4];
#pragma unroll
      for (int ii = 0; ii < 8; ++ii)
#pragma unroll
        for (int q = 0; q < 4; ++q) sum[ii][q] = T(0);
      for (int jb = 0; jb < nb; ++jb) {
        const int nj = min(NPAD, N - jb * NPAD);
        __syncthreads();
        if (nb > 1) load_sig(ib, jb);
        for (int idx = tid; idx < nj * DP; idx += DNT) {
          const int j = idx / DP, pp = idx % DP;
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
            for (int q = 0; q < 4; ++q) sum[ii][q] = fma(sv[ii], xv[q], sum[ii][q]);
        }
      }
      // z = hw - sum; sums of this thread's 4 points for each of its 8 orbitals
      T ss = T(0), sy = T(0), yy = T(0);
#pragma unroll
      for (int ii = 0; ii < 8; ++ii) {
        const int i = ib * NPAD + i0 + ii;
        T ww = T(0), wz = T(0), zz = T(0);
        if (i < N) {
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const i64 gp = p0 + pl0 + q;
            if (gp >= ng) continue;
            const i64 e = (i64)i * ng + gp;
            const T w = W[e];
            const T z = HW[e] - sum[ii][q];
            Z[e] = z;
            ww = fma(w, w, ww);
            wz = fma(w, z, wz);
            zz = fma(z, z, zz);
            if (hist) {
              const T s = w - Wp[e];
              const T y = z - Zp[e];
              ss = fma(s, s, ss);
              sy = fma(s, y, sy);
              yy = fma(y, y, yy);
            }
          }
        }
        // the 8 lanes of a warp holding the same orbitals (same ig): sum over pg
        T v3[3] = {ww, wz, zz};
#pragma unroll
        for (int k = 0; k < 3; ++k) {
#pragma unroll
          for (int o = 4; o < 32; o <<= 1) v3[k] += __shfl_xor_sync(0xffffffffu, v3[k], o);
        }
        if (pg == 0 && i < N) {
#pragma unroll
          for (int k = 0; k < 3; ++k) acc[((i64)pw * N + i) * 3 + k] += (double)v3[k];
        }
      }
      bss += (double)ss;
      bsy += (double)sy;
      byy += (double)yy;
    }
  }
  // Barzilai-Borwein partials of the CTA
  double b3[3] = {bss, bsy, byy};
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    double v = b3[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[warp][k] = v;
  }
  __syncthreads();
  if (tid < 3) {
    double v = 0.0;
    for (int wi = 0; wi < DNT / 32; ++wi) v += red[wi][tid];
    a.bpart[(i64)blockIdx.x * 3 + tid] = v;
  }
  for (int idx = tid; idx < N * 3; idx += DNT) a.opart[(i64)blockIdx.x * N * 3 + idx] = acc[idx] + acc[N * 3 + idx];
}

__global__ void __launch_bounds__(256) k_direction_control(DirCtrlArgs a) {
  State* st = a.st;
  if (st->done || st->s != 0) return;
  __shared__ double sh[3];
  __shared__ double zred[256 / 32];
  const int tid = threadIdx.x, N = a.N;
  double zz = 0.0;
  for (int idx = tid; idx < N * 3; idx += 256) {
    double v = 0.0;
    for (int b = 0; b < a.nblk; ++b) v += a.opart[(i64)b * N * 3 + idx];
    a.dpart[idx] = v;
    if (idx % 3 == 2) zz += v;
  }
  if (tid < 3) {
    double v = 0.0;
    for (int b = 0; b < a.nblk; ++b) v += a.bpart[(i64)b * 3 + tid];
    sh[tid] = v;
  }
  for (int o = 16; o > 0; o >>= 1) zz += __shfl_xor_sync(0xffffffffu, zz, o);
  if ((tid & 31) == 0) zred[tid >> 5] = zz;
  __syncthreads();
  if (tid != 0) return;
  double zt = 0.0;
  for (int w = 0; w < 256 / 32; ++w) zt += zred[w];
  st->znorm2 = a.dV * zt;
  double tau = a.tau0;
  if (st->l > 0) {
    const double ss = a.dV * sh[0], sy = fabs(a.dV * sh[1]), yy = a.dV * sh[2];
    int variant = a.bb_variant;
    if (variant == 3) variant = (st->l % 2 == 0) ? 1 : 2;
    tau = (variant == 1) ? (sy > 0.0 ? ss / sy : NAN) : (yy > 0.0 ? sy / yy : NAN);
    if (!isfinite(tau) || tau <= 0.0) tau = a.tau0;
  }
  tau = fmin(fmax(tau, a.tau_min), a.tau_max);
  st->tau_bb = tau;
  st->tau_trial = tau;
}

template <typename T>
size_t direction_smem(int N) {
  return (size_t)(NPAD * NPAD + NPAD * XS) * sizeof(T) + (size_t)2 * N * 3 * sizeof(double);
}

}  // namespace

int direction_grid(i64 ng) {
  const i64 nchunks = (ng + DP - 1) / DP;
  return (int)std::max<i64>(1, std::min<i64>(nchunks, num_sms()));
}

void configure_direction() {
  cudaFuncSetAttribute(k_direction<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)direction_smem<float>(POU_DIR_MAX_N));
  cudaFuncSetAttribute(k_direction<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)direction_smem<double>(POU_DIR_MAX_N_FP64));
}

template <typename T>
void launch_direction(const DirArgs<T>& a, cudaStream_t s) {
  const int nchunks = (int)((a.ng + DP - 1) / DP);
  prof_begin("direction_full", s);
  k_direction<T><<<direction_grid(a.ng), DNT, direction_smem<T>(a.N), s>>>(a, nchunks);
  prof_end(s);
}
template void launch_direction<float>(const DirArgs<float>&, cudaStream_t);
template void launch_direction<double>(const DirArgs<double>&, cudaStream_t);

void launch_direction_control(const DirCtrlArgs& a, cudaStream_t s) {
  prof_begin("direction_control", s);
  k_direction_control<<<1, 256, 0, s>>>(a);
  prof_end(s);
}

}  // namespace pou
