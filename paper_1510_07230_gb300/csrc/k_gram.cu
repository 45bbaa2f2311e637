// Cholesky-QR contractions of Sec. 3.2 on CUDA cores:
//   * Gram S = <Wt^T Wt> of the trial block Wt = W - tau Z
//     = (1 + tau sigma_i) w_i - tau hw_i, formed on the fly from W and HW
//     (so Z is never stored), split over the grid dimension with one FP64
//     partial per split and a deterministic reduction;
//   * rotation W_new = Wt R^-1 (R^-1 upper triangular) fused with the
//     density rho = f sum_j w_new_j^2.
// In the FP32 form every product is an FP32 FMA (round to nearest); the
// split partials are FP64.  The coefficients (1 + tau sigma_i) and tau are
// rounded to the working type once and the same rounded values are used by
// the Gram, the exact FP64 Gram diagonal and the rotation, so that the
// normalisation of every new orbital is consistent to FP64 accuracy.
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

__device__ __forceinline__ void tri_index(int t, int* ti, int* tj) {
  int r = 0, rem = t;
  while (rem >= 16 - r) {
    rem -= 16 - r;
    ++r;
  }
  *ti = r;
  *tj = r + rem;
}

template <typename T>
__device__ __forceinline__ T trial_value(const T* W, const T* H, T coef, T tau, i64 off) {
  // (1 + tau sigma) w - tau hw
  return coef * W[off] - tau * H[off];
}

template <typename T>
__global__ void __launch_bounds__(GNT) k_gram(GramArgs<T> a, i64 chunk, int nsup, int npair) {
  constexpr int RT = GT<T>::RT, ST = GT<T>::ST, BK = GT<T>::BK;
  __shared__ __align__(16) T As[BK][ST + 4];
  __shared__ __align__(16) T Bs[BK][ST + 4];
  __shared__ T coefs[ST], coefs2[ST];

  if (a.st && a.st->done) return;
  const bool general = (a.B != nullptr);
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
  int ti = 0, tj = 0;
  bool active = true;
  if (diag) {
    if (tid < 136)
      tri_index(tid, &ti, &tj);
    else
      active = false;
  } else {
    ti = tid / 16;
    tj = tid % 16;
  }

  const i64 ng = a.ng;
  const int N = a.N;
  const i64 k0 = (i64)blockIdx.x * chunk;
  const i64 k1 = min(ng, k0 + chunk);

  const T* Wa;
  const T* Ha = nullptr;
  const T* Bsrc;
  T tauT = T(0);
  if (a.trial) {
    const int cur = a.st->cur;
    Wa = a.W[cur];
    Ha = a.HW[cur];
    Bsrc = Wa;
    const double tau = a.st->tau_trial;
    tauT = (T)tau;
    for (int r = tid; r < ST; r += GNT) {
      const int gi = I * ST + r, gj = J * ST + r;
      coefs[r] = gi < N ? (T)(1.0 + tau * a.sigma[cur][gi]) : T(0);
      coefs2[r] = gj < N ? (T)(1.0 + tau * a.sigma[cur][gj]) : T(0);
    }
  } else {
    Wa = a.A;
    Bsrc = general ? a.B : a.A;
  }
  __syncthreads();

  T acc[RT][RT];
#pragma unroll
  for (int r = 0; r < RT; ++r)
#pragma unroll
    for (int c = 0; c < RT; ++c) acc[r][c] = T(0);

  for (i64 kk = k0; kk < k1; kk += BK) {
    for (int idx = tid; idx < ST * BK; idx += GNT) {
      const int r = idx / BK, k = idx % BK;
      const int gi = I * ST + r;
      const i64 gk = kk + k;
      T v = T(0);
      if (gi < N && gk < k1) {
        const i64 off = (i64)gi * ng + gk;
        v = a.trial ? trial_value(Wa, Ha, coefs[r], tauT, off) : Wa[off];
      }
      As[k][r] = v;
      if (!diag) {
        const int gj = J * ST + r;
        T u = T(0);
        if (gj < N && gk < k1) {
          const i64 off = (i64)gj * ng + gk;
          u = a.trial ? trial_value(Wa, Ha, coefs2[r], tauT, off) : Bsrc[off];
        }
        Bs[k][r] = u;
      }
    }
    __syncthreads();
    if (active) {
      const T(*Bt)[ST + 4] = diag ? As : Bs;
#pragma unroll 4
      for (int k = 0; k < BK; ++k) {
        T av[RT], bv[RT];
#pragma unroll
        for (int r = 0; r < RT; ++r) av[r] = As[k][ti * RT + r];
#pragma unroll
        for (int c = 0; c < RT; ++c) bv[c] = Bt[k][tj * RT + c];
#pragma unroll
        for (int r = 0; r < RT; ++r)
#pragma unroll
          for (int c = 0; c < RT; ++c) acc[r][c] = fma(av[r], bv[c], acc[r][c]);
      }
    }
    __syncthreads();
  }

  if (!active) return;
  double* out = a.split + ((i64)blockIdx.x * npair + p) * (i64)(ST * ST);
#pragma unroll
  for (int r = 0; r < RT; ++r)
#pragma unroll
    for (int c = 0; c < RT; ++c) out[(ti * RT + r) * ST + tj * RT + c] = (double)acc[r][c];
}

__global__ void k_gram_reduce(GramReduceArgs a) {
  if (a.st && a.st->done) return;
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
  for (int k = 0; k < a.nsplit; ++k) s += a.split[off + k * stride];
  s *= a.dV;
  if (a.trial && r == c) {
    // exact FP64 norm of the trial column from the H-apply sums of W[cur]:
    // ||a w - tau hw||^2 = a^2 <w,w> - 2 a tau <w,hw> + tau^2 <hw,hw>
    const int cur = a.st->cur;
    const double tau = a.st->tau_trial;
    double coef = 1.0 + tau * a.sigma[cur][r];
    double t = tau;
    if (a.fp32_coef) {
      coef = (double)(float)coef;
      t = (double)(float)tau;
    }
    const double* pp = a.part[cur] + (i64)r * NP;
    s = a.dV * (coef * coef * pp[P_WW] - 2.0 * coef * t * pp[P_HW] + t * t * pp[P_HH]);
  }
  a.S[(i64)r * N + c] = s;
  if (!a.general) a.S[(i64)c * N + r] = s;
}

// --------------------------------------------------------------- rotation
constexpr int RNT = 256;
constexpr int RP = 64;  // points per chunk

template <typename T>
__global__ void __launch_bounds__(RNT) k_rotate(RotArgs<T> a, int nchunks) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int N = a.N;
  const int NPAD = 128;
  T* Rs = reinterpret_cast<T*>(smem_raw);                 // [NPAD][NPAD]
  T* Xs = Rs + NPAD * NPAD;                               // [NPAD][RP + 4]
  T* Rlo = Xs + NPAD * (RP + 4);                          // [NPAD] low part of the diagonal
  T* coefs = Rlo + NPAD;                                  // [NPAD]
  float* rsum = reinterpret_cast<float*>(coefs + NPAD);   // [4][RP]
  constexpr int XS = RP + 4;

  if (a.st && a.st->done) return;
  const int tid = threadIdx.x;
  int cur = 0;
  const T* Wsrc;
  const T* Hsrc = nullptr;
  T* out;
  double* rho;
  T tauT = T(0);
  if (a.trial) {
    cur = a.st->cur;
    Wsrc = a.W[cur];
    Hsrc = a.HW[cur];
    out = a.Wout[1 - cur];
    rho = a.rho[1 - cur];
    const double tau = a.st->tau_trial;
    tauT = (T)tau;
    for (int i = tid; i < NPAD; i += RNT) coefs[i] = i < N ? (T)(1.0 + tau * a.sigma[cur][i]) : T(0);
  } else if (a.st) {
    cur = a.st->cur;
    Wsrc = a.A;
    out = a.Wout[1 - cur];
    rho = a.rho[1 - cur];
  } else {
    Wsrc = a.A;
    out = a.B;
    rho = a.rho_out;
  }
  for (int idx = tid; idx < NPAD * NPAD; idx += RNT) {
    const int i = idx / NPAD, j = idx % NPAD;
    const double v = (i < N && j < N) ? a.Rinv[(i64)i * N + j] : 0.0;
    Rs[idx] = (T)v;
    if (i == j) Rlo[i] = (T)(v - (double)(T)v);
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
      T v = T(0);
      if (gp < ng) {
        const i64 off = (i64)i * ng + gp;
        v = a.trial ? coefs[i] * Wsrc[off] - tauT * Hsrc[off] : Wsrc[off];
      }
      Xs[i * XS + pp] = v;
    }
    __syncthreads();

    T acc[8][4];
#pragma unroll
    for (int jj = 0; jj < 8; ++jj)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[jj][q] = T(0);
    for (int i = 0; i < imax; ++i) {
      T rv[8], xv[4];
#pragma unroll
      for (int jj = 0; jj < 8; ++jj) rv[jj] = Rs[i * NPAD + j0 + jj];
#pragma unroll
      for (int q = 0; q < 4; ++q) xv[q] = Xs[i * XS + pl0 + q];
#pragma unroll
      for (int jj = 0; jj < 8; ++jj)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[jj][q] = fma(rv[jj], xv[q], acc[jj][q]);
    }
    // low part of the diagonal of R^-1 (zero in FP64)
#pragma unroll
    for (int jj = 0; jj < 8; ++jj) {
      const int j = j0 + jj;
      if (j < N) {
        const T lo = Rlo[j];
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[jj][q] = fma(lo, Xs[j * XS + pl0 + q], acc[jj][q]);
      }
    }
    // store and density
    float sq[4] = {0.f, 0.f, 0.f, 0.f};
    double sqd[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
    for (int jj = 0; jj < 8; ++jj) {
      const int j = j0 + jj;
      if (j < N) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const i64 gp = p0 + pl0 + q;
          if (gp < ng) out[(i64)j * ng + gp] = acc[jj][q];
          if (sizeof(T) == 8)
            sqd[q] += (double)acc[jj][q] * (double)acc[jj][q];
          else
            sq[q] += (float)acc[jj][q] * (float)acc[jj][q];
        }
      }
    }
    if (rho != nullptr) {
      if (sizeof(T) == 8) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          sqd[q] += __shfl_xor_sync(0xffffffffu, sqd[q], 1);
          sqd[q] += __shfl_xor_sync(0xffffffffu, sqd[q], 2);
        }
      } else {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          sq[q] += __shfl_xor_sync(0xffffffffu, sq[q], 1);
          sq[q] += __shfl_xor_sync(0xffffffffu, sq[q], 2);
        }
      }
    }
    __syncthreads();  // Xs no longer read; reuse a region for the density
    if (rho != nullptr) {
      double* dsum = reinterpret_cast<double*>(Xs);  // [4][RP]
      if (jg == 0) {
#pragma unroll
        for (int q = 0; q < 4; ++q)
          dsum[jw * RP + pl0 + q] = (sizeof(T) == 8) ? sqd[q] : (double)sq[q];
      }
      __syncthreads();
      if (tid < RP) {
        const i64 gp = p0 + tid;
        if (gp < ng) {
          const double s = dsum[tid] + dsum[RP + tid] + dsum[2 * RP + tid] + dsum[3 * RP + tid];
          rho[gp] = F_OCC * s;
        }
      }
      __syncthreads();
    }
    (void)rsum;
  }
}

template <typename T>
__global__ void k_density(const T* U, i64 ng, int N, double* rho) {
  const i64 p = (i64)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= ng) return;
  double s = 0.0;
  int i = 0;
  while (i < N) {
    T part = T(0);
    const int e = min(N, i + 8);
    for (; i < e; ++i) {
      const T v = U[(i64)i * ng + p];
      part = fma(v, v, part);
    }
    s += (double)part;
  }
  rho[p] = F_OCC * s;
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
  if (b > 152 * 16) b = 152 * 16;
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
  const i64 target = (4 * 152 + np - 1) / np;
  i64 c = (ng + target - 1) / target;
  c = ((c + BK - 1) / BK) * BK;
  c = std::max<i64>(c, 1024);
  c = std::min<i64>(c, 16384);
  *npair = np;
  *chunk = c;
  *nsplit = (int)((ng + c - 1) / c);
}
template void gram_layout<float>(i64, int, bool, int*, int*, i64*);
template void gram_layout<double>(i64, int, bool, int*, int*, i64*);

template <typename T>
void launch_gram(const GramArgs<T>& a, cudaStream_t s) {
  int nsplit, npair;
  i64 chunk;
  gram_layout<T>(a.ng, a.N, a.B != nullptr, &nsplit, &npair, &chunk);
  const int nsup = (a.N + GT<T>::ST - 1) / GT<T>::ST;
  dim3 grid(nsplit, npair);
  prof_begin("gram", s);
  k_gram<T><<<grid, GNT, 0, s>>>(a, chunk, nsup, npair);
  prof_end(s);
}
template void launch_gram<float>(const GramArgs<float>&, cudaStream_t);
template void launch_gram<double>(const GramArgs<double>&, cudaStream_t);

void launch_gram_reduce(const GramReduceArgs& a, cudaStream_t s) {
  dim3 block(32, 8);
  dim3 grid((a.N + 31) / 32, (a.N + 7) / 8);
  prof_begin("gram_reduce", s);
  k_gram_reduce<<<grid, block, 0, s>>>(a);
  prof_end(s);
}

template <typename T>
static size_t rotate_smem() {
  const int NPAD = 128;
  return sizeof(T) * ((size_t)NPAD * NPAD + (size_t)NPAD * (RP + 4) + 2 * NPAD) + sizeof(float) * 4 * RP;
}

void configure_rotate() {
  cudaFuncSetAttribute(k_rotate<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rotate_smem<float>());
  cudaFuncSetAttribute(k_rotate<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rotate_smem<double>());
}

template <typename T>
void launch_rotate(const RotArgs<T>& a, cudaStream_t s) {
  const size_t smem = rotate_smem<T>();
  const int nchunks = (int)((a.ng + RP - 1) / RP);
  const int per_sm = sizeof(T) == 4 ? 2 : 1;
  const int grid = std::min(nchunks, 152 * per_sm);
  prof_begin("rotate_density", s);
  k_rotate<T><<<grid, RNT, smem, s>>>(a, nchunks);
  prof_end(s);
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
