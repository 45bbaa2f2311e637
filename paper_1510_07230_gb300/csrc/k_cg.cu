// Conjugate-gradient subproblem solver (config solver = 1): Sec. 3.1 lists
// the conjugate gradient method among the solvers of the per-orbital
// subproblems.  Each orbital moves along
//   d_i = z_i + beta_i (d_i' - gamma_i w_i),   z_i = hw_i - sigma_ii w_i,
// with the Polak-Ribiere coefficient beta_i = max(0, <z_i, z_i - z_i'> /
// <z_i', z_i'>) (the previous direction d_i' projected off w_i, gamma_i =
// <w_i, d_i'>), capped so that <z_i, d_i> >= <z_i, z_i> / 2, and takes the
// Newton step of its frozen-potential Rayleigh quotient along d_i:
//   tau_i = <z_i, d_i> / <d_i, (H - sigma_ii) d_i>
// (tau_0 where that is not a positive number).  The trial point is
// w_i - tau delta^s f_i d_i with tau the mean of the tau_i and f_i = tau_i / tau.
//
// One pass of a step (State::s == 0 only; a backtracking pass keeps D):
//   k_cg_dots   per orbital <z,z>, <z,z'>, <z',z'>, <z,d'>, <w,d'>, <z,w>
//   k_cg_beta   beta_i, gamma_i
//   k_cg_form   D[cur] = d, Zs[cur] = z, per orbital <w,w>, <w,d>, <d,d>, <z,d>
//   H-apply on D[cur] (mode 4): <d,d>, <d, H d>
//   k_cg_step   tau_i, tau, f_i, the trial-diagonal sums and sum_i f_i <z_i, d_i>
// Grid of the two streaming kernels: (chunks of the grid, orbitals); each CTA
// writes its per-orbital partial sums, reduced in a fixed order by the
// one-CTA kernels.
#include "pou_internal.cuh"

namespace pou {

namespace {

constexpr int CNT = 256;
constexpr int SUB = 16;  // FP32 products accumulated per thread before promotion to FP64

__device__ __forceinline__ double cta_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  double r = 0.0;
  for (int w = 0; w < CNT / 32; ++w) r += sh[w];
  return r;
}

template <typename T>
__global__ void __launch_bounds__(CNT) k_cg_dots(CgArgs<T> a) {
  const State* st = a.st;
  if (st->done || st->s != 0 || st->l == 0) return;
  __shared__ double sh[CNT / 32];
  const int cur = st->cur, i = blockIdx.y;
  const i64 ng = a.ng, base = (i64)i * ng;
  const T* w = a.W[cur] + base;
  const T* hw = a.HW[cur] + base;
  const T* zp = a.Zs[1 - cur] + base;
  const T* dp = a.D[1 - cur] + base;
  const T sig = (T)a.sigma[cur][i];
  double acc[CG_NS] = {0, 0, 0, 0, 0, 0};
  T part[CG_NS] = {0, 0, 0, 0, 0, 0};
  int cnt = 0;
  for (i64 p = (i64)blockIdx.x * CNT + threadIdx.x; p < ng; p += (i64)gridDim.x * CNT) {
    const T wv = w[p], z = hw[p] - sig * wv, zo = zp[p], dv = dp[p];
    part[0] += z * z;
    part[1] += z * zo;
    part[2] += zo * zo;
    part[3] += z * dv;
    part[4] += wv * dv;
    part[5] += z * wv;
    if (++cnt == SUB) {
      for (int k = 0; k < CG_NS; ++k) {
        acc[k] += (double)part[k];
        part[k] = T(0);
      }
      cnt = 0;
    }
  }
  for (int k = 0; k < CG_NS; ++k) {
    const double v = cta_sum(acc[k] + (double)part[k], sh);
    if (threadIdx.x == 0) a.opart[((i64)i * a.nch + blockIdx.x) * CG_NS + k] = v;
  }
}

template <typename T>
__global__ void __launch_bounds__(CNT) k_cg_form(CgArgs<T> a) {
  const State* st = a.st;
  if (st->done || st->s != 0) return;
  __shared__ double sh[CNT / 32];
  const int cur = st->cur, i = blockIdx.y;
  const i64 ng = a.ng, base = (i64)i * ng;
  const T* w = a.W[cur] + base;
  const T* hw = a.HW[cur] + base;
  const T* dp = a.D[1 - cur] + base;
  T* d = a.D[cur] + base;
  T* zs = a.Zs[cur] + base;
  const T sig = (T)a.sigma[cur][i];
  const bool hist = st->l > 0;
  const T beta = hist ? (T)a.coef[2 * i] : T(0), gamma = hist ? (T)a.coef[2 * i + 1] : T(0);
  double acc[4] = {0, 0, 0, 0};
  T part[4] = {0, 0, 0, 0};
  int cnt = 0;
  for (i64 p = (i64)blockIdx.x * CNT + threadIdx.x; p < ng; p += (i64)gridDim.x * CNT) {
    const T wv = w[p], z = hw[p] - sig * wv;
    const T dv = hist ? z + beta * (dp[p] - gamma * wv) : z;
    d[p] = dv;
    zs[p] = z;
    part[0] += wv * wv;
    part[1] += wv * dv;
    part[2] += dv * dv;
    part[3] += z * dv;
    if (++cnt == SUB) {
      for (int k = 0; k < 4; ++k) {
        acc[k] += (double)part[k];
        part[k] = T(0);
      }
      cnt = 0;
    }
  }
  for (int k = 0; k < 4; ++k) {
    const double v = cta_sum(acc[k] + (double)part[k], sh);
    if (threadIdx.x == 0) a.opart[((i64)i * a.nch + blockIdx.x) * CG_NS + k] = v;
  }
}

// beta_i and gamma_i from the k_cg_dots sums (raw, without dV)
__global__ void __launch_bounds__(CNT) k_cg_beta(CgCtrlArgs a) {
  const State* st = a.st;
  if (st->done || st->s != 0 || st->l == 0) return;
  for (int i = threadIdx.x; i < a.N; i += CNT) {
    double v[CG_NS] = {0, 0, 0, 0, 0, 0};
    for (int b = 0; b < a.nch; ++b)
      for (int k = 0; k < CG_NS; ++k) v[k] += a.opart[((i64)i * a.nch + b) * CG_NS + k];
    const double zz = v[0], zzp = v[1], zpzp = v[2], zdp = v[3], wdp = v[4], zw = v[5];
    const double gamma = a.dV * wdp;                // <w, d'> with <w, w> = 1
    double beta = zpzp > 0.0 ? fmax(zz - zzp, 0.0) / zpzp : 0.0;
    const double zd = zdp - gamma * zw;             // <z, d' - gamma w>
    if (zd < 0.0) beta = fmin(beta, 0.5 * zz / (-zd));
    if (!isfinite(beta)) beta = 0.0;
    a.coef[2 * i] = beta;
    a.coef[2 * i + 1] = gamma;
  }
}

// per-orbital Newton steps, their mean tau and the factors f_i; the sums for
// the trial-column norms; the Eq. (ene-de) decrease sum_i f_i <z_i, d_i>
__global__ void __launch_bounds__(CNT) k_cg_step(CgCtrlArgs a) {
  State* st = a.st;
  if (st->done || st->s != 0) return;
  __shared__ double sh[CNT / 32];
  __shared__ double tsum;
  const int cur = st->cur;
  double tloc = 0.0;
  for (int i = threadIdx.x; i < a.N; i += CNT) {
    double v[4] = {0, 0, 0, 0};
    for (int b = 0; b < a.nch; ++b)
      for (int k = 0; k < 4; ++k) v[k] += a.opart[((i64)i * a.nch + b) * CG_NS + k];
    double dd2 = 0.0, dhd = 0.0;
    const double* tp = a.tilepart + (i64)i * a.ntile * NPT;
    for (int j = 0; j < a.ntile; ++j) {
      dd2 += tp[(i64)j * NPT + P_WW];
      dhd += tp[(i64)j * NPT + P_HW];
    }
    const double zd = a.dV * v[3];
    const double den = a.dV * (dhd - a.sigma[cur][i] * dd2);
    double t = (den > 0.0 && zd > 0.0) ? zd / den : a.tau0;
    if (!isfinite(t) || t <= 0.0) t = a.tau0;
    t = fmin(fmax(t, a.tau_min), a.tau_max);
    a.tfac[i] = t;  // the step itself for now; divided by the mean below
    a.dpart[3 * i] = v[0];
    a.dpart[3 * i + 1] = v[1];
    a.dpart[3 * i + 2] = v[2];
    a.coef[2 * i] = zd;  // kept for the decrease
    tloc += t;
  }
  const double ts = cta_sum(tloc, sh);
  if (threadIdx.x == 0) tsum = ts;
  __syncthreads();
  const double tau = tsum / a.N;
  double dec = 0.0;
  for (int i = threadIdx.x; i < a.N; i += CNT) {
    const double f = a.tfac[i] / tau;
    a.tfac[i] = f;
    dec += f * a.coef[2 * i];
  }
  const double dsum = cta_sum(dec, sh);
  if (threadIdx.x == 0) {
    st->tau_bb = tau;
    st->tau_trial = tau;
    st->znorm2 = dsum;
  }
}

}  // namespace

int cg_chunks(i64 ng) {
  // enough CTAs per orbital to fill the GPU a few times for N >= 4
  const i64 per = (ng + CNT - 1) / CNT;
  return (int)std::max<i64>(1, std::min<i64>(per, 2LL * num_sms()));
}

template <typename T>
void launch_cg_dots(const CgArgs<T>& a, cudaStream_t s) {
  prof_begin("cg_dots", s);
  k_cg_dots<T><<<dim3(a.nch, a.N), CNT, 0, s>>>(a);
  prof_end(s);
}
template <typename T>
void launch_cg_form(const CgArgs<T>& a, cudaStream_t s) {
  prof_begin("cg_form", s);
  k_cg_form<T><<<dim3(a.nch, a.N), CNT, 0, s>>>(a);
  prof_end(s);
}
template void launch_cg_dots<float>(const CgArgs<float>&, cudaStream_t);
template void launch_cg_dots<double>(const CgArgs<double>&, cudaStream_t);
template void launch_cg_form<float>(const CgArgs<float>&, cudaStream_t);
template void launch_cg_form<double>(const CgArgs<double>&, cudaStream_t);

void launch_cg_beta(const CgCtrlArgs& a, cudaStream_t s) {
  prof_begin("cg_beta", s);
  k_cg_beta<<<1, CNT, 0, s>>>(a);
  prof_end(s);
}
void launch_cg_step(const CgCtrlArgs& a, cudaStream_t s) {
  prof_begin("cg_step", s);
  k_cg_step<<<1, CNT, 0, s>>>(a);
  prof_end(s);
}

}  // namespace pou
