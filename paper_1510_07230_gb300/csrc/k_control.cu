// Controller of one pass of Algorithm E (Sec. 3.2), one CTA:
//   * reduces the H-apply sums of the trial block and the potential-pass
//     energy sums (fixed order, deterministic),
//   * E(W(tau)) = kinetic + external + Hartree + exchange (Eq. energy),
//   * nonmonotone test E(W(tau)) <= C^l - rho1 tau ||Z^l||_F^2 (Eq. ene-de);
//     on failure tau <- tau delta (the next pass rebuilds the trial from the
//     kept W^l, HW^l); after max_backtrack reductions the trial is accepted
//     and counted,
//   * on acceptance: Q^(l+1) = eta Q^l + 1, C^(l+1) = (eta Q^l C^l + E)/Q^(l+1),
//     the pair holding W^(l+1) becomes current, sigma_ii = <H w_i, w_i>,
//     ||Z||_F^2 and the Barzilai-Borwein step for the next step from
//     S = W^(l+1) - W^l and Y = Z^(l+1) - Z^l, using
//       tr<S^T S> = dV sum p_ss,
//       tr<S^T Y> = dV sum (p_sb - dsigma p_sw),
//       tr<Y^T Y> = dV sum (p_bb - 2 dsigma p_bw + dsigma^2 p_ww),
//     with dsigma_i = sigma_i - sigma'_i (Y = b - dsigma w).
#include "pou_internal.cuh"

namespace pou {

namespace {

constexpr int KNT = 256;
constexpr double kTauSpread = 10.0;  // per-orbital steps stay within this factor of the common one

__device__ double block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  double r = 0.0;
  for (int w = 0; w < KNT / 32; ++w) r += sh[w];
  return r;
}

__global__ void __launch_bounds__(KNT) k_control(CtrlArgs a) {
  __shared__ double sh[KNT / 32];
  __shared__ double esum[NE];
  State* st = a.st;
  if (st->done) return;
  if (a.refresh && !st->diag_now) return;
  const int cur = st->cur;
  // refresh: the rotated current pair's own sums; otherwise the trial's
  const int t = a.refresh ? cur : 1 - cur;
  const int N = a.N;
  const int tid = threadIdx.x;
  double* part = a.part[t];
  // per-orbital sums over tiles (fixed order), and the sigma' they refer to
  for (int idx = tid; idx < N * NP; idx += KNT) {
    const int i = idx / NP, k = idx % NP;
    if (k == P_SIGP) {
      // the sigma' the H-apply used (refresh: the eigenvalue), as it was rounded there
      const double sp = a.init ? 0.0 : a.sigma[cur][i];
      part[idx] = a.fp32 ? (double)(float)sp : sp;
      continue;
    }
    const double* src = a.tilepart + (i64)i * a.ntile * NPT + k;
    double s = 0.0;
    for (int j = 0; j < a.ntile; ++j) s += src[(i64)j * NPT];
    part[idx] = s;
  }
  if (tid < NE) {
    double s = 0.0;
    for (int b = 0; b < a.neblk; ++b) s += a.epart[(i64)b * NE + tid];
    esum[tid] = s;
  }
  __syncthreads();
  // nonlocal energy f sum_ip C_ip^2 of the trial (refresh: unchanged by a rotation)
  double enl = 0.0;
  if (a.nlC[t] && !a.refresh)
    for (int idx = tid; idx < N * a.P; idx += KNT) enl += a.nlC[t][idx] * a.nlC[t][idx];
  const double dV = a.dV;
  double kin = 0.0, ss = 0.0, sy = 0.0, yy = 0.0, zz = 0.0;
  __syncthreads();  // part[] complete (P_SIGP reads sigma[cur] before sigma[t] is written)
  for (int i = tid; i < N; i += KNT) {
    const double* p = part + i * NP;
    const double sig = dV * p[P_HW];
    const double sigp = p[P_SIGP];
    // ||z||^2 with z = hw - sigma w = z' - (sigma - sigma') w
    const double dz = sig - sigp;
    zz += p[P_ZZ] - 2.0 * dz * p[P_ZW] + dz * dz * p[P_WW];
    kin += a.kc[0] * p[P_KX] + a.kc[1] * p[P_KY] + a.kc[2] * p[P_KZ];
    if (!a.init && !a.refresh) {
      const double ds = sig - sigp;
      ss += p[P_SS];
      sy += p[P_SB] - ds * p[P_SW];
      yy += p[P_BB] - 2.0 * ds * p[P_BW] + ds * ds * p[P_WW];
    }
    a.sigma[t][i] = sig;
  }
  kin = block_sum(kin, sh);
  zz = block_sum(zz, sh);
  ss = block_sum(ss, sh);
  sy = block_sum(sy, sh);
  yy = block_sum(yy, sh);
  enl = block_sum(enl, sh);
  if (tid != 0) return;
  if (a.refresh) {
    // rho, V and E are unchanged by a rotation within the span
    st->znorm2 = zz * dV;
    st->diag_now = 0;
    st->diag_count += 1;
    return;
  }

  const double ekin = F_OCC * dV * kin;
  const double eext = dV * esum[E_EXT] + F_OCC * enl;
  const double eh = 0.5 * dV * esum[E_H];
  const double ex = dV * esum[E_X];
  const double E = ekin + eext + eh + ex;
  st->terms_trial[0] = ekin;
  st->terms_trial[1] = eext;
  st->terms_trial[2] = eh;
  st->terms_trial[3] = ex;
  zz *= dV;
  ss *= dV;
  sy = fabs(sy * dV);
  yy *= dV;
  if (!a.init && st->chol_fail) {
    // the trial's Gram matrix was not positive definite: rejected like a
    // trial failing Eq. (ene-de), the step shrinks (the Cholesky kernel turns
    // it into a breakdown once max_backtrack reductions are spent)
    st->chol_fail = 0;
    st->passes += 1;
    st->s += 1;
    st->backtracks += 1;
    st->tau_trial = st->tau_bb * pow(a.delta, (double)st->s);
    return;
  }
  if (!isfinite(E)) {
    st->status = 5;  // POU_ENAN
    st->done = 1;
    return;
  }
  if (a.init) {
    st->cur = t;
    st->E_cur = E;
    for (int k = 0; k < 4; ++k) st->terms_cur[k] = st->terms_trial[k];
    st->C = E;
    st->Q = 1.0;
    st->znorm2 = zz;
    st->tau_bb = a.tau0;
    st->tau_trial = a.tau0;
    st->last_tau = 0.0;
    st->s = 0;
    st->l = 0;
    st->passes = st->backtracks = st->forced = st->n_df = 0;
    st->df[0] = st->df[1] = st->df[2] = 0.0;
    st->gram_off_acc = 0.0;
    st->converged = 0;
    st->reorth_count = 0;
    st->diag_now = 0;
    st->diag_count = 0;
    st->orth_now = 1;
    st->done = 1;
    if (a.tfac)
      for (int i = 0; i < N; ++i) a.tfac[i] = 1.0;  // first step: tau_0 for every orbital
    return;
  }
  st->passes += 1;
  // Algorithm M, intermediate step (n_org > 1): the trial W - tau Z is taken
  // as it is, without Orth, the Eq. (ene-de) test or backtracking; C, Q and
  // the reference energy stay those of the last orthonormalised step
  const bool orth = st->orth_now != 0;
  bool accept = !orth || E <= st->C - a.rho1 * st->tau_trial * st->znorm2;
  if (!accept && st->s >= a.max_backtrack) {
    accept = true;
    st->forced += 1;
  }
  if (!accept) {
    st->s += 1;
    st->backtracks += 1;
    st->tau_trial = st->tau_bb * pow(a.delta, (double)st->s);
    return;
  }
  if (orth) {
    const double Qn = a.eta * st->Q + 1.0;
    st->C = (a.eta * st->Q * st->C + E) / Qn;
    st->Q = Qn;
    const double df = fabs(st->E_cur - E) / (fabs(st->E_cur) + 1.0);
    st->df[2] = st->df[1];
    st->df[1] = st->df[0];
    st->df[0] = df;
    st->n_df += 1;
    st->last_tau = st->tau_trial;
    st->E_cur = E;
    for (int k = 0; k < 4; ++k) st->terms_cur[k] = st->terms_trial[k];
    st->gram_off_acc = st->gram_off_trial;
  }
  if (st->l < HIST_MAX) {
    a.hist_E[st->l] = orth ? E : NAN;  // no energy of a non-orthonormal iterate
    a.hist_tau[st->l] = st->tau_trial;
  }
  st->cur = t;
  st->l += 1;
  st->znorm2 = zz;
  // Barzilai-Borwein step shared by all orbitals
  int variant = a.bb_variant;
  if (variant == 3) variant = (st->l % 2 == 0) ? 1 : 2;
  double tau = (variant == 1) ? (sy > 0.0 ? ss / sy : NAN) : (yy > 0.0 ? sy / yy : NAN);
  if (!isfinite(tau) || tau <= 0.0) tau = a.tau0;
  tau = fmin(fmax(tau, a.tau_min), a.tau_max);
  st->tau_bb = tau;
  st->tau_trial = tau;
  st->s = 0;
  if (a.tfac) {
    // per-orbital steps (the tau_i of Sec. 3.2): the same quotient from the
    // orbital's own s_i, y_i, kept as a factor on the common tau; the
    // Eq. (ene-de) decrease becomes sum_i tau_i ||z_i||^2 = tau * znorm2
    double zf = 0.0;
    for (int i = 0; i < N; ++i) {
      const double* p = part + i * NP;
      const double ds = a.sigma[t][i] - p[P_SIGP];
      const double ssi = p[P_SS];
      const double syi = fabs(p[P_SB] - ds * p[P_SW]);
      const double yyi = p[P_BB] - 2.0 * ds * p[P_BW] + ds * ds * p[P_WW];
      double ti = (variant == 1) ? (syi > 0.0 ? ssi / syi : NAN) : (yyi > 0.0 ? syi / yyi : NAN);
      if (!isfinite(ti) || ti <= 0.0) ti = a.tau0;
      ti = fmin(fmax(ti, a.tau_min), a.tau_max);
      // within a factor kTauSpread of the common step: an orbital whose own
      // <s_i, y_i> is near zero cannot take over the trial
      const double fi = fmin(fmax(ti / tau, 1.0 / kTauSpread), kTauSpread);
      a.tfac[i] = fi;
      zf += fi * (p[P_ZZ] - 2.0 * ds * p[P_ZW] + ds * ds * p[P_WW]);
    }
    st->znorm2 = zf * dV;
  }
  // Algorithm M: subspace diagonalisation every n_diag steps (after an
  // orthonormalised step), before the next trial; Orth every n_org steps
  st->diag_now = (orth && a.n_diag > 0 && st->l % a.n_diag == 0) ? 1 : 0;
  st->orth_now = (a.n_org <= 1 || st->l % a.n_org == 0) ? 1 : 0;
  if (st->l >= st->target_l) st->done = 1;
  if (orth && st->e_tol > 0.0 && st->n_df >= 3 && (st->df[0] + st->df[1] + st->df[2]) / 3.0 < st->e_tol) {
    st->converged = 1;
    st->done = 1;
  }
}

}  // namespace

void launch_control(const CtrlArgs& a, cudaStream_t s) {
  prof_begin("control", s);
  k_control<<<1, KNT, 0, s>>>(a);
  prof_end(s);
}

}  // namespace pou
