// Rotation W_new = Wt R^-1 of the FP32 form (Orth by Cholesky-QR, Sec. 3.2)
// on the 5th-generation tensor cores, fused with the density
// rho = f sum_j w_new_j^2 (Sec. 2), for N <= 128 orbitals (k_rotate_tc; up to
// 512 with k_rotate_tc_big further below) and upper triangular R^-1 (the
// dense subspace rotation of Algorithm M runs on the CUDA cores).
//
// Split of the work.  Output j at point p is
//   w_new_j(p) = sum_{i < j} x_i(p) R_ij  +  R_jj x_j(p),
// x = Wt (trial: (1 + tau sigma_i) w_i - tau hw_i from the FP64 coefficients,
// formed as a double-float exactly as the trial Gram matrix forms it) or the
// block itself.  The
// off-diagonal sum runs on the tensor cores as D = X R_off with M = 128 grid
// points (tensor-memory lanes), N = outputs j (columns) and K = orbitals i,
// both operands split into TF32 pairs: D = Xhi Rhi + Xhi Rlo + Xlo Rhi, which
// carries the sum to about 2^-21 of its own size.  R_off is upper
// triangular, so K atom k (orbitals 32k .. 32k+31) only feeds outputs
// j >= 32k: its MMAs run with N = 128 - 32k and only those rows of R are
// stored.  The tensor core adds into its FP32 accumulator with truncation (a
// bias toward zero of a fraction of an ulp per accumulation), so the
// dominant Xhi Rhi part is kept in two accumulators (atoms 0-1 and 2-3,
// eight accumulations each), the small cross terms in a third, and the three
// are added on the CUDA cores with round-to-nearest.  The self term R_jj x_j
// is formed on the CUDA cores with a double-float R_jj and stored with
// unbiased (dithered) rounding, because near convergence the corrections
// that keep each orbital normalised are below half an ulp of its elements.
//
// The whole 128-point X tile stays in shared memory (four atom slots) until
// the epilogue has used it: Xhi = tf32(x) and Xlo = x - Xhi (exact in FP32
// for a plain block, rounded once from the double-float trial point; the
// tensor core reads its leading TF32 bits), so that x = Xhi + Xlo (35 bits)
// is available to the self term without reading w and hw again.
//
// With points on the lanes, every global access of the epilogue (the output,
// the density) is one 128-byte segment of one row per warp instruction, and
// the density of a point is a per-thread sum.
//
// Pipeline per tile of 128 points (one CTA per SM, 512 threads: 16 warps,
// four per SM sub-partition, so that each thread may hold 128 registers):
//   warps 0-7   (producers) load one 32-orbital K atom of the tile at a time
//               (eight lanes per 128-byte row segment), two atoms ahead, form
//               Wt, split it and write it K-major (128-byte swizzle) into the
//               atom's slot once the previous tile's MMAs and epilogue are
//               done with it; warp 0 also allocates tensor memory, and its
//               lane 0 issues the MMAs of an atom once all producers wrote it;
//   warps 8-15  (epilogue; two warps per TMEM lane quadrant, 64 output
//               columns each) add the three accumulators into the 128 free
//               tensor-memory columns and release them at once, so the next
//               tile's MMAs overlap the rest: the self term from the resident
//               X tile, the stores and the squares for the density; each
//               warp frees an atom slot as soon as it has read its columns.
// Tile rows are permuted within each 32-point group (row 8e + q holds point
// 4q + e) so that the producers' transposing shared-memory stores hit 32
// distinct banks; the epilogue lane of a row is then row mod 32.
#include "pou_internal.cuh"
#include "tc_ptx.cuh"

#include <algorithm>

namespace pou {

namespace {

constexpr int TPTS = 128;                  // points per tile (= M)
constexpr int PROD_WARPS = 8, EPI_WARPS = 8;
constexpr int EPI0 = PROD_WARPS;           // first epilogue warp
constexpr int NTHR = (EPI0 + EPI_WARPS) * 32;
constexpr int ATOM = 128 * 128;            // bytes of one K atom: 128 rows x 128 bytes
constexpr int SLOT = 2 * ATOM;             // one X atom: hi rows, then lo rows
// R_off as the B operand, rows j >= 32 k of atom k (K = i): 128, 96, 64, 32 rows
__host__ __device__ constexpr int r_rows(int k) { return 128 - 32 * k; }
__host__ __device__ constexpr int r_row0(int k) { return 128 * k - 16 * k * (k - 1); }
constexpr int R_BYTES = 128 * (128 + 96 + 64 + 32);
constexpr int OFF_RHI = 0;
constexpr int OFF_RLO = OFF_RHI + R_BYTES;
constexpr int OFF_X = OFF_RLO + R_BYTES;           // four X atom slots (one tile)
constexpr int OFF_SELF = OFF_X + 4 * SLOT;         // 128 x float2: R_jj as (hi, lo)
constexpr int OFF_COEF = OFF_SELF + 128 * 8;       // 128 x float4: 1 + t_i sigma_i, t_i as (hi, lo)
constexpr int OFF_DENS = OFF_COEF + 128 * 16;      // [4 quadrants][32] x (s, c)
static_assert(OFF_COEF % 16 == 0, "coefficient entries must be 16-byte aligned");
constexpr int OFF_BAR = OFF_DENS + 4 * 32 * 8;
// barriers: full[4], empty[4], accf, acce, fin; then tmem slot, abort flag
constexpr int NBAR = 11;
constexpr int OFF_MISC = OFF_BAR + NBAR * 8;
constexpr int SMEM_BYTES = OFF_MISC + 16 + 1024;  // + alignment slack
constexpr uint32_t TMEM_COLS = 512;
constexpr uint32_t COL_HH1 = 128, COL_X = 256;   // accumulators: hh0 at 0, hh1, cross terms
constexpr uint32_t COL_OFF = 384;                // epilogue copy of the summed accumulators
// the empty barrier of a slot: the MMA commit and the four epilogue warps reading its columns
constexpr int EMPTY_ARRIVALS = 1 + 4;

static_assert(OFF_RLO % 1024 == 0 && OFF_X % 1024 == 0, "swizzled tiles need 1024-byte alignment");
static_assert(SMEM_BYTES <= 232448, "tensor-core rotation exceeds the shared-memory opt-in limit");

__device__ unsigned int g_rotate_tc_aborts = 0;

__device__ __forceinline__ void f2_add(float& s, float& c, float b, float extra) {
  const float t = s + b;
  const float bp = t - s;
  c += ((s - (t - bp)) + (b - bp)) + extra;
  s = t;
}

// lowbias32 integer mixer (C. Wellons, hash-prospector): counter-based
// uniform bits for the dithered rounding of the self term.
__device__ __forceinline__ unsigned mix32(unsigned x) {
  x ^= x >> 16;
  x *= 0x7feb352dU;
  x ^= x >> 15;
  x *= 0x846ca68bU;
  x ^= x >> 16;
  return x;
}
__device__ __forceinline__ void named_bar(int id, int nthreads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// uniform offset in (-ulp/2, ulp/2) of x from one byte
__device__ __forceinline__ float dither(float x, unsigned byte) {
  const float ulp = __uint_as_float(__float_as_uint(x) & 0x7f800000u) * 1.1920928955078125e-7f;
  return ((float)byte * (1.0f / 256.0f) - 0.498046875f) * ulp;
}

__global__ void __launch_bounds__(NTHR, 1) k_rotate_tc(RotArgs<float> a, i64 ntiles) {
  extern __shared__ unsigned char smem_raw[];
  if (a.st && a.st->done) return;
  if (!gate_open(a.st, a.gate)) return;

  const uint32_t raw_addr = tc::smem_u32(smem_raw);
  const uint32_t pad = (1024u - (raw_addr & 1023u)) & 1023u;
  unsigned char* smem = smem_raw + pad;
  const uint32_t sbase = raw_addr + pad;
  float2* self = reinterpret_cast<float2*>(smem + OFF_SELF);  // R_jj as (hi, lo)
  float2* dens = reinterpret_cast<float2*>(smem + OFF_DENS);
  float4* coefs = reinterpret_cast<float4*>(smem + OFF_COEF);
  const uint32_t bar0 = sbase + OFF_BAR;
  auto full_bar = [&](int k) { return bar0 + 8u * k; };
  auto empty_bar = [&](int k) { return bar0 + 8u * (4 + k); };
  const uint32_t accf_bar = bar0 + 64u, acce_bar = bar0 + 72u, fin_bar = bar0 + 80u;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + OFF_MISC);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + OFF_MISC + 4);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int N = a.N;
  const i64 ng = a.ng;

  // sources and destinations of the mode (see RotArgs)
  int cur = 0;
  const float* Wsrc;
  const float* Hsrc = nullptr;
  float* out;
  double* rho;
  double tau = 0.0;
  if (a.trial) {
    cur = a.st->cur;
    Wsrc = a.W[cur];
    Hsrc = a.HW[cur];
    out = a.Wout[1 - cur];
    rho = a.rho[1 - cur];
    tau = a.st->tau_trial;
  } else if (a.st) {
    cur = a.st->cur;
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

  // B operand = strictly upper R (row j, K index i) split into TF32 pairs,
  // rows j >= 32 k of atom k only; the self-term coefficients R_jj; the
  // trial coefficients 1 + tau sigma_i
  for (int idx = tid; idx < 320 * 32; idx += NTHR) {
    const int row = idx >> 5, il = idx & 31;  // stored row, K index within the atom
    const int k = row < 128 ? 0 : (row < 224 ? 1 : (row < 288 ? 2 : 3));
    const int r = row - r_row0(k);           // j - 32 k
    const int i = 32 * k + il, j = 32 * k + r;
    double v = 0.0;
    if (i < j && j < N) v = a.Rinv[(i64)i * N + j];
    const float hi = tc::to_tf32((float)v);
    const float lo = tc::to_tf32((float)(v - (double)hi));
    const int off = row * 128 + (((il >> 2) ^ (r & 7)) << 4) + (il & 3) * 4;
    *reinterpret_cast<float*>(smem + OFF_RHI + off) = hi;
    *reinterpret_cast<float*>(smem + OFF_RLO + off) = lo;
  }
  for (int j = tid; j < 128; j += NTHR) {
    double A = 0.0, cf = 1.0, t = tau;
    if (j < N) {
      A = a.Rinv[(i64)j * N + j];
      if (a.trial && a.tfac) t = tau * a.tfac[j];
      if (a.trial) cf = 1.0 + t * a.sigma[cur][j];
    }
    const float ah = (float)A, ch = (float)cf, th = (float)t;
    self[j] = make_float2(ah, (float)(A - (double)ah));
    coefs[j] = make_float4(ch, (float)(cf - (double)ch), th, (float)(t - (double)th));
  }
  if (tid == 0) {
    for (int k = 0; k < 4; ++k) {
      tc::mbar_init(full_bar(k), PROD_WARPS * 32);
      tc::mbar_init(empty_bar(k), EMPTY_ARRIVALS);
    }
    tc::mbar_init(accf_bar, 1);
    tc::mbar_init(acce_bar, EPI_WARPS * 32);
    tc::mbar_init(fin_bar, 1);
    *abort_flag = 0;
    tc::mbar_init_fence();
  }
  if (warp == 0) {
    tc::tmem_alloc(tc::smem_u32(tmem_slot), TMEM_COLS);
    tc::tmem_relinquish();
  }
  tc::fence_proxy_async_smem();  // R tiles written by the generic proxy
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tmem_slot;

  const i64 G = gridDim.x;
  const i64 t0 = ntiles * (i64)blockIdx.x / G, t1 = ntiles * (i64)(blockIdx.x + 1) / G;
  const int nmine = (int)(t1 - t0);
  const int natoms = 4 * nmine;
  const bool vec4 = (ng % 4 == 0) && ((reinterpret_cast<uintptr_t>(Wsrc) & 15u) == 0) &&
                    (Hsrc == nullptr || (reinterpret_cast<uintptr_t>(Hsrc) & 15u) == 0);

  if (warp < PROD_WARPS) {
    // ------------------------------------------------------------ producers
    // Atom u = 4 t + k of this CTA (tile t, orbitals 32 k .. 32 k + 31) goes
    // to slot u & 1.  Thread (warp w, lane l) owns orbital 32 k + 4 w + l / 8
    // and the four points 4 q .. 4 q + 3 (q = l % 8) of each 32-point group g.
    const int q = lane & 7, isub = lane >> 3;
    auto issue = [&](int u, float4 (&wv)[4], float4 (&hv)[4]) {
      const int k = u & 3;
      const i64 p0 = (t0 + (u >> 2)) * TPTS + 4 * q;
      const int i = 32 * k + 4 * warp + isub;
#pragma unroll
      for (int g = 0; g < 4; ++g) {
        wv[g] = make_float4(0.f, 0.f, 0.f, 0.f);
        hv[g] = wv[g];
      }
      if (i >= N) return;
      const i64 base = (i64)i * ng + p0;
#pragma unroll
      for (int g = 0; g < 4; ++g) {
        const i64 p = p0 + 32 * g;
        if (vec4) {
          if (p < ng) {  // ng % 4 == 0: a chunk is wholly inside the row or past it
            wv[g] = __ldg(reinterpret_cast<const float4*>(Wsrc + base + 32 * g));
            if (Hsrc) hv[g] = __ldg(reinterpret_cast<const float4*>(Hsrc + base + 32 * g));
          }
        } else {
          float w1[4] = {0.f, 0.f, 0.f, 0.f}, h1[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
          for (int e = 0; e < 4; ++e)
            if (p + e < ng) {
              w1[e] = Wsrc[base + 32 * g + e];
              if (Hsrc) h1[e] = Hsrc[base + 32 * g + e];
            }
          wv[g] = make_float4(w1[0], w1[1], w1[2], w1[3]);
          hv[g] = make_float4(h1[0], h1[1], h1[2], h1[3]);
        }
      }
    };
    bool issued = false;
    // one atom: loads for atom u + 2 go into the register set that held
    // atom u - 1; atom u is written from (w, h) into slot u % 4
    auto step = [&](int u, const float4 (&w)[4], const float4 (&h)[4], float4 (&wl)[4], float4 (&hl)[4]) -> bool {
      if (u + 2 < natoms) issue(u + 2, wl, hl);
      const int k = u & 3, t = u >> 2;
      // the previous tile's MMAs and epilogue are done with the slot
      if (t > 0 && !tc::mbar_wait(empty_bar(k), (t - 1) & 1, abort_flag)) return false;
      unsigned char* xs = smem + OFF_X + k * SLOT;
      const float4 cf = coefs[32 * k + 4 * warp + isub];
#pragma unroll
      for (int g = 0; g < 4; ++g) {
        const float x[4] = {w[g].x, w[g].y, w[g].z, w[g].w};
        const float h4[4] = {h[g].x, h[g].y, h[g].z, h[g].w};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int row = 32 * g + 8 * e + q;  // holds point 32 g + 4 q + e; row % 8 == q
          float hi, lo;
          if (Hsrc) {
            tc::trial_split(cf.x, cf.y, x[e], cf.z, cf.w, h4[e], hi, lo);
          } else {
            hi = tc::to_tf32(x[e]);
            lo = x[e] - hi;  // exact
          }
          const int off = row * 128 + ((warp ^ q) << 4) + isub * 4;
          *reinterpret_cast<float*>(xs + off) = hi;
          *reinterpret_cast<float*>(xs + ATOM + off) = lo;
        }
      }
      tc::fence_proxy_async_smem();
      tc::mbar_arrive(full_bar(k));
      if (warp == 0) {
        // ---------------------------------------------------- MMA issue
        int ok = 1;
        if (lane == 0) {
          if (k == 0 && t > 0) ok = tc::mbar_wait(acce_bar, (t - 1) & 1, abort_flag);
          if (ok) ok = tc::mbar_wait(full_bar(k), t & 1, abort_flag);
          if (ok) {
            tc::fence_after_sync();
            const uint32_t xh = sbase + OFF_X + k * SLOT, xl = xh + ATOM;
            const uint32_t rh = sbase + OFF_RHI + r_row0(k) * 128, rl = sbase + OFF_RLO + r_row0(k) * 128;
            // outputs j >= 32 k only: columns 32 k .. 127, N = 128 - 32 k
            const uint32_t c0 = 32u * k;
            const uint32_t dhh = tmem + ((k >> 1) ? COL_HH1 : 0u) + c0, dx = tmem + COL_X + c0;
            const uint32_t idesc = tc::idesc_tf32(128, r_rows(k));
#pragma unroll
            for (int s4 = 0; s4 < 4; ++s4) {
              const uint64_t axh = tc::desc_sw128(xh + 32u * s4), axl = tc::desc_sw128(xl + 32u * s4);
              const uint64_t brh = tc::desc_sw128(rh + 32u * s4), brl = tc::desc_sw128(rl + 32u * s4);
              tc::mma_tf32(dhh, axh, brh, idesc, ((k & 1) == 0 && s4 == 0) ? 0u : 1u);
              tc::mma_tf32(dx, axh, brl, idesc, (k == 0 && s4 == 0) ? 0u : 1u);
              tc::mma_tf32(dx, axl, brh, idesc, 1u);
            }
            issued = true;
            tc::mma_commit(empty_bar(k));
            if (k == 3) tc::mma_commit(accf_bar);
          }
        }
        if (!__shfl_sync(0xffffffffu, ok, 0)) return false;
      }
      return true;
    };
    float4 wA[4], hA[4], wB[4], hB[4], wC[4], hC[4];
    if (natoms > 0) issue(0, wA, hA);
    if (natoms > 1) issue(1, wB, hB);
    for (int u = 0; u < natoms; u += 3) {
      if (!step(u, wA, hA, wC, hC)) break;
      if (u + 1 >= natoms || !step(u + 1, wB, hB, wA, hA)) break;
      if (u + 2 >= natoms || !step(u + 2, wC, hC, wB, hB)) break;
    }
    if (warp == 0 && lane == 0 && issued) {
      // every MMA issued has completed before tensor memory is released
      tc::mma_commit(fin_bar);
      tc::mbar_wait(fin_bar, 0, abort_flag, 4000000000ull);
    }
    __syncwarp();
  } else {
    // ------------------------------------------------------------ epilogue
    const int quad = warp & 3;              // TMEM lane quadrant: tile points 32 quad .. 32 quad + 31
    const int jh = (warp - EPI0) >> 2;      // output columns 64 jh .. 64 jh + 63
    const int pt = 32 * quad + 4 * (lane & 7) + (lane >> 3);  // tile point of this thread's lane
    const uint32_t lane_base = tmem + ((uint32_t)(quad * 32) << 16);
    const uint32_t off_col = COL_OFF + (uint32_t)(64 * jh);  // this warp's copy of its 64 sums
    const unsigned seed32 = mix32((unsigned)(a.st ? a.st->passes : 0) * 4u + (unsigned)a.sr_salt + 0x85ebca6bu);
    // this lane's tile row in the X slots (row 32 quad + lane holds point pt)
    const int row = 32 * quad + lane;
    // density of this lane's point over the 64 columns: four independent
    // double-float chains (one per column mod 4), so that the compensated
    // additions do not form one serial dependency
    float rs[4], rc[4];
    // one 8-column group: self term, dithered rounding, store, squares
    auto finish = [&](i64 p, int g) {
      uint32_t ov[8];
      tc::tmem_ld8(lane_base + off_col + (uint32_t)(8 * g), ov);
      const int j0 = 64 * jh + 8 * g;
      const unsigned char* xs = smem + OFF_X + (j0 >> 5) * SLOT;
      float xh[8], xl[8];  // x = xh + xl
#pragma unroll
      for (int h4 = 0; h4 < 2; ++h4) {
        const int chunk = ((j0 & 31) >> 2) + h4;
        const int off = row * 128 + ((chunk ^ (row & 7)) << 4);
        const float4 vh = *reinterpret_cast<const float4*>(xs + off);
        const float4 vl = *reinterpret_cast<const float4*>(xs + ATOM + off);
        xh[4 * h4 + 0] = vh.x, xh[4 * h4 + 1] = vh.y, xh[4 * h4 + 2] = vh.z, xh[4 * h4 + 3] = vh.w;
        xl[4 * h4 + 0] = vl.x, xl[4 * h4 + 1] = vl.y, xl[4 * h4 + 2] = vl.z, xl[4 * h4 + 3] = vl.w;
      }
      tc::tmem_wait_ld();
#pragma unroll
      for (int m4 = 0; m4 < 8; m4 += 4) {
        // one 32-bit draw per (4 columns, point): one byte per element
        const unsigned bits = mix32(seed32 ^ mix32((unsigned)((j0 + m4) >> 2) * 0x9e3779b1u ^ (unsigned)p));
#pragma unroll
        for (int m = m4; m < m4 + 4; ++m) {
          const int j = j0 + m;
          const float2 c = self[j];  // R_jj (hi, lo)
          const float d = dither(xh[m], (bits >> (8 * (m - m4))) & 0xffu);
          // R_jj x = (c.x + c.y)(xh + xl), one rounding at the output's scale
          const float o = fmaf(c.x, xh[m], fmaf(c.x, xl[m], fmaf(c.y, xh[m], __uint_as_float(ov[m]) + d)));
          if (p < ng && j < N) {
            out[(i64)j * ng + p] = o;
            const float sq = o * o;
            f2_add(rs[m - m4], rc[m - m4], sq, fmaf(o, o, -sq));
          }
        }
      }
    };
    for (int t = 0; t < nmine; ++t) {
      const i64 p = (t0 + t) * TPTS + pt;
      if (!tc::mbar_wait(accf_bar, t & 1, abort_flag)) break;
      tc::fence_after_sync();
      // off-diagonal sums: the accumulators added and copied to this warp's
      // free tensor-memory columns, then released (outputs j < 64 receive
      // nothing from atoms 2-3: the hh1 columns 0..63 are never written)
#pragma unroll 1
      for (int c = 0; c < 64; c += 16) {
        uint32_t h0[16], h1[16], xx[16];
        tc::tmem_ld16(lane_base + (uint32_t)(64 * jh + c), h0);
        if (jh) tc::tmem_ld16(lane_base + COL_HH1 + (uint32_t)(64 * jh + c), h1);
        tc::tmem_ld16(lane_base + COL_X + (uint32_t)(64 * jh + c), xx);
        tc::tmem_wait_ld();
        if (jh) {
#pragma unroll
          for (int m = 0; m < 16; ++m)
            h0[m] = __float_as_uint((__uint_as_float(h0[m]) + __uint_as_float(h1[m])) + __uint_as_float(xx[m]));
        } else {
#pragma unroll
          for (int m = 0; m < 16; ++m) h0[m] = __float_as_uint(__uint_as_float(h0[m]) + __uint_as_float(xx[m]));
        }
        tc::tmem_st16(lane_base + off_col + (uint32_t)c, h0);
      }
      tc::tmem_wait_st();
      tc::fence_before_sync();
      tc::mbar_arrive(acce_bar);  // accumulators free: the next tile's MMAs may start

#pragma unroll
      for (int c = 0; c < 4; ++c) rs[c] = rc[c] = 0.f;
#pragma unroll 1
      for (int g = 0; g < 8; ++g) {
        finish(p, g);
        if ((g & 3) == 3) {
          // this warp has read its columns of atom 2 jh + g / 4
          __syncwarp();
          if (lane == 0) tc::mbar_arrive(empty_bar(2 * jh + (g >> 2)));
        }
      }
      f2_add(rs[0], rc[0], rs[1], rc[1]);
      f2_add(rs[2], rc[2], rs[3], rc[3]);
      f2_add(rs[0], rc[0], rs[2], rc[2]);
      if (rho != nullptr) {
        // the two warps of this quadrant hold the two column halves
        float2* dq = dens + quad * 32;
        if (jh == 1) dq[lane] = make_float2(rs[0], rc[0]);
        named_bar(1 + quad, 64);
        if (jh == 0 && p < ng) {
          const float2 o2 = dq[lane];
          rho[p] = F_OCC * (((double)rs[0] + (double)rc[0]) + ((double)o2.x + (double)o2.y));
        }
        named_bar(1 + quad, 64);
      }
    }
  }

  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, TMEM_COLS);
  }
  if (*abort_flag != 0 && tid == 0) {
    atomicAdd(&g_rotate_tc_aborts, 1u);
    if (a.st) {
      State* w = const_cast<State*>(a.st);
      w->status = 3;  // POU_ECUDA: a pipeline wait gave up
      w->done = 1;
    }
  }
}


// ===========================================================================
// N > 128 (up to 512 orbitals).  Output columns j are taken in chunks of 128
// (passes jc = 0 .. nb - 1 over each tile); pass jc accumulates the K atoms
// k = 0 .. 4 jc + 3 (orbitals i < 128 (jc + 1), the others have R_ij = 0).
// R^-1 is too large for shared memory: it is split into TF32 pairs and laid
// out in the swizzled operand format once per launch (k_rimg, one 32 KB
// image per (jc, k)), and each atom's image is streamed into one of two R
// slots with cp.async by the producers, one atom ahead.  X atoms cycle
// through the four X slots; the last four atoms of a pass are the chunk's
// own orbitals, whose X values the epilogue needs for the self term, so a
// slot's first use in a pass also waits for the previous pass's epilogue to
// release it.  The density of a point is summed over the passes of its tile.
// Accumulators as above, with hh0 taking the first half of a pass's atoms.
constexpr int BIG_MAXN = 512;
constexpr int B_OFF_R = 0;                             // two R atom slots (hi rows, then lo rows)
constexpr int B_OFF_X = 2 * SLOT;                      // four X atom slots
constexpr int B_OFF_SELF = B_OFF_X + 4 * SLOT;         // BIG_MAXN x float2: R_jj (hi, lo)
constexpr int B_OFF_COEF = B_OFF_SELF + BIG_MAXN * 8;  // BIG_MAXN x float4: 1 + t_i sigma_i, t_i
constexpr int B_OFF_DENS = B_OFF_COEF + BIG_MAXN * 16;
static_assert(B_OFF_COEF % 16 == 0, "coefficient entries must be 16-byte aligned");
constexpr int B_OFF_BAR = B_OFF_DENS + 4 * 32 * 8;
// barriers: fullx[4], emptyx[4], xfree[4], fullr[2], emptyr[2], accf, acce, fin
constexpr int B_NBAR = 19;
constexpr int B_OFF_MISC = B_OFF_BAR + B_NBAR * 8;
constexpr int B_SMEM = B_OFF_MISC + 16 + 1024;
constexpr uint32_t IDESC128 = tc::idesc_tf32(128, 128);
static_assert(B_SMEM <= 232448, "tensor-core rotation (N > 128) exceeds the shared-memory opt-in limit");

__host__ __device__ constexpr int big_atoms(int jc) { return 4 * jc + 4; }
__host__ __device__ constexpr int big_atom0(int jc) { return 2 * jc * (jc + 1); }  // image index of (jc, 0)

// split R^-1 (strictly upper part) into the per-(jc, k) operand images
__global__ void __launch_bounds__(256) k_rimg(RotArgs<float> a) {
  if (a.st && a.st->done) return;
  if (!gate_open(a.st, a.gate)) return;
  const int N = a.N, nb = (N + 127) / 128;
  int jc = 0;
  while (jc + 1 < nb && big_atom0(jc + 1) <= (int)blockIdx.x) ++jc;
  const int k = (int)blockIdx.x - big_atom0(jc);
  unsigned char* base = reinterpret_cast<unsigned char*>(a.rimg) + (size_t)blockIdx.x * SLOT;
  for (int idx = threadIdx.x; idx < 128 * 32; idx += 256) {
    const int r = idx >> 5, il = idx & 31;
    const int i = 32 * k + il, j = 128 * jc + r;
    double v = 0.0;
    if (i < j && j < N) v = a.Rinv[(i64)i * N + j];
    const float hi = tc::to_tf32((float)v);
    const float lo = tc::to_tf32((float)(v - (double)hi));
    const int off = r * 128 + (((il >> 2) ^ (r & 7)) << 4) + (il & 3) * 4;
    *reinterpret_cast<float*>(base + off) = hi;
    *reinterpret_cast<float*>(base + ATOM + off) = lo;
  }
}

__global__ void __launch_bounds__(NTHR, 1) k_rotate_tc_big(RotArgs<float> a, i64 ntiles) {
  extern __shared__ unsigned char smem_raw[];
  if (a.st && a.st->done) return;
  if (!gate_open(a.st, a.gate)) return;

  const uint32_t raw_addr = tc::smem_u32(smem_raw);
  const uint32_t pad = (1024u - (raw_addr & 1023u)) & 1023u;
  unsigned char* smem = smem_raw + pad;
  const uint32_t sbase = raw_addr + pad;
  float2* self = reinterpret_cast<float2*>(smem + B_OFF_SELF);
  float4* coefs = reinterpret_cast<float4*>(smem + B_OFF_COEF);
  float2* dens = reinterpret_cast<float2*>(smem + B_OFF_DENS);
  const uint32_t bar0 = sbase + B_OFF_BAR;
  auto fullx = [&](int k) { return bar0 + 8u * k; };
  auto emptyx = [&](int k) { return bar0 + 8u * (4 + k); };
  auto xfree = [&](int k) { return bar0 + 8u * (8 + k); };
  auto fullr = [&](int k) { return bar0 + 8u * (12 + k); };
  auto emptyr = [&](int k) { return bar0 + 8u * (14 + k); };
  const uint32_t accf_bar = bar0 + 8u * 16, acce_bar = bar0 + 8u * 17, fin_bar = bar0 + 8u * 18;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + B_OFF_MISC);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + B_OFF_MISC + 4);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int N = a.N;
  const i64 ng = a.ng;
  const int nb = (N + 127) / 128, per_tile = big_atom0(nb);

  int cur = 0;
  const float* Wsrc;
  const float* Hsrc = nullptr;
  float* out;
  double* rho;
  double tau = 0.0;
  if (a.trial) {
    cur = a.st->cur;
    Wsrc = a.W[cur];
    Hsrc = a.HW[cur];
    out = a.Wout[1 - cur];
    rho = a.rho[1 - cur];
    tau = a.st->tau_trial;
  } else if (a.st) {
    cur = a.st->cur;
    Wsrc = a.src_trial_slot ? a.Wout[1 - cur] : a.A;
    out = a.Wout[1 - cur];
    rho = a.rho[1 - cur];
  } else {
    Wsrc = a.A;
    out = a.B;
    rho = a.rho_out;
  }
  const unsigned char* img = reinterpret_cast<const unsigned char*>(a.rimg);

  for (int j = tid; j < BIG_MAXN; j += NTHR) {
    double A = 0.0, cf = 1.0, t = tau;
    if (j < N) {
      A = a.Rinv[(i64)j * N + j];
      if (a.trial && a.tfac) t = tau * a.tfac[j];
      if (a.trial) cf = 1.0 + t * a.sigma[cur][j];
    }
    const float ah = (float)A, ch = (float)cf, th = (float)t;
    self[j] = make_float2(ah, (float)(A - (double)ah));
    coefs[j] = make_float4(ch, (float)(cf - (double)ch), th, (float)(t - (double)th));
  }
  if (tid == 0) {
    for (int k = 0; k < 4; ++k) {
      tc::mbar_init(fullx(k), PROD_WARPS * 32);
      tc::mbar_init(emptyx(k), 1);
      tc::mbar_init(xfree(k), 4);
    }
    for (int k = 0; k < 2; ++k) {
      tc::mbar_init(fullr(k), PROD_WARPS * 32);
      tc::mbar_init(emptyr(k), 1);
    }
    tc::mbar_init(accf_bar, 1);
    tc::mbar_init(acce_bar, EPI_WARPS * 32);
    tc::mbar_init(fin_bar, 1);
    *abort_flag = 0;
    tc::mbar_init_fence();
  }
  if (warp == 0) {
    tc::tmem_alloc(tc::smem_u32(tmem_slot), TMEM_COLS);
    tc::tmem_relinquish();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tmem_slot;

  const i64 G = gridDim.x;
  const i64 t0 = ntiles * (i64)blockIdx.x / G, t1 = ntiles * (i64)(blockIdx.x + 1) / G;
  const int nmine = (int)(t1 - t0);
  const int ntot = nmine * per_tile;  // atoms of this CTA
  const bool vec4 = (ng % 4 == 0) && ((reinterpret_cast<uintptr_t>(Wsrc) & 15u) == 0) &&
                    (Hsrc == nullptr || (reinterpret_cast<uintptr_t>(Hsrc) & 15u) == 0);
  // atom u -> (tile tt, pass jc, K atom k)
  auto decode = [&](int u, int& tt, int& jc, int& k) {
    tt = u / per_tile;
    k = u - tt * per_tile;
    jc = 0;
    while (k >= big_atoms(jc)) {
      k -= big_atoms(jc);
      ++jc;
    }
  };

  if (warp < PROD_WARPS) {
    // ------------------------------------------------------------ producers
    const int q = lane & 7, isub = lane >> 3;
    auto issue = [&](int u, float4 (&wv)[4], float4 (&hv)[4]) {
      int tt, jc, k;
      decode(u, tt, jc, k);
      const i64 p0 = (t0 + tt) * TPTS + 4 * q;
      const int i = 32 * k + 4 * warp + isub;
#pragma unroll
      for (int g = 0; g < 4; ++g) {
        wv[g] = make_float4(0.f, 0.f, 0.f, 0.f);
        hv[g] = wv[g];
      }
      if (i >= N) return;
      const i64 base = (i64)i * ng + p0;
#pragma unroll
      for (int g = 0; g < 4; ++g) {
        const i64 p = p0 + 32 * g;
        if (vec4) {
          if (p < ng) {
            wv[g] = __ldg(reinterpret_cast<const float4*>(Wsrc + base + 32 * g));
            if (Hsrc) hv[g] = __ldg(reinterpret_cast<const float4*>(Hsrc + base + 32 * g));
          }
        } else {
          float w1[4] = {0.f, 0.f, 0.f, 0.f}, h1[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
          for (int e = 0; e < 4; ++e)
            if (p + e < ng) {
              w1[e] = Wsrc[base + 32 * g + e];
              if (Hsrc) h1[e] = Hsrc[base + 32 * g + e];
            }
          wv[g] = make_float4(w1[0], w1[1], w1[2], w1[3]);
          hv[g] = make_float4(h1[0], h1[1], h1[2], h1[3]);
        }
      }
    };
    // R image of atom u into R slot u & 1 (cp.async, completed one step later)
    auto rcopy = [&](int u) {
      int tt, jc, k;
      decode(u, tt, jc, k);
      const unsigned char* src = img + (size_t)(big_atom0(jc) + k) * SLOT;
      const uint32_t dst = sbase + B_OFF_R + (uint32_t)((u & 1) * SLOT);
      for (int c = tid; c < SLOT / 16; c += PROD_WARPS * 32) tc::cp_async16(dst + 16u * c, src + 16 * c);
      tc::cp_async_commit();
    };
    bool issued = false;
    auto step = [&](int u, const float4 (&w)[4], const float4 (&h)[4], float4 (&wl)[4], float4 (&hl)[4]) -> bool {
      if (u + 2 < ntot) issue(u + 2, wl, hl);
      int tt, jc, k;
      decode(u, tt, jc, k);
      const int P = tt * nb + jc, slot = u & 3;
      // X slot: the MMAs of its previous atom are done, and for a pass's
      // first use, the previous pass's epilogue has read its columns
      if (u >= 4 && !tc::mbar_wait(emptyx(slot), ((u >> 2) - 1) & 1, abort_flag)) return false;
      if (k < 4 && P > 0 && !tc::mbar_wait(xfree(slot), (P - 1) & 1, abort_flag)) return false;
      unsigned char* xs = smem + B_OFF_X + slot * SLOT;
      const float4 cf = coefs[min(32 * k + 4 * warp + isub, BIG_MAXN - 1)];
#pragma unroll
      for (int g = 0; g < 4; ++g) {
        const float x[4] = {w[g].x, w[g].y, w[g].z, w[g].w};
        const float h4[4] = {h[g].x, h[g].y, h[g].z, h[g].w};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int row = 32 * g + 8 * e + q;
          float hi, lo;
          if (Hsrc) {
            tc::trial_split(cf.x, cf.y, x[e], cf.z, cf.w, h4[e], hi, lo);
          } else {
            hi = tc::to_tf32(x[e]);
            lo = x[e] - hi;
          }
          const int off = row * 128 + ((warp ^ q) << 4) + isub * 4;
          *reinterpret_cast<float*>(xs + off) = hi;
          *reinterpret_cast<float*>(xs + ATOM + off) = lo;
        }
      }
      // this thread's R copies for atom u (issued one step earlier) have landed
      tc::cp_async_wait_all();
      tc::fence_proxy_async_smem();
      tc::mbar_arrive(fullx(slot));
      tc::mbar_arrive(fullr(u & 1));
      if (warp == 0) {
        // ---------------------------------------------------- MMA issue
        int ok = 1;
        if (lane == 0) {
          const int natoms = big_atoms(jc), half = natoms / 2;
          if (k == 0 && P > 0) ok = tc::mbar_wait(acce_bar, (P - 1) & 1, abort_flag);
          if (ok) ok = tc::mbar_wait(fullx(slot), (u >> 2) & 1, abort_flag);
          if (ok) ok = tc::mbar_wait(fullr(u & 1), (u >> 1) & 1, abort_flag);
          if (ok) {
            tc::fence_after_sync();
            const uint32_t xh = sbase + B_OFF_X + slot * SLOT, xl = xh + ATOM;
            const uint32_t rh = sbase + B_OFF_R + (u & 1) * SLOT, rl = rh + ATOM;
            const uint32_t dhh = tmem + (k < half ? 0u : COL_HH1), dx = tmem + COL_X;
#pragma unroll
            for (int s4 = 0; s4 < 4; ++s4) {
              const uint64_t axh = tc::desc_sw128(xh + 32u * s4), axl = tc::desc_sw128(xl + 32u * s4);
              const uint64_t brh = tc::desc_sw128(rh + 32u * s4), brl = tc::desc_sw128(rl + 32u * s4);
              tc::mma_tf32(dhh, axh, brh, IDESC128, ((k == 0 || k == half) && s4 == 0) ? 0u : 1u);
              tc::mma_tf32(dx, axh, brl, IDESC128, (k == 0 && s4 == 0) ? 0u : 1u);
              tc::mma_tf32(dx, axl, brh, IDESC128, 1u);
            }
            issued = true;
            tc::mma_commit(emptyx(slot));
            tc::mma_commit(emptyr(u & 1));
            if (k == natoms - 1) tc::mma_commit(accf_bar);
          }
        }
        if (!__shfl_sync(0xffffffffu, ok, 0)) return false;
      }
      // R image of atom u + 1 into the other slot once the MMAs of atom u - 1 are done with it
      if (u + 1 < ntot) {
        if (u + 1 >= 2 && !tc::mbar_wait(emptyr((u + 1) & 1), (((u + 1) >> 1) - 1) & 1, abort_flag)) return false;
        rcopy(u + 1);
      }
      return true;
    };
    float4 wA[4], hA[4], wB[4], hB[4], wC[4], hC[4];
    if (ntot > 0) {
      issue(0, wA, hA);
      rcopy(0);
    }
    if (ntot > 1) issue(1, wB, hB);
    for (int u = 0; u < ntot; u += 3) {
      if (!step(u, wA, hA, wC, hC)) break;
      if (u + 1 >= ntot || !step(u + 1, wB, hB, wA, hA)) break;
      if (u + 2 >= ntot || !step(u + 2, wC, hC, wB, hB)) break;
    }
    tc::cp_async_wait_all();
    if (warp == 0 && lane == 0 && issued) {
      tc::mma_commit(fin_bar);
      tc::mbar_wait(fin_bar, 0, abort_flag, 4000000000ull);
    }
    __syncwarp();
  } else {
    // ------------------------------------------------------------ epilogue
    const int quad = warp & 3;
    const int jh = (warp - EPI0) >> 2;
    const int pt = 32 * quad + 4 * (lane & 7) + (lane >> 3);
    const int row = 32 * quad + lane;
    const uint32_t lane_base = tmem + ((uint32_t)(quad * 32) << 16);
    const uint32_t off_col = COL_OFF + (uint32_t)(64 * jh);
    const unsigned seed32 = mix32((unsigned)(a.st ? a.st->passes : 0) * 4u + (unsigned)a.sr_salt + 0x85ebca6bu);
    float rs[4] = {0.f, 0.f, 0.f, 0.f}, rc[4] = {0.f, 0.f, 0.f, 0.f};
    const int npass = nmine * nb;
    for (int P = 0; P < npass; ++P) {
      const int tt = P / nb, jc = P - tt * nb;
      const i64 p = (t0 + tt) * TPTS + pt;
      if (!tc::mbar_wait(accf_bar, P & 1, abort_flag)) break;
      tc::fence_after_sync();
#pragma unroll 1
      for (int c = 0; c < 64; c += 16) {
        uint32_t h0[16], h1[16], xx[16];
        tc::tmem_ld16(lane_base + (uint32_t)(64 * jh + c), h0);
        tc::tmem_ld16(lane_base + COL_HH1 + (uint32_t)(64 * jh + c), h1);
        tc::tmem_ld16(lane_base + COL_X + (uint32_t)(64 * jh + c), xx);
        tc::tmem_wait_ld();
#pragma unroll
        for (int m = 0; m < 16; ++m)
          h0[m] = __float_as_uint((__uint_as_float(h0[m]) + __uint_as_float(h1[m])) + __uint_as_float(xx[m]));
        tc::tmem_st16(lane_base + off_col + (uint32_t)c, h0);
      }
      tc::tmem_wait_st();
      tc::fence_before_sync();
      tc::mbar_arrive(acce_bar);

      if (jc == 0) {
#pragma unroll
        for (int c = 0; c < 4; ++c) rs[c] = rc[c] = 0.f;
      }
#pragma unroll 1
      for (int g = 0; g < 8; ++g) {
        uint32_t ov[8];
        tc::tmem_ld8(lane_base + off_col + (uint32_t)(8 * g), ov);
        const int jl0 = 64 * jh + 8 * g, j0 = 128 * jc + jl0;
        const unsigned char* xs = smem + B_OFF_X + (jl0 >> 5) * SLOT;
        float xh[8], xl[8];
#pragma unroll
        for (int h4 = 0; h4 < 2; ++h4) {
          const int chunk = ((jl0 & 31) >> 2) + h4;
          const int off = row * 128 + ((chunk ^ (row & 7)) << 4);
          const float4 vh = *reinterpret_cast<const float4*>(xs + off);
          const float4 vl = *reinterpret_cast<const float4*>(xs + ATOM + off);
          xh[4 * h4 + 0] = vh.x, xh[4 * h4 + 1] = vh.y, xh[4 * h4 + 2] = vh.z, xh[4 * h4 + 3] = vh.w;
          xl[4 * h4 + 0] = vl.x, xl[4 * h4 + 1] = vl.y, xl[4 * h4 + 2] = vl.z, xl[4 * h4 + 3] = vl.w;
        }
        tc::tmem_wait_ld();
#pragma unroll
        for (int m4 = 0; m4 < 8; m4 += 4) {
          const unsigned bits = mix32(seed32 ^ mix32((unsigned)((j0 + m4) >> 2) * 0x9e3779b1u ^ (unsigned)p));
#pragma unroll
          for (int m = m4; m < m4 + 4; ++m) {
            const int j = j0 + m;
            const float2 c = self[min(j, BIG_MAXN - 1)];
            const float d = dither(xh[m], (bits >> (8 * (m - m4))) & 0xffu);
            const float o = fmaf(c.x, xh[m], fmaf(c.x, xl[m], fmaf(c.y, xh[m], __uint_as_float(ov[m]) + d)));
            if (p < ng && j < N) {
              out[(i64)j * ng + p] = o;
              const float sq = o * o;
              f2_add(rs[m - m4], rc[m - m4], sq, fmaf(o, o, -sq));
            }
          }
        }
        if ((g & 3) == 3) {
          __syncwarp();
          if (lane == 0) tc::mbar_arrive(xfree(2 * jh + (g >> 2)));
        }
      }
      if (jc == nb - 1 && rho != nullptr) {
        float s0 = rs[0], c0 = rc[0], s2 = rs[2], c2 = rc[2];
        f2_add(s0, c0, rs[1], rc[1]);
        f2_add(s2, c2, rs[3], rc[3]);
        f2_add(s0, c0, s2, c2);
        float2* dq = dens + quad * 32;
        if (jh == 1) dq[lane] = make_float2(s0, c0);
        named_bar(1 + quad, 64);
        if (jh == 0 && p < ng) {
          const float2 o2 = dq[lane];
          rho[p] = F_OCC * (((double)s0 + (double)c0) + ((double)o2.x + (double)o2.y));
        }
        named_bar(1 + quad, 64);
      }
    }
  }

  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, TMEM_COLS);
  }
  if (*abort_flag != 0 && tid == 0) {
    atomicAdd(&g_rotate_tc_aborts, 1u);
    if (a.st) {
      State* w = const_cast<State*>(a.st);
      w->status = 3;
      w->done = 1;
    }
  }
}

bool g_configured = false;

}  // namespace

int rotate_tc_grid(i64 ng) {
  const i64 ntiles = (ng + TPTS - 1) / TPTS;
  return (int)std::max<i64>(1, std::min<i64>(num_sms(), ntiles));
}

void configure_rotate_tc() {
  if (g_configured) return;
  cudaFuncSetAttribute(k_rotate_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
  cudaFuncSetAttribute(k_rotate_tc_big, cudaFuncAttributeMaxDynamicSharedMemorySize, B_SMEM);
  g_configured = true;
}

size_t rotate_rimg_bytes(int N) {
  if (N <= 128) return 0;
  return (size_t)big_atom0((N + 127) / 128) * SLOT;
}

void launch_rotate_tc(const RotArgs<float>& a, cudaStream_t s) {
  configure_rotate_tc();
  const i64 ntiles = (a.ng + TPTS - 1) / TPTS;
  prof_begin(rotate_prof_name(a.trial, a.src_trial_slot, a.src_cur_slot), s);
  if (a.N <= 128) {
    k_rotate_tc<<<rotate_tc_grid(a.ng), NTHR, SMEM_BYTES, s>>>(a, ntiles);
  } else {
    k_rimg<<<big_atom0((a.N + 127) / 128), 256, 0, s>>>(a);
    k_rotate_tc_big<<<rotate_tc_grid(a.ng), NTHR, B_SMEM, s>>>(a, ntiles);
  }
  prof_end(s);
}

}  // namespace pou
