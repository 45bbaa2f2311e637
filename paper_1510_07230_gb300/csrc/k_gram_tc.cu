// Gram matrix of the FP32 form on the 5th-generation tensor cores
// (Cholesky-QR, Sec. 3.2: S = <Wt^T Wt> of the trial block
// Wt = (1 + tau sigma_i) w_i - tau hw_i, of the second-pass block, or of a
// caller's block), for N <= 512 orbitals.
//
// The N x N matrix is cut into 128 x 128 blocks (I, J), I <= J; each CTA
// computes one block over one range of grid points, and the CTAs of one
// range are launched side by side, so that the rows they share are read
// from HBM about once.  A diagonal block streams its 128 rows; an
// off-diagonal block alternates tiles of rows I and rows J of the same 32
// points through the ring, so that every producer thread still holds four
// rows of one block at a time.
//
// Precision: every value x of the block is split into hi = tf32(x) and
// lo = x - hi (exact in FP32 for a plain block; for the trial block x is
// formed from the FP64 coefficients as a double-float and lo is its
// remainder rounded once); the tensor core reads the leading TF32 bits of lo
// (truncation), so x = hi + lo + O(2^-22 x), bit for bit the split the
// tensor-core rotation applies to the block it rotates.  On a diagonal block
// two MMAs of shape M = N = 128, K = 8 per K step accumulate
// D += Hi Hi^T + Hi (2 Lo)^T, so that the symmetric part
// (D + D^T) / 2 = Hi Hi^T + Hi Lo^T + Lo Hi^T is the Gram to about 2^-21
// relative per product (random sign); the reduction kernel takes that
// symmetric part.  An off-diagonal block takes the three products
// D += Jhi Ihi^T + Jhi Ilo^T + Jlo Ihi^T.  The tensor core adds into its FP32
// accumulator with truncation, which biases long sums toward zero, so the
// accumulator is restarted every PERIOD stages (64 grid points) and each
// partial is added into a compensated pair (sum, error) that also lives in
// tensor memory (TwoSum, round to nearest).  The diagonal, the one entry
// whose products all have one sign, is summed exactly on the CUDA cores from
// the FP32 values (double-float) and replaces the tensor-core diagonal; for
// the trial block the reduction replaces it with the FP64 norm from the
// H-apply sums instead.
//
// Roles (one CTA per SM, 416 threads: 13 warps, at most four per SM
// sub-partition, so that each thread may hold 128 registers):
//   warps 0-7   load W (and HW) from global memory two stages ahead (so that
//               each SM keeps two stages of loads in flight), form Wt, split
//               it into TF32 pairs, write the swizzled operand tiles and sum
//               the diagonal;
//   warps 8-11  promote the accumulator into the compensated pair (TMEM lane
//               quadrant = warp - 8) and write the split partial;
//   warp 12     allocates tensor memory; one lane issues the MMAs.
// Stages of 32 grid points (one 128-byte row per orbital) pass through a
// ring guarded by mbarriers; tensor memory holds two accumulators (double
// buffer, so that promoting one period overlaps the MMAs of the next), the
// sum and the error term: 4 x 128 of its 512 columns.
#include "pou_internal.cuh"
#include "tc_ptx.cuh"

#include <algorithm>

namespace pou {

namespace {

constexpr int KB = 32;               // grid points per stage (128 bytes per orbital row)
constexpr int STAGES = 4;
constexpr int PERIOD = 2;            // stages per tensor-memory accumulation period
constexpr int PROD_WARPS = 8, EPI_WARPS = 4;
constexpr int EPI0 = PROD_WARPS;     // first promotion warp
constexpr int MMA_WARP = PROD_WARPS + EPI_WARPS;
constexpr int NTHR = (MMA_WARP + 1) * 32;
constexpr int NPROD = PROD_WARPS * 32;
constexpr int TILE = 128 * 128;      // bytes: 128 rows x 128 bytes
constexpr int STAGE_BYTES = 2 * TILE;  // hi tile, then 2*lo tile
constexpr int OFF_DIAG = STAGES * STAGE_BYTES;  // 128 doubles
constexpr int OFF_BAR = OFF_DIAG + 128 * 8;
// barriers: full[STAGES], empty[STAGES], accf[2], acce[2], fin; then tmem slot, abort flag, coefs
constexpr int NBAR = 2 * STAGES + 5;
constexpr int OFF_MISC = OFF_BAR + NBAR * 8;
constexpr int OFF_COEF = (OFF_MISC + 16 + 15) / 16 * 16;  // float4 entries: 16-byte aligned
static_assert(OFF_COEF % 16 == 0, "coefficient entries must be 16-byte aligned");
constexpr int MAXN = 512;            // orbitals: at most four 128-row blocks
constexpr int SMEM_BYTES = OFF_COEF + MAXN * 16 + 1024;  // + alignment slack
constexpr uint32_t TMEM_COLS = 512;
constexpr uint32_t COL_SUM = 256, COL_ERR = 384;
constexpr uint32_t IDESC = tc::idesc_tf32(128, 128);

static_assert(SMEM_BYTES <= 232448, "tensor-core Gram exceeds the shared-memory opt-in limit");

__device__ unsigned int g_gram_tc_aborts = 0;

__device__ __forceinline__ void two_sum_into(float& s, float& c, float v) {
  const float t = s + v;
  const float bp = t - s;
  c += (s - (t - bp)) + (v - bp);
  s = t;
}

// VEC: rows start on 16-byte boundaries and ng % 4 == 0 (float4 loads); the
// other instantiation loads element by element.  TRIAL: the block is the
// trial point formed from W[cur] and HW[cur]; its diagonal is left to the
// reduction (the FP64 norm from the H-apply sums), which frees the
// producers' diagonal registers for the double-float split.
template <bool VEC, bool TRIAL>
__global__ void __launch_bounds__(NTHR, 1) k_gram_tc(GramArgs<float> a, i64 nkb, int nsplit) {
  extern __shared__ unsigned char smem_raw[];
  if (a.st && a.st->done) return;
  if (!gate_open(a.st, a.gate)) return;

  // 1024-byte aligned base for the swizzled operand tiles
  const uint32_t raw_addr = tc::smem_u32(smem_raw);
  const uint32_t pad = (1024u - (raw_addr & 1023u)) & 1023u;
  unsigned char* smem = smem_raw + pad;
  const uint32_t sbase = raw_addr + pad;
  double* diag = reinterpret_cast<double*>(smem + OFF_DIAG);
  const uint32_t bar0 = sbase + OFF_BAR;
  auto full_bar = [&](int s) { return bar0 + 8u * s; };
  auto empty_bar = [&](int s) { return bar0 + 8u * (STAGES + s); };
  auto accf_bar = [&](int b) { return bar0 + 8u * (2 * STAGES + b); };
  auto acce_bar = [&](int b) { return bar0 + 8u * (2 * STAGES + 2 + b); };
  const uint32_t fin_bar = bar0 + 8u * (2 * STAGES + 4);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + OFF_MISC);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + OFF_MISC + 4);
  // per orbital: 1 + t_i sigma_i and its step t_i, each as (hi, lo)
  float4* coefs = reinterpret_cast<float4*>(smem + OFF_COEF);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int N = a.N;
  const i64 ng = a.ng;

  // block pair (I, J) of this CTA and its contiguous range of 32-point
  // chunks (pairs in upper row-major order).  With one block (N <= 128) CTA
  // = split.  With several, an off-diagonal pair streams two tiles per chunk
  // and a diagonal one a single tile, so a diagonal pair takes two splits at
  // once: every CTA then streams the same number of tiles.  CTAs come in
  // groups of npair + noff: split 2q for every pair (the diagonal ones
  // covering splits 2q and 2q + 1, whose slot they fill with zeros), then
  // split 2q + 1 for the off-diagonal pairs.
  const int nsup = (N + 127) / 128, npair = nsup * (nsup + 1) / 2, noff = npair - nsup;
  int pair;
  i64 split;
  if (nsup == 1) {
    pair = 0;
    split = blockIdx.x;
  } else {
    const int q = (int)(blockIdx.x / (npair + noff)), r = (int)(blockIdx.x % (npair + noff));
    if (r < npair) {
      pair = r;
      split = 2 * q;
    } else {
      // the (r - npair)-th off-diagonal pair
      int k = r - npair, Io = 0;
      for (; k >= nsup - 1 - Io; k -= nsup - 1 - Io, ++Io) {
      }
      pair = Io * nsup - Io * (Io - 1) / 2 + 1 + k;
      split = 2 * q + 1;
    }
  }
  int I = 0, J = 0;
  for (int p = pair; p >= nsup - I; p -= nsup - I, ++I) {
  }
  J = I + (pair - (I * nsup - I * (I - 1) / 2));
  const bool offd = I != J;
  const i64 G = nsplit;
  const i64 split_end = (nsup > 1 && !offd) ? (split + 2 < G ? split + 2 : G) : split + 1;
  const i64 zslot = (nsup > 1 && !offd && split + 1 < G) ? split + 1 : -1;  // slot this CTA zeroes
  const i64 kb0 = nkb * split / G, kb1 = nkb * split_end / G;
  // steps: one 128-row tile each; an off-diagonal block takes the I and the
  // J tile of every chunk in turn
  const int nmine = (int)(kb1 - kb0) * (offd ? 2 : 1);
  const int nper = (nmine + PERIOD - 1) / PERIOD;

  const float* Wa;
  const float* Ha = nullptr;
  if (TRIAL) {
    const int cur = a.st->cur;
    Wa = a.W[cur];
    Ha = a.HW[cur];
    const double tau = a.st->tau_trial;
    for (int r = tid; r < MAXN; r += NTHR) {
      const double t = (r < N && a.tfac) ? tau * a.tfac[r] : tau;
      const double cf = r < N ? 1.0 + t * a.sigma[cur][r] : 0.0;
      const float ch = (float)cf, th = (float)t;
      coefs[r] = make_float4(ch, (float)(cf - (double)ch), th, (float)(t - (double)th));
    }
  } else if (a.src_trial_slot) {
    Wa = a.W[1 - a.st->cur];
  } else {
    Wa = a.A;
  }
  for (int r = tid; r < 128; r += NTHR) diag[r] = 0.0;
  if (tid == 0) {
    for (int s = 0; s < STAGES; ++s) {
      tc::mbar_init(full_bar(s), NPROD);
      tc::mbar_init(empty_bar(s), 1);
    }
    for (int b = 0; b < 2; ++b) {
      tc::mbar_init(accf_bar(b), 1);
      tc::mbar_init(acce_bar(b), EPI_WARPS * 32);
    }
    tc::mbar_init(fin_bar, 1);
    *abort_flag = 0;
    tc::mbar_init_fence();
  }
  if (warp == MMA_WARP) {
    tc::tmem_alloc(tc::smem_u32(tmem_slot), TMEM_COLS);
    tc::tmem_relinquish();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tmem_slot;

  if (warp < PROD_WARPS) {
    // ------------------------------------------------------------ producers
    const int pt = tid;
    const int c = pt & 7;         // 16-byte chunk of the row: points 4c .. 4c+3
    const int r0 = pt >> 3;       // rows r0 + 32 q
    float ds[4] = {0.f, 0.f, 0.f, 0.f}, dc[4] = {0.f, 0.f, 0.f, 0.f};  // diagonal, double-float
    // step i: chunk kb0 + i (diagonal) or kb0 + i / 2, rows of block I or J
    auto rbase = [&](int i) { return 128 * ((offd && (i & 1)) ? J : I); };
    auto load = [&](int i, float4 (&wv)[4], float4 (&hv)[4]) {
      const i64 kb = kb0 + (offd ? (i >> 1) : i);
      const int rb = rbase(i);
      const i64 p = kb * KB + 4 * c;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int r = rb + r0 + 32 * q;
        wv[q] = make_float4(0.f, 0.f, 0.f, 0.f);
        hv[q] = wv[q];
        if (r >= N) continue;
        const i64 off = (i64)r * ng + p;
        if (VEC) {
          // ng % 4 == 0: a chunk is either wholly inside the row or past its end
          if (p < ng) {
            wv[q] = __ldg(reinterpret_cast<const float4*>(Wa + off));
            if (TRIAL) hv[q] = __ldg(reinterpret_cast<const float4*>(Ha + off));
          }
        } else {
          float t[4] = {0.f, 0.f, 0.f, 0.f}, u[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
          for (int e = 0; e < 4; ++e)
            if (p + e < ng) {
              t[e] = Wa[off + e];
              if (TRIAL) u[e] = Ha[off + e];
            }
          wv[q] = make_float4(t[0], t[1], t[2], t[3]);
          hv[q] = make_float4(u[0], u[1], u[2], u[3]);
        }
      }
    };
    // one stage: loads for stage i + 2 go into the register set that held
    // stage i - 1; stage i is written from (w, h)
    // lo is stored doubled for the symmetric two-product form of a diagonal block
    const float lo_scale = offd ? 1.0f : 2.0f;
    auto step = [&](int i, const float4 (&w)[4], const float4 (&h)[4], float4 (&wl)[4], float4 (&hl)[4]) -> bool {
      if (i + 2 < nmine) load(i + 2, wl, hl);
      const int s = i % STAGES, n = i / STAGES;
      if (n > 0 && !tc::mbar_wait(empty_bar(s), (n - 1) & 1, abort_flag)) return false;
      unsigned char* hi_t = smem + s * STAGE_BYTES;
      unsigned char* lo_t = hi_t + TILE;
      const int rb = rbase(i);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int r = r0 + 32 * q;  // row within the tile
        const float x[4] = {w[q].x, w[q].y, w[q].z, w[q].w};
        float hi[4], lo[4];
        if (TRIAL) {
          const float4 cf = coefs[rb + r];
          const float hv4[4] = {h[q].x, h[q].y, h[q].z, h[q].w};
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            tc::trial_split(cf.x, cf.y, x[e], cf.z, cf.w, hv4[e], hi[e], lo[e]);
            lo[e] *= lo_scale;
          }
        } else {
          float sq = 0.f;
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            hi[e] = tc::to_tf32(x[e]);
            lo[e] = lo_scale * (x[e] - hi[e]);  // exact; the tensor core reads its leading TF32 bits
            sq = fmaf(x[e], x[e], sq);
          }
          two_sum_into(ds[q], dc[q], sq);
        }
        const int off = r * 128 + ((c ^ (r & 7)) << 4);
        *reinterpret_cast<float4*>(hi_t + off) = make_float4(hi[0], hi[1], hi[2], hi[3]);
        *reinterpret_cast<float4*>(lo_t + off) = make_float4(lo[0], lo[1], lo[2], lo[3]);
      }
      tc::fence_proxy_async_smem();
      tc::mbar_arrive(full_bar(s));
      return true;
    };
    float4 wA[4], hA[4], wB[4], hB[4], wC[4], hC[4];
    if (nmine > 0) load(0, wA, hA);
    if (nmine > 1) load(1, wB, hB);
    for (int i = 0; i < nmine; i += 3) {
      if (!step(i, wA, hA, wC, hC)) break;
      if (i + 1 >= nmine || !step(i + 1, wB, hB, wA, hA)) break;
      if (i + 2 >= nmine || !step(i + 2, wC, hC, wB, hB)) break;
    }
    // the eight lanes that share a row hold its diagonal in parts (the sums
    // of an off-diagonal block are not used)
#pragma unroll
    for (int q = 0; q < (TRIAL ? 0 : 4); ++q) {
#pragma unroll
      for (int o = 1; o <= 4; o <<= 1) {
        const float os = __shfl_xor_sync(0xffffffffu, ds[q], o);
        const float oc = __shfl_xor_sync(0xffffffffu, dc[q], o);
        two_sum_into(ds[q], dc[q], os);
        dc[q] += oc;
      }
      if (c == 0) diag[r0 + 32 * q] = (double)ds[q] + (double)dc[q];
    }
  } else if (warp == MMA_WARP) {
    // ------------------------------------------------------------ MMA issue
    // single: one TF32 product hi hi per K step (the plain TF32 form); else
    // the split products hi hi + hi lo + lo hi (hi hi + 2 hi lo on a
    // diagonal block)
    const bool single = a.tf32_single != 0;
    if (lane == 0) {
      int it = 0;
      bool ok = true, issued = false;
      for (int per = 0; per < nper && ok; ++per) {
        const int b = per & 1, use = per >> 1;
        if (use > 0 && !tc::mbar_wait(acce_bar(b), (use - 1) & 1, abort_flag)) break;
        tc::fence_after_sync();
        const uint32_t d = tmem + (uint32_t)(b * 128);
        if (offd) {
          // one chunk per period: tile I in stage s0, tile J in stage s1
          const int s0 = it % STAGES, s1 = (it + 1) % STAGES;
          if (!tc::mbar_wait(full_bar(s0), (it / STAGES) & 1, abort_flag) ||
              !tc::mbar_wait(full_bar(s1), ((it + 1) / STAGES) & 1, abort_flag)) {
            ok = false;
            break;
          }
          tc::fence_after_sync();
          const uint32_t ih = sbase + (uint32_t)(s0 * STAGE_BYTES), il = ih + TILE;
          const uint32_t jh = sbase + (uint32_t)(s1 * STAGE_BYTES), jl = jh + TILE;
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const uint64_t djh = tc::desc_sw128(jh + 32u * k), djl = tc::desc_sw128(jl + 32u * k);
            const uint64_t dih = tc::desc_sw128(ih + 32u * k), dil = tc::desc_sw128(il + 32u * k);
            // D[j][i] (TMEM lane = row of block J)
            tc::mma_tf32(d, djh, dih, IDESC, k == 0 ? 0u : 1u);
            if (!single) {
              tc::mma_tf32(d, djh, dil, IDESC, 1u);
              tc::mma_tf32(d, djl, dih, IDESC, 1u);
            }
          }
          issued = true;
          tc::mma_commit(empty_bar(s0));
          tc::mma_commit(empty_bar(s1));
          it += 2;
          tc::mma_commit(accf_bar(b));
          continue;
        }
        const int end = std::min(nmine, it + PERIOD);
        for (bool first = true; it < end; ++it, first = false) {
          const int s = it % STAGES, n = it / STAGES;
          if (!tc::mbar_wait(full_bar(s), n & 1, abort_flag)) {
            ok = false;
            break;
          }
          tc::fence_after_sync();
          const uint32_t hi_a = sbase + (uint32_t)(s * STAGE_BYTES), lo_a = hi_a + TILE;
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const uint64_t dh = tc::desc_sw128(hi_a + 32u * k), dl = tc::desc_sw128(lo_a + 32u * k);
            tc::mma_tf32(d, dh, dh, IDESC, (first && k == 0) ? 0u : 1u);
            if (!single) tc::mma_tf32(d, dh, dl, IDESC, 1u);
          }
          issued = true;
          tc::mma_commit(empty_bar(s));
        }
        if (ok) tc::mma_commit(accf_bar(b));
      }
      // every MMA issued has completed before tensor memory is released
      if (issued) {
        tc::mma_commit(fin_bar);
        tc::mbar_wait(fin_bar, 0, abort_flag, 4000000000ull);
      }
    }
    __syncwarp();
  } else {
    // ------------------------------------------------------------ promotion
    const int quad = warp - EPI0;
    const uint32_t lane_base = tmem + ((uint32_t)(quad * 32) << 16);
    for (int per = 0; per < nper; ++per) {
      const int b = per & 1, use = per >> 1;
      if (!tc::mbar_wait(accf_bar(b), use & 1, abort_flag)) break;
      tc::fence_after_sync();
#pragma unroll 1
      for (int c0 = 0; c0 < 128; c0 += 16) {
        uint32_t x[16], sv[16], cv[16];
        tc::tmem_ld16(lane_base + (uint32_t)(b * 128 + c0), x);
        if (per > 0) {
          tc::tmem_ld16(lane_base + COL_SUM + c0, sv);
          tc::tmem_ld16(lane_base + COL_ERR + c0, cv);
        }
        tc::tmem_wait_ld();
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          float s = 0.f, e = 0.f;
          if (per > 0) {
            s = __uint_as_float(sv[j]);
            e = __uint_as_float(cv[j]);
          }
          two_sum_into(s, e, __uint_as_float(x[j]));
          sv[j] = __float_as_uint(s);
          cv[j] = __float_as_uint(e);
        }
        tc::tmem_st16(lane_base + COL_SUM + c0, sv);
        tc::tmem_st16(lane_base + COL_ERR + c0, cv);
      }
      tc::tmem_wait_st();
      tc::fence_before_sync();
      tc::mbar_arrive(acce_bar(b));
    }
  }

  tc::fence_before_sync();
  __syncthreads();
  // split partial of block (I, J), stored column-major: entry (i, j) of a
  // diagonal block at [j][i] (the reduction symmetrises), entry (i, j) of an
  // off-diagonal block (TMEM lane = j) at [i][j]
  const bool bad = *abort_flag != 0;
  double* out = a.split + (split * npair + pair) * (128 * 128);
  double* zout = zslot >= 0 ? a.split + (zslot * npair + pair) * (128 * 128) : nullptr;
  if (warp >= EPI0 && warp < MMA_WARP) {
    tc::fence_after_sync();
    const int quad = warp - EPI0;
    const int row = quad * 32 + lane;  // TMEM lane
    const uint32_t lane_base = tmem + ((uint32_t)(quad * 32) << 16);
#pragma unroll 1
    for (int c0 = 0; c0 < 128; c0 += 16) {
      uint32_t sv[16], cv[16];
      tc::tmem_ld16(lane_base + COL_SUM + c0, sv);
      tc::tmem_ld16(lane_base + COL_ERR + c0, cv);
      tc::tmem_wait_ld();
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int col = c0 + j;
        double v = (double)__uint_as_float(sv[j]) + (double)__uint_as_float(cv[j]);
        if (nper == 0) v = 0.0;
        if (!offd && col == row) v = diag[row];
        if (bad) v = __longlong_as_double(0x7ff8000000000000ll);
        out[(i64)col * 128 + row] = v;
        if (zout) zout[(i64)col * 128 + row] = 0.0;
      }
    }
    tc::fence_before_sync();
  }
  __syncthreads();
  if (warp == MMA_WARP) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, TMEM_COLS);
  }
  if (bad && tid == 0) {
    atomicAdd(&g_gram_tc_aborts, 1u);
    if (a.st) {
      State* w = const_cast<State*>(a.st);
      w->status = 3;  // POU_ECUDA: a pipeline wait gave up
      w->done = 1;
    }
  }
}

bool g_configured = false;

}  // namespace

int gram_tc_ctas(int nsplit, int nsup) {
  if (nsup == 1) return nsplit;
  const int npair = nsup * (nsup + 1) / 2, noff = npair - nsup;
  return nsplit * noff + (nsplit + 1) / 2 * nsup;
}

bool gram_tc_eligible(const GramArgs<float>& a) {
  return a.B == nullptr && !a.src_cur_pair && a.N >= 1 && a.N <= MAXN;
}


void configure_gram_tc() {
  if (g_configured) return;
  cudaFuncSetAttribute(k_gram_tc<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
  cudaFuncSetAttribute(k_gram_tc<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
  cudaFuncSetAttribute(k_gram_tc<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
  cudaFuncSetAttribute(k_gram_tc<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
  g_configured = true;
}

void launch_gram_tc(const GramArgs<float>& a, int nsplit, cudaStream_t s) {
  configure_gram_tc();
  const i64 nkb = (a.ng + KB - 1) / KB;
  prof_begin(gram_prof_name(a.trial, a.src_trial_slot, a.src_cur_pair), s);
  // one CTA per (split, block pair), a diagonal pair's CTA covering two
  // splits when there are several blocks; a CTA without stages writes zeros
  const int nsup = (a.N + 127) / 128, npair = nsup * (nsup + 1) / 2, noff = npair - nsup;
  const int nblk = gram_tc_ctas(nsplit, nsup);
  // the source rows of the mode: W[cur] and HW[cur] (trial), W[1 - cur], or A
  bool vec = (a.ng % 4) == 0;
  auto aligned = [](const float* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; };
  if (a.trial || a.src_trial_slot) {
    for (int k = 0; k < 2; ++k) vec = vec && aligned(a.W[k]) && (!a.trial || aligned(a.HW[k]));
  } else {
    vec = vec && aligned(a.A);
  }
  if (a.trial) {
    if (vec)
      k_gram_tc<true, true><<<nblk, NTHR, SMEM_BYTES, s>>>(a, nkb, nsplit);
    else
      k_gram_tc<false, true><<<nblk, NTHR, SMEM_BYTES, s>>>(a, nkb, nsplit);
  } else if (vec) {
    k_gram_tc<true, false><<<nblk, NTHR, SMEM_BYTES, s>>>(a, nkb, nsplit);
  } else {
    k_gram_tc<false, false><<<nblk, NTHR, SMEM_BYTES, s>>>(a, nkb, nsplit);
  }
  prof_end(s);
}

}  // namespace pou

namespace pou {
namespace {
// Self-test of the bounded barrier wait every tensor-core kernel relies on:
// one thread waits on an mbarrier that expects one arrival and gets none, so
// the wait gives up after limit_ns and records it; no tensor memory is held
// and nothing else waits.
__global__ void k_wait_selftest(uint64_t limit_ns, int* out) {
  __shared__ __align__(8) uint64_t bar;
  __shared__ volatile int abort_flag;
  if (threadIdx.x == 0) {
    abort_flag = 0;
    const uint32_t b = tc::smem_u32(&bar);
    tc::mbar_init(b, 1);
    tc::mbar_init_fence();
    const bool ok = tc::mbar_wait(b, 0, &abort_flag, limit_ns);
    out[0] = ok ? 0 : 1;
    out[1] = abort_flag;
  }
}
}  // namespace

int wait_selftest(double limit_s, int* timed_out) {
  int* d = nullptr;
  if (cudaMalloc(&d, 2 * sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    return 2;
  }
  const uint64_t ns = (uint64_t)(limit_s * 1e9);
  k_wait_selftest<<<1, 32>>>(ns, d);
  int h[2] = {0, 0};
  const cudaError_t e1 = cudaGetLastError();
  const cudaError_t e2 = cudaMemcpy(h, d, sizeof h, cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e1 != cudaSuccess || e2 != cudaSuccess) return 3;
  *timed_out = (h[0] == 1 && h[1] == 1) ? 1 : 0;
  return 0;
}

}  // namespace pou
