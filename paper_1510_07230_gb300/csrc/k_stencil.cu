// H-apply pass: HW = -1/2 Lap_h W + V W on a uniform periodic grid, fused
// with the per-orbital sums the iteration needs (Sec. 3.2):
//   sigma_ii = <H w_i, w_i>, the kinetic energy f <w_i, -1/2 Lap_h w_i>
//   (Eq. energy, kept per axis without the 1/h^2 factors), the sums of
//   z' = hw - sigma' w, and the Barzilai-Borwein traces against the current
//   iterate W' (S = W - W', Y = Z - Z').
//
// The gradient difference is formed from the step itself,
//   hw - hw' = -1/2 Lap_h s + V s + (V - V') w',   s = w - w',
// with V - V' formed from the FP64 potentials by the potential pass (once per
// grid point), so that every operand is as small as the step: for tiny steps
// an FP32 difference of two H-products would be all rounding noise.  HW' is
// therefore never read.
//
// Layout: one orbital after another, [nz][ny][nx] each, x fastest.
// One CTA = one orbital x a 32x8 (x, y) tile x a range of z planes.  Planes
// stream through a shared-memory ring (cp.async, PF planes in flight): each
// stage holds the plane of w (and w') with an x/y halo of width R (periodic
// wrap), V and, with history, V - V'.  Each thread keeps its
// column's z-neighbours in register queues.  Second differences are sums of
// neighbour differences, (u[+d] - u) + (u[-d] - u), exact for smooth fields.
#include "pou_internal.cuh"

namespace pou {

long long g_launches = 0;
thread_local ProfRecorder* g_prof = nullptr;

int num_sms() {
  constexpr int kMaxDev = 64;
  static int cache[kMaxDev] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) {
    cudaGetLastError();
    return 152;  // GB300; the launch that follows reports the device error
  }
  if (cache[dev] == 0) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) {
      cudaGetLastError();
      v = 152;
    }
    cache[dev] = v;
  }
  return cache[dev];
}

namespace {

constexpr int TX = 32;
constexpr int TY = 8;
constexpr int NT = TX * TY;
constexpr int PF = 2;  // planes in flight beyond the one being consumed

__device__ __forceinline__ int wrapi(int v, int n) {
  v %= n;
  return v < 0 ? v + n : v;
}

template <int BYTES>
__device__ __forceinline__ void cp_async(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(s), "l"(gmem), "n"(BYTES));
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}
// 16-byte copy through L2 only (both addresses 16-byte aligned)
__device__ __forceinline__ void cp_async16_cg(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem));
}

template <typename T, int R>
struct Stage {
  T w[TY + 2 * R][TX + 2 * R];
  T p[TY + 2 * R][TX + 2 * R];  // w' (history only)
  T v[TY][TX];
  T dv[TY][TX];  // V - V' (history only)
};

// Compensated (Kahan) running sum: the sums that enter the energy and the
// Gram diagonal run over a whole z range per thread, where plain FP32
// accumulation would cost about 1e-9 relative.
template <typename T>
struct Ksum {
  T s, c;
  __device__ __forceinline__ void add(T x) {
    const T y = x - c;
    const T t = s + y;
    c = (t - s) - y;
    s = t;
  }
  __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

template <typename T, int R>
__global__ void __launch_bounds__(NT) k_apply_h(ApplyArgs<T> a) {
  constexpr int S = R + 2 + PF;  // ring: freed plane, computing plane .. arrived plane, in flight
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Stage<T, R>* ring = reinterpret_cast<Stage<T, R>*>(smem_raw);
  __shared__ double red[NT / 32][NPT];

  if (a.st && a.st->done) return;
  if (a.mode == 3 && !a.st->diag_now) return;
  if (a.mode == 4 && a.st->s != 0) return;
  const int cur = a.st ? a.st->cur : 0;
  const int t = (a.mode == 2) ? 0 : ((a.mode == 3 || a.mode == 4) ? cur : 1 - cur);
  const bool prev = (a.mode == 0);
  const int nx = a.nx, ny = a.ny, nz = a.nz;
  const i64 ng = (i64)nx * ny * nz;
  const int orb = blockIdx.z;
  const T* w = a.W[t] + (i64)orb * ng;
  T* hw = a.HW[t] ? a.HW[t] + (i64)orb * ng : nullptr;
  const T* V = a.V[t];
  const T* wp = prev ? a.W[cur] + (i64)orb * ng : nullptr;
  const T* dVp = prev ? a.dV : nullptr;
  // sigma' the z' sums refer to: the reference iterate's (mode 0) or the
  // eigenvalue of the rotated orbital (mode 3)
  const T sigp = (prev || a.mode == 3) ? (T)a.sigma[cur][orb] : T(0);

  const int ntx = (nx + TX - 1) / TX;
  const int tx0 = (blockIdx.x % ntx) * TX;
  const int ty0 = (blockIdx.x / ntx) * TY;
  const int z0 = (int)(((i64)blockIdx.y * nz) / a.nzc);
  const int z1 = (int)(((i64)(blockIdx.y + 1) * nz) / a.nzc);

  const int lx = threadIdx.x, ly = threadIdx.y;
  const int tid = ly * TX + lx;
  const int x = tx0 + lx, y = ty0 + ly;
  const bool act = (x < nx) && (y < ny);
  // every thread of the tile tracks its (wrapped) column so that tile cells
  // past the grid edge hold the periodic neighbours
  const i64 col = (i64)wrapi(y, ny) * nx + wrapi(x, nx);
  const i64 pl = (i64)nx * ny;

  // halo cell owned by this thread (80 R cells per plane)
  int hx = -1, hy = 0, sx = 0, sy = 0;
  if (tid < 2 * R * TY) {  // left / right columns
    const int side = tid / (R * TY), r = tid % (R * TY);
    const int row = r / R, d = r % R;
    sy = row + R;
    sx = side == 0 ? d : TX + R + d;
    hx = wrapi(side == 0 ? tx0 - R + d : tx0 + TX + d, nx);
    hy = wrapi(ty0 + row, ny);
  } else if (tid < 2 * R * TY + 2 * R * TX) {  // top / bottom rows
    const int u = tid - 2 * R * TY;
    const int side = u / (R * TX), r = u % (R * TX);
    const int d = r / TX, c = r % TX;
    sx = c + R;
    sy = side == 0 ? d : TY + R + d;
    hx = wrapi(tx0 + c, nx);
    hy = wrapi(side == 0 ? ty0 - R + d : ty0 + TY + d, ny);
  }
  const i64 hcol = (hx >= 0) ? (i64)hy * nx + hx : 0;

  // plane pa is needed for pa in [z0 - R, z1 + R); it lives in stage (pa - z0 + R) mod S
  const int a_first = z0 - R, a_last = z1 + R;  // exclusive end
  auto stage_of = [&](int pa) { return (pa - a_first) % S; };
  auto issue = [&](int pa) {
    if (pa < a_last) {
      Stage<T, R>& g = ring[stage_of(pa)];
      const i64 zo = (i64)wrapi(pa, nz) * pl;
      cp_async<sizeof(T)>(&g.w[ly + R][lx + R], w + zo + col);
      if (hx >= 0) cp_async<sizeof(T)>(&g.w[sy][sx], w + zo + hcol);
      if (prev) {
        cp_async<sizeof(T)>(&g.p[ly + R][lx + R], wp + zo + col);
        if (hx >= 0) cp_async<sizeof(T)>(&g.p[sy][sx], wp + zo + hcol);
      }
      if (pa >= z0 && pa < z1) {
        cp_async<sizeof(T)>(&g.v[ly][lx], V + zo + col);
        if (prev) cp_async<sizeof(T)>(&g.dv[ly][lx], dVp + zo + col);
      }
    }
    cp_commit();  // one group per plane, empty past the end
  };

  for (int pa = a_first; pa < a_first + PF + 1; ++pa) issue(pa);

  T qw[2 * R + 1], qp[2 * R + 1];
#pragma unroll
  for (int j = 0; j <= 2 * R; ++j) qw[j] = qp[j] = T(0);
  T acc[NPT];
#pragma unroll
  for (int k = 0; k < NPT; ++k) acc[k] = T(0);
  // compensated: P_WW, P_ZW, P_ZZ, P_KX, P_KY, P_KZ
  Ksum<T> kww{T(0), T(0)}, kzw{T(0), T(0)}, kzz{T(0), T(0)}, kkx{T(0), T(0)}, kky{T(0), T(0)}, kkz{T(0), T(0)};
  const T ihx2 = a.ihx2, ihy2 = a.ihy2, ihz2 = a.ihz2;

  for (int pa = a_first; pa < a_last; ++pa) {
    cp_wait<PF>();    // plane pa has landed (this thread's copies)
    __syncthreads();  // ... everyone's; and plane pa - R - 1 is no longer read
    issue(pa + PF + 1);
    const Stage<T, R>& ga = ring[stage_of(pa)];
    // shift the z queues and append the centre values of plane pa
#pragma unroll
    for (int j = 0; j < 2 * R; ++j) {
      qw[j] = qw[j + 1];
      qp[j] = qp[j + 1];
    }
    qw[2 * R] = ga.w[ly + R][lx + R];
    qp[2 * R] = prev ? ga.p[ly + R][lx + R] : T(0);
    const int z = pa - R;
    if (z < z0 || !act) continue;
    const Stage<T, R>& g = ring[stage_of(z)];
    const int cx = lx + R, cy = ly + R;
    const T c = qw[R];
    // second differences of w along each axis, without 1/h^2 (order 4: 16 d1 - d2)
    T ex, ey, ez;
    {
      const T dx1 = (g.w[cy][cx + 1] - c) + (g.w[cy][cx - 1] - c);
      const T dy1 = (g.w[cy + 1][cx] - c) + (g.w[cy - 1][cx] - c);
      const T dz1 = (qw[R + 1] - c) + (qw[R - 1] - c);
      if (R == 1) {
        ex = dx1;
        ey = dy1;
        ez = dz1;
      } else {
        const T dx2 = (g.w[cy][cx + 2] - c) + (g.w[cy][cx - 2] - c);
        const T dy2 = (g.w[cy + 2][cx] - c) + (g.w[cy - 2][cx] - c);
        const T dz2 = (qw[R + 2] - c) + (qw[R - 2] - c);
        ex = T(16) * dx1 - dx2;
        ey = T(16) * dy1 - dy2;
        ez = T(16) * dz1 - dz2;
      }
    }
    const i64 idx = (i64)z * pl + col;
    const T lap = ihx2 * ex + ihy2 * ey + ihz2 * ez;
    const T kin = T(-0.5) * lap;
    const T vv = g.v[ly][lx];
    T h = kin + vv * c;
    if (a.nl) h += a.nl[(i64)orb * ng + idx];
    if (hw) hw[idx] = a.out_scale * h;
    const T zp = h - sigp * c;
    kww.add(c * c);
    acc[P_HW] += h * c;
    kzw.add(zp * c);
    kzz.add(zp * zp);
    kkx.add(c * ex);
    kky.add(c * ey);
    kkz.add(c * ez);
    if (prev) {
      // s = w - w' and H applied to it
      const T sc = c - qp[R];
      auto sv = [&](int yy, int xx) { return g.w[yy][xx] - g.p[yy][xx]; };
      T fx, fy, fz;
      {
        const T sx1 = (sv(cy, cx + 1) - sc) + (sv(cy, cx - 1) - sc);
        const T sy1 = (sv(cy + 1, cx) - sc) + (sv(cy - 1, cx) - sc);
        const T sz1 = ((qw[R + 1] - qp[R + 1]) - sc) + ((qw[R - 1] - qp[R - 1]) - sc);
        if (R == 1) {
          fx = sx1;
          fy = sy1;
          fz = sz1;
        } else {
          const T sx2 = (sv(cy, cx + 2) - sc) + (sv(cy, cx - 2) - sc);
          const T sy2 = (sv(cy + 2, cx) - sc) + (sv(cy - 2, cx) - sc);
          const T sz2 = ((qw[R + 2] - qp[R + 2]) - sc) + ((qw[R - 2] - qp[R - 2]) - sc);
          fx = T(16) * sx1 - sx2;
          fy = T(16) * sy1 - sy2;
          fz = T(16) * sz1 - sz2;
        }
      }
      const T dvv = g.dv[ly][lx];
      T hs = T(-0.5) * (ihx2 * fx + ihy2 * fy + ihz2 * fz) + vv * sc + dvv * qp[R];
      if (a.nls) hs += a.nls[(i64)orb * ng + idx];
      const T b = hs - sigp * sc;  // (hw - hw') - sigma' s
      acc[P_SS] += sc * sc;
      acc[P_SB] += sc * b;
      acc[P_SW] += sc * c;
      acc[P_BB] += b * b;
      acc[P_BW] += b * c;
    }
  }
  cp_wait<0>();

  if (a.tilepart == nullptr) return;
  // block reduction of the sums, promoted to FP64 before combining threads
  const int lane = tid & 31, warp = tid >> 5;
  double fin[NPT];
#pragma unroll
  for (int k = 0; k < NPT; ++k) fin[k] = (double)acc[k];
  fin[P_WW] = kww.value();
  fin[P_ZW] = kzw.value();
  fin[P_ZZ] = kzz.value();
  fin[P_KX] = kkx.value();
  fin[P_KY] = kky.value();
  fin[P_KZ] = kkz.value();
#pragma unroll
  for (int k = 0; k < NPT; ++k) {
    double v = fin[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[warp][k] = v;
  }
  __syncthreads();
  if (tid < NPT) {
    double v = 0.0;
#pragma unroll
    for (int wi = 0; wi < NT / 32; ++wi) v += red[wi][tid];
    const int ntile = gridDim.x * gridDim.y;
    const int tile = blockIdx.y * gridDim.x + blockIdx.x;
    a.tilepart[((i64)orb * ntile + tile) * NPT + tid] = v;
  }
}

// ----------------------------------------------------------------------------
// Paired variant (even nx): each thread owns two adjacent x points, so every
// copy and shared-memory access moves two elements, and the per-plane address
// arithmetic, the z-queue shifts and the compensated additions are shared by
// the pair.  Stage indices are compile-time (the plane loop is unrolled by the
// ring size) and plane offsets advance incrementally (no integer division).
// The x halo is two elements wide on each side for both stencils, which keeps
// the pairs 2-element aligned.
template <typename T>
struct Vec2;
template <>
struct Vec2<float> {
  typedef float2 type;
};
template <>
struct Vec2<double> {
  typedef double2 type;
};

constexpr int PTX = 2 * TX;        // points per tile row
constexpr int PRW = PTX + 4;       // shared row: 2 halo cells each side
constexpr int PPF = 2;             // planes in flight

template <typename T, int R>
struct PStage {
  T w[TY + 2 * R][PRW];
  T p[TY + 2 * R][PRW];
  T v[TY][PTX];
  T dv[TY][PTX];
};

template <typename T, int R>
__global__ void __launch_bounds__(NT, sizeof(T) == 4 ? 2 : 1) k_apply_h_pair(ApplyArgs<T> a) {
  typedef typename Vec2<T>::type V2;
  constexpr int S = R + 2 + PPF;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  PStage<T, R>* ring = reinterpret_cast<PStage<T, R>*>(smem_raw);
  __shared__ double red[NT / 32][NPT];

  if (a.st && a.st->done) return;
  if (a.mode == 3 && !a.st->diag_now) return;
  if (a.mode == 4 && a.st->s != 0) return;
  const int cur = a.st ? a.st->cur : 0;
  const int t = (a.mode == 2) ? 0 : ((a.mode == 3 || a.mode == 4) ? cur : 1 - cur);
  const bool prev = (a.mode == 0);
  const int nx = a.nx, ny = a.ny, nz = a.nz;
  const i64 pl = (i64)nx * ny;
  const i64 ng = pl * nz;
  const int orb = blockIdx.z;
  const T* w = a.W[t] + (i64)orb * ng;
  T* hw = a.HW[t] ? a.HW[t] + (i64)orb * ng : nullptr;
  const T* V = a.V[t];
  const T* wp = prev ? a.W[cur] + (i64)orb * ng : nullptr;
  const T* dVp = prev ? a.dV : nullptr;
  const T sigp = (prev || a.mode == 3) ? (T)a.sigma[cur][orb] : T(0);

  const int ntx = (nx + PTX - 1) / PTX;
  const int tx0 = (blockIdx.x % ntx) * PTX;
  const int ty0 = (blockIdx.x / ntx) * TY;
  const int z0 = (int)(((i64)blockIdx.y * nz) / a.nzc);
  const int z1 = (int)(((i64)(blockIdx.y + 1) * nz) / a.nzc);
  const int lx = threadIdx.x, ly = threadIdx.y;
  const int tid = ly * TX + lx;
  const int x = tx0 + 2 * lx, y = ty0 + ly;
  const bool act0 = (x < nx) && (y < ny);
  const bool act1 = (x + 1 < nx) && (y < ny);
  const i64 col = (i64)wrapi(y, ny) * nx + wrapi(x, nx);  // even: the pair never straddles the wrap

  // halo pair owned by this thread: 2 TY x-halo pairs, then 2 R rows of TX pairs
  int hs = -1, hrow = 0, hcol_s = 0;
  i64 hcol = 0;
  if (tid < 2 * TY) {
    const int side = tid / TY, row = tid % TY;
    hrow = row + R;
    hcol_s = side == 0 ? 0 : PTX + 2;
    hcol = (i64)wrapi(ty0 + row, ny) * nx + wrapi(side == 0 ? tx0 - 2 : tx0 + PTX, nx);
    hs = 1;
  } else if (tid < 2 * TY + 2 * R * TX) {
    const int u = tid - 2 * TY;
    const int side = u / (R * TX), r = u % (R * TX);
    const int d = r / TX, c = r % TX;
    hrow = side == 0 ? d : TY + R + d;
    hcol_s = 2 + 2 * c;
    hcol = (i64)wrapi(side == 0 ? ty0 - R + d : ty0 + TY + d, ny) * nx + wrapi(tx0 + 2 * c, nx);
    hs = 1;
  }

  const int a_first = z0 - R, a_last = z1 + R;
  // wrapped plane index of the next plane to issue, advanced incrementally
  int zi = a_first;
  int zw = wrapi(a_first, nz);
  auto issue_next = [&](int k) {  // k: compile-time stage of plane zi
    if (zi < a_last) {
      PStage<T, R>& g = ring[k];
      const i64 zo = (i64)zw * pl;
      cp_async<2 * sizeof(T)>(&g.w[ly + R][2 + 2 * lx], w + zo + col);
      if (hs >= 0) cp_async<2 * sizeof(T)>(&g.w[hrow][hcol_s], w + zo + hcol);
      if (prev) {
        cp_async<2 * sizeof(T)>(&g.p[ly + R][2 + 2 * lx], wp + zo + col);
        if (hs >= 0) cp_async<2 * sizeof(T)>(&g.p[hrow][hcol_s], wp + zo + hcol);
      }
      if (zi >= z0 && zi < z1) {
        cp_async<2 * sizeof(T)>(&g.v[ly][2 * lx], V + zo + col);
        if (prev) cp_async<2 * sizeof(T)>(&g.dv[ly][2 * lx], dVp + zo + col);
      }
    }
    cp_commit();
    ++zi;
    zw = (zw + 1 == nz) ? 0 : zw + 1;
  };

#pragma unroll
  for (int k = 0; k <= PPF; ++k) issue_next(k);

  V2 qw[2 * R + 1], qp[2 * R + 1];
#pragma unroll
  for (int j = 0; j <= 2 * R; ++j) {
    qw[j].x = qw[j].y = T(0);
    qp[j].x = qp[j].y = T(0);
  }
  T acc[NPT];
#pragma unroll
  for (int k = 0; k < NPT; ++k) acc[k] = T(0);
  Ksum<T> kww{T(0), T(0)}, kzw{T(0), T(0)}, kzz{T(0), T(0)}, kkx{T(0), T(0)}, kky{T(0), T(0)}, kkz{T(0), T(0)};
  const T ihx2 = a.ihx2, ihy2 = a.ihy2, ihz2 = a.ihz2;
  const int cx = 2 + 2 * lx, cy = ly + R;
  const i64 zpl0 = (i64)z0 * pl;

  for (int base = a_first; base < a_last; base += S) {
#pragma unroll
    for (int k = 0; k < S; ++k) {
      const int pa = base + k;
      if (pa >= a_last) break;
      cp_wait<PPF>();
      __syncthreads();
      issue_next((k + PPF + 1) % S);
      const PStage<T, R>& ga = ring[k];
#pragma unroll
      for (int j = 0; j < 2 * R; ++j) {
        qw[j] = qw[j + 1];
        qp[j] = qp[j + 1];
      }
      qw[2 * R] = *reinterpret_cast<const V2*>(&ga.w[cy][cx]);
      if (prev) qp[2 * R] = *reinterpret_cast<const V2*>(&ga.p[cy][cx]);
      const int z = pa - R;
      if (z < z0 || !act0) continue;
      const PStage<T, R>& g = ring[(k + S - R) % S];
      // pair of centres and their neighbours along x (elements cx-2 .. cx+3)
      const V2 wl = *reinterpret_cast<const V2*>(&g.w[cy][cx - 2]);
      const V2 wc = qw[R];
      const V2 wr = *reinterpret_cast<const V2*>(&g.w[cy][cx + 2]);
      const V2 wu1 = *reinterpret_cast<const V2*>(&g.w[cy - 1][cx]);
      const V2 wd1 = *reinterpret_cast<const V2*>(&g.w[cy + 1][cx]);
      const V2 vv2 = *reinterpret_cast<const V2*>(&g.v[ly][2 * lx]);
      T exa[2], eya[2], eza[2], ha[2];
      // element e of the pair: centre c, x neighbours xm1, xp1 (xm2, xp2)
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const T c = e ? wc.y : wc.x;
        const T xm1 = e ? wc.x : wl.y, xp1 = e ? wr.x : wc.y;
        const T ym1 = e ? wu1.y : wu1.x, yp1 = e ? wd1.y : wd1.x;
        const T zm1 = e ? qw[R - 1].y : qw[R - 1].x, zp1 = e ? qw[R + 1].y : qw[R + 1].x;
        const T dx1 = (xp1 - c) + (xm1 - c);
        const T dy1 = (yp1 - c) + (ym1 - c);
        const T dz1 = (zp1 - c) + (zm1 - c);
        T ex, ey, ez;
        if (R == 1) {
          ex = dx1;
          ey = dy1;
          ez = dz1;
        } else {
          const T xm2 = e ? wl.y : wl.x, xp2 = e ? wr.y : wr.x;
          const V2 wu2 = *reinterpret_cast<const V2*>(&g.w[cy - 2][cx]);
          const V2 wd2 = *reinterpret_cast<const V2*>(&g.w[cy + 2][cx]);
          const T ym2 = e ? wu2.y : wu2.x, yp2 = e ? wd2.y : wd2.x;
          const T zm2 = e ? qw[R - 2].y : qw[R - 2].x, zp2 = e ? qw[R + 2].y : qw[R + 2].x;
          ex = T(16) * dx1 - ((xp2 - c) + (xm2 - c));
          ey = T(16) * dy1 - ((yp2 - c) + (ym2 - c));
          ez = T(16) * dz1 - ((zp2 - c) + (zm2 - c));
        }
        exa[e] = ex;
        eya[e] = ey;
        eza[e] = ez;
        const T vv = e ? vv2.y : vv2.x;
        ha[e] = T(-0.5) * (ihx2 * ex + ihy2 * ey + ihz2 * ez) + vv * c;
      }
      const i64 idx = zpl0 + (i64)(z - z0) * pl + col;
      if (a.nl) {
        ha[0] += a.nl[(i64)orb * ng + idx];
        if (act1) ha[1] += a.nl[(i64)orb * ng + idx + 1];
      }
      if (hw) {
        V2 o;
        o.x = a.out_scale * ha[0];
        o.y = a.out_scale * ha[1];
        if (act1)
          *reinterpret_cast<V2*>(hw + idx) = o;
        else
          hw[idx] = o.x;
      }
      // sums over the pair (the second point counts only inside the grid)
      const T m1 = act1 ? T(1) : T(0);
      const T c0 = wc.x, c1 = wc.y * m1;
      const T zp0 = ha[0] - sigp * c0, zp1 = (ha[1] - sigp * wc.y) * m1;
      kww.add(c0 * c0 + c1 * c1);
      acc[P_HW] += ha[0] * c0 + ha[1] * c1;
      kzw.add(zp0 * c0 + zp1 * c1);
      kzz.add(zp0 * zp0 + zp1 * zp1);
      kkx.add(c0 * exa[0] + c1 * exa[1]);
      kky.add(c0 * eya[0] + c1 * eya[1]);
      kkz.add(c0 * eza[0] + c1 * eza[1]);
      if (prev) {
        const V2 pc = qp[R];
        const V2 pl2 = *reinterpret_cast<const V2*>(&g.p[cy][cx - 2]);
        const V2 pr2 = *reinterpret_cast<const V2*>(&g.p[cy][cx + 2]);
        const V2 pu1 = *reinterpret_cast<const V2*>(&g.p[cy - 1][cx]);
        const V2 pd1 = *reinterpret_cast<const V2*>(&g.p[cy + 1][cx]);
        const V2 dv2 = *reinterpret_cast<const V2*>(&g.dv[ly][2 * lx]);
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          const T me = e ? m1 : T(1);
          const T c = e ? wc.y : wc.x;
          const T sc = c - (e ? pc.y : pc.x);
          // s = w - w' at the neighbours
          const T sxm1 = e ? (wc.x - pc.x) : (wl.y - pl2.y), sxp1 = e ? (wr.x - pr2.x) : (wc.y - pc.y);
          const T sym1 = e ? (wu1.y - pu1.y) : (wu1.x - pu1.x), syp1 = e ? (wd1.y - pd1.y) : (wd1.x - pd1.x);
          const T szm1 = e ? (qw[R - 1].y - qp[R - 1].y) : (qw[R - 1].x - qp[R - 1].x);
          const T szp1 = e ? (qw[R + 1].y - qp[R + 1].y) : (qw[R + 1].x - qp[R + 1].x);
          const T sx1 = (sxp1 - sc) + (sxm1 - sc);
          const T sy1 = (syp1 - sc) + (sym1 - sc);
          const T sz1 = (szp1 - sc) + (szm1 - sc);
          T fx, fy, fz;
          if (R == 1) {
            fx = sx1;
            fy = sy1;
            fz = sz1;
          } else {
            const V2 wu2 = *reinterpret_cast<const V2*>(&g.w[cy - 2][cx]);
            const V2 wd2 = *reinterpret_cast<const V2*>(&g.w[cy + 2][cx]);
            const V2 pu2 = *reinterpret_cast<const V2*>(&g.p[cy - 2][cx]);
            const V2 pd2 = *reinterpret_cast<const V2*>(&g.p[cy + 2][cx]);
            const T sxm2 = e ? (wl.y - pl2.y) : (wl.x - pl2.x), sxp2 = e ? (wr.y - pr2.y) : (wr.x - pr2.x);
            const T sym2 = e ? (wu2.y - pu2.y) : (wu2.x - pu2.x), syp2 = e ? (wd2.y - pd2.y) : (wd2.x - pd2.x);
            const T szm2 = e ? (qw[R - 2].y - qp[R - 2].y) : (qw[R - 2].x - qp[R - 2].x);
            const T szp2 = e ? (qw[R + 2].y - qp[R + 2].y) : (qw[R + 2].x - qp[R + 2].x);
            fx = T(16) * sx1 - ((sxp2 - sc) + (sxm2 - sc));
            fy = T(16) * sy1 - ((syp2 - sc) + (sym2 - sc));
            fz = T(16) * sz1 - ((szp2 - sc) + (szm2 - sc));
          }
          const T vv = e ? vv2.y : vv2.x;
          const T dvv = e ? dv2.y : dv2.x;
          const T wpc = e ? pc.y : pc.x;
          T hsv = T(-0.5) * (ihx2 * fx + ihy2 * fy + ihz2 * fz) + vv * sc + dvv * wpc;
          if (a.nls && (e == 0 || act1)) hsv += a.nls[(i64)orb * ng + idx + e];
          const T b = (hsv - sigp * sc) * me;
          const T sm = sc * me;
          acc[P_SS] += sm * sc;
          acc[P_SB] += sm * b;
          acc[P_SW] += sm * c;
          acc[P_BB] += b * b;
          acc[P_BW] += b * c;
        }
      }
    }
  }
  cp_wait<0>();

  if (a.tilepart == nullptr) return;
  const int lane = tid & 31, warp = tid >> 5;
  double fin[NPT];
#pragma unroll
  for (int k = 0; k < NPT; ++k) fin[k] = (double)acc[k];
  fin[P_WW] = kww.value();
  fin[P_ZW] = kzw.value();
  fin[P_ZZ] = kzz.value();
  fin[P_KX] = kkx.value();
  fin[P_KY] = kky.value();
  fin[P_KZ] = kkz.value();
#pragma unroll
  for (int k = 0; k < NPT; ++k) {
    double v = fin[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[warp][k] = v;
  }
  __syncthreads();
  if (tid < NPT) {
    double v = 0.0;
#pragma unroll
    for (int wi = 0; wi < NT / 32; ++wi) v += red[wi][tid];
    const int ntile = gridDim.x * gridDim.y;
    const int tile = blockIdx.y * gridDim.x + blockIdx.x;
    a.tilepart[((i64)orb * ntile + tile) * NPT + tid] = v;
  }
}

// ----------------------------------------------------------------------------
// FP32 form with nx % 4 == 0 and 16-byte aligned blocks.  Each thread owns
// two adjacent x points (one float2 per array) for the arithmetic; the planes
// are copied in 16-byte chunks (four points), each chunk by one thread.
// Differences from the paired kernel above, each removing per-point work:
//   * the step s = w - w' is formed once per cell when its plane arrives (each
//     thread converts the chunks it copied itself, before the barrier), so the
//     s-stencil reads s directly; the (V - V') w' term is formed there too and
//     stored in the V - V' slot;
//   * the z-neighbours live in circular register queues of the ring's length,
//     indexed at compile time (the plane loop is unrolled by the ring size),
//     so the queues are never shifted;
//   * on cubic grids the three per-axis kinetic sums are one sum of
//     w (e_x + e_y + e_z) (the FP64 coefficients are then equal);
//   * the tile is 32 points x 16 rows, so grids of 32k points in x tile
//     exactly.
namespace pk {

constexpr int TXP = 16;         // threads per tile row
constexpr int TYP = 16;         // tile rows
constexpr int NTP = TXP * TYP;  // threads per CTA
constexpr int PW = 2 * TXP;     // points per tile row
constexpr int CX0 = 4;          // first centre column of a shared row
constexpr int ROW = PW + 2 * CX0;  // shared row: a 16-byte halo chunk each side
constexpr int CH = PW / 4;      // 16-byte chunks per tile row
constexpr int PFP = 2;          // planes in flight

template <int R, bool HIST, bool NLT>
struct Stage {
  float w[TYP + 2 * R][ROW];
  float s[HIST ? TYP + 2 * R : 1][ROW];  // w' on arrival, then s = w - w'
  float v[TYP][PW];
  float dv[HIST ? TYP : 1][PW];          // V - V' on arrival, then (V - V') w'
  float nl[NLT ? TYP : 1][PW];           // nonlocal part of H w (projectors)
  float nls[NLT && HIST ? TYP : 1][PW];  // ... of H s
};

// Per-lane FP32 arithmetic on the pair, each lane rounded as one scalar
// operation (no contraction across helpers).  Measured against the packed
// f32x2 instructions of sm_100+ in the same kernel: equal time and bit-equal
// results, while this form needs fewer registers (80 on cubic grids: three
// CTAs per SM).
__device__ __forceinline__ float2 add2(float2 a, float2 b) {
  return make_float2(__fadd_rn(a.x, b.x), __fadd_rn(a.y, b.y));
}
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
  return make_float2(__fsub_rn(a.x, b.x), __fsub_rn(a.y, b.y));
}
__device__ __forceinline__ float2 mul2(float2 a, float2 b) {
  return make_float2(__fmul_rn(a.x, b.x), __fmul_rn(a.y, b.y));
}
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {
  return make_float2(__fmaf_rn(a.x, b.x, c.x), __fmaf_rn(a.y, b.y, c.y));
}
__device__ __forceinline__ float2 splat(float x) { return make_float2(x, x); }
__device__ __forceinline__ float2 lds2(const float* p) { return *reinterpret_cast<const float2*>(p); }
__device__ __forceinline__ void sts2(float* p, float2 v) { *reinterpret_cast<float2*>(p) = v; }

// Compensated (Kahan) sum per lane, with the compensation kept negated so
// that the product enters through one FMA: y = a b - c, t = s + y,
// c = (t - s) - y.
struct K2 {
  float2 s, nc;
  __device__ __forceinline__ void add_prod(float2 a, float2 b) {
    const float2 y = fma2(a, b, nc);
    const float2 t = add2(s, y);
    nc = add2(sub2(s, t), y);
    s = t;
  }
  __device__ __forceinline__ double value() const {
    return ((double)s.x + (double)nc.x) + ((double)s.y + (double)nc.y);
  }
};

// Second differences of one array at the pair (no 1/h^2), for order R:
// (u[+d] - u) + (u[-d] - u); order 4 combines 16 d1 - d2.  xm2/xp2 are the
// pairs (x-2, x-1) and (x+2, x+3) of the shared row.
template <int R>
__device__ __forceinline__ void second_diffs(float2 c, float2 xm2, float2 xp2, float2 ym1, float2 yp1, float2 ym2,
                                             float2 yp2, float2 zm1, float2 zp1, float2 zm2, float2 zp2, float2& ex,
                                             float2& ey, float2& ez) {
  const float2 xm1 = make_float2(xm2.y, c.x), xp1 = make_float2(c.y, xp2.x);
  const float2 dx1 = add2(sub2(xp1, c), sub2(xm1, c));
  const float2 dy1 = add2(sub2(yp1, c), sub2(ym1, c));
  const float2 dz1 = add2(sub2(zp1, c), sub2(zm1, c));
  if (R == 1) {
    ex = dx1;
    ey = dy1;
    ez = dz1;
  } else {
    const float2 s16 = splat(16.f);
    // -(d2) formed directly, so that 16 d1 - d2 is one FMA
    const float2 ndx2 = add2(sub2(c, xp2), sub2(c, xm2));
    const float2 ndy2 = add2(sub2(c, yp2), sub2(c, ym2));
    const float2 ndz2 = add2(sub2(c, zp2), sub2(c, zm2));
    ex = fma2(s16, dx1, ndx2);
    ey = fma2(s16, dy1, ndy2);
    ez = fma2(s16, dz1, ndz2);
  }
}

template <int R, bool HIST, bool CUBIC, bool NLT>
__global__ void __launch_bounds__(NTP, (CUBIC && !NLT) ? 3 : 2) k_apply_h_pk(ApplyArgs<float> a) {
  constexpr int S = R + 2 + PFP;  // ring of planes; also the length of the register queues
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Stage<R, HIST, NLT>* ring = reinterpret_cast<Stage<R, HIST, NLT>*>(smem_raw);
  __shared__ double red[NTP / 32][NPT];

  if (a.st && a.st->done) return;
  if (a.mode == 3 && !a.st->diag_now) return;
  if (a.mode == 4 && a.st->s != 0) return;
  const int cur = a.st ? a.st->cur : 0;
  const int t = (a.mode == 2) ? 0 : ((a.mode == 3 || a.mode == 4) ? cur : 1 - cur);
  const int nx = a.nx, ny = a.ny, nz = a.nz;
  const i64 pl = (i64)nx * ny;
  const i64 ng = pl * nz;
  const int orb = blockIdx.z;
  const float* w = a.W[t] + (i64)orb * ng;
  float* hw = a.HW[t] ? a.HW[t] + (i64)orb * ng : nullptr;
  const float* V = a.V[t];
  const float* wp = HIST ? a.W[cur] + (i64)orb * ng : nullptr;
  const float* dVp = HIST ? a.dV : nullptr;
  const float* nlp = NLT ? a.nl + (i64)orb * ng : nullptr;
  const float* nlsp = (NLT && HIST) ? a.nls + (i64)orb * ng : nullptr;
  const float sigp = (HIST || a.mode == 3) ? (float)a.sigma[cur][orb] : 0.f;

  const int ntx = (nx + PW - 1) / PW;
  const int tx0 = (blockIdx.x % ntx) * PW;
  const int ty0 = (blockIdx.x / ntx) * TYP;
  const int z0 = (int)(((i64)blockIdx.y * nz) / a.nzc);
  const int z1 = (int)(((i64)(blockIdx.y + 1) * nz) / a.nzc);
  const int lx = threadIdx.x, ly = threadIdx.y;
  const int tid = ly * TXP + lx;
  const int x = tx0 + 2 * lx, y = ty0 + ly;
  const bool act = (x < nx) && (y < ny);  // nx even: the pair is inside when its first point is
  const i64 col = (i64)wrapi(y, ny) * nx + wrapi(x, nx);

  // 16-byte chunks this thread copies (nx % 4 == 0, so that a chunk of four
  // points never straddles the periodic wrap).  Threads 0 .. TYP CH - 1 own
  // a centre chunk (row cr, points 4 cc ..) of w, w', V - V' and the step's
  // nonlocal part; the others own the same chunk of V and the nonlocal part,
  // and the first 2 R CH + 2 TYP of them a halo chunk of w and w' (y halo
  // rows, then the x halos: columns tx0 - 4 .. tx0 - 1 and tx0 + 32 ..
  // tx0 + 35).  Points past the grid in a ragged tile are copied from their
  // periodic images, so that the halo after the last point is in place.
  const bool cowner = tid < TYP * CH;
  const int cu = cowner ? tid : tid - TYP * CH;
  const int cr = cu / CH, cc = cu % CH;
  const i64 ccol = (i64)wrapi(ty0 + cr, ny) * nx + wrapi(tx0 + 4 * cc, nx);
  const int csrow = cr + R, cscol = CX0 + 4 * cc;  // shared cell of the chunk in w / w'
  int hrow = -1, hcs = 0;
  i64 hcol = 0;
  if (!cowner) {
    if (cu < 2 * R * CH) {
      const int side = cu / (R * CH), r = cu % (R * CH);
      const int d = r / CH, c = r % CH;
      hrow = side == 0 ? d : TYP + R + d;
      hcs = CX0 + 4 * c;
      hcol = (i64)wrapi(side == 0 ? ty0 - R + d : ty0 + TYP + d, ny) * nx + wrapi(tx0 + 4 * c, nx);
    } else if (cu < 2 * R * CH + 2 * TYP) {
      const int u = cu - 2 * R * CH;
      const int side = u / TYP, row = u % TYP;
      hrow = row + R;
      hcs = side == 0 ? 0 : CX0 + PW;
      hcol = (i64)wrapi(ty0 + row, ny) * nx + wrapi(side == 0 ? tx0 - 4 : tx0 + PW, nx);
    }
  }
  const int cx = CX0 + 2 * lx, cy = ly + R;

  const int a_first = z0 - R, a_last = z1 + R;
  int zi = a_first;
  int zw = wrapi(a_first, nz);
  auto issue_next = [&](int k) {
    if (zi < a_last) {
      Stage<R, HIST, NLT>& g = ring[k];
      const i64 zo = (i64)zw * pl;
      const bool cen = zi >= z0 && zi < z1;
      if (cowner) {
        cp_async16_cg(&g.w[csrow][cscol], w + zo + ccol);
        if constexpr (HIST) {
          cp_async16_cg(&g.s[csrow][cscol], wp + zo + ccol);
          if (cen) cp_async16_cg(&g.dv[cr][4 * cc], dVp + zo + ccol);
          if constexpr (NLT)
            if (cen) cp_async16_cg(&g.nls[cr][4 * cc], nlsp + zo + ccol);
        }
      } else {
        if (cen) {
          cp_async16_cg(&g.v[cr][4 * cc], V + zo + ccol);
          if constexpr (NLT) cp_async16_cg(&g.nl[cr][4 * cc], nlp + zo + ccol);
        }
        if (hrow >= 0) {
          cp_async16_cg(&g.w[hrow][hcs], w + zo + hcol);
          if constexpr (HIST) cp_async16_cg(&g.s[hrow][hcs], wp + zo + hcol);
        }
      }
    }
    cp_commit();
    ++zi;
    zw = (zw + 1 == nz) ? 0 : zw + 1;
  };
#pragma unroll
  for (int k = 0; k <= PFP; ++k) issue_next(k);

  float2 qw[S], qs[S];
#pragma unroll
  for (int j = 0; j < S; ++j) qw[j] = qs[j] = splat(0.f);
  K2 kww{}, kzw{}, kzz{}, kkx{}, kky{}, kkz{};
  float2 ahw = splat(0.f), ass = splat(0.f), asb = splat(0.f), asw = splat(0.f), abb = splat(0.f),
         abw = splat(0.f);
  // -1/2 times the stencil scales, applied in FP32 to form H w (the sums use the raw differences)
  const float2 cxk = splat(-0.5f * a.ihx2), cyk = splat(-0.5f * a.ihy2), czk = splat(-0.5f * a.ihz2);
  const float2 nsig = splat(-sigp);
  const bool scale_out = a.out_scale != 1.f;
  const float2 oscale = splat(a.out_scale);
  const i64 zpl0 = (i64)z0 * pl;

  for (int base = a_first; base < a_last; base += S) {
#pragma unroll
    for (int k = 0; k < S; ++k) {
      const int pa = base + k;
      if (pa >= a_last) break;
      cp_wait<PFP>();
      Stage<R, HIST, NLT>& ga = ring[k];
      if constexpr (HIST) {
        // plane pa has landed for this thread's own copies: convert the
        // cells it copied (each pair lane by lane, as one scalar operation)
        auto conv = [&](int row, int c0) {
#pragma unroll
          for (int h = 0; h < 4; h += 2)
            sts2(&ga.s[row][c0 + h], sub2(lds2(&ga.w[row][c0 + h]), lds2(&ga.s[row][c0 + h])));
        };
        if (cowner) {
          if (pa >= z0 && pa < z1) {
#pragma unroll
            for (int h = 0; h < 4; h += 2)
              sts2(&ga.dv[cr][4 * cc + h], mul2(lds2(&ga.dv[cr][4 * cc + h]), lds2(&ga.s[csrow][cscol + h])));
          }
          conv(csrow, cscol);
        } else if (hrow >= 0) {
          conv(hrow, hcs);
        }
      }
      __syncthreads();
      // queue the centre values of plane pa (copied and converted by their owners)
      qw[k] = lds2(&ga.w[cy][cx]);
      if constexpr (HIST) qs[k] = lds2(&ga.s[cy][cx]);
      issue_next((k + PFP + 1) % S);
      const int z = pa - R;
      if (z < z0 || !act) continue;
      const int iz = (k + S - R) % S;  // queue slot and ring stage of plane z
      const Stage<R, HIST, NLT>& g = ring[iz];
      const float2 c = qw[iz];
      float2 ex, ey, ez;
      second_diffs<R>(c, lds2(&g.w[cy][cx - 2]), lds2(&g.w[cy][cx + 2]), lds2(&g.w[cy - 1][cx]),
                      lds2(&g.w[cy + 1][cx]), R == 2 ? lds2(&g.w[cy - 2][cx]) : c,
                      R == 2 ? lds2(&g.w[cy + 2][cx]) : c, qw[(iz + S - 1) % S], qw[(iz + 1) % S],
                      qw[(iz + S - 2) % S], qw[(iz + 2) % S], ex, ey, ez);
      const float2 vv = lds2(&g.v[ly][2 * lx]);
      float2 h;
      if (CUBIC) {
        const float2 e = add2(add2(ex, ey), ez);
        h = fma2(vv, c, mul2(cxk, e));
        kkx.add_prod(c, e);
      } else {
        h = fma2(vv, c, fma2(cxk, ex, fma2(cyk, ey, mul2(czk, ez))));
        kkx.add_prod(c, ex);
        kky.add_prod(c, ey);
        kkz.add_prod(c, ez);
      }
      if constexpr (NLT) h = add2(h, lds2(&g.nl[ly][2 * lx]));
      if (hw) {
        const i64 idx = zpl0 + (i64)(z - z0) * pl + col;
        *reinterpret_cast<float2*>(hw + idx) = scale_out ? mul2(oscale, h) : h;
      }
      const float2 zp = fma2(nsig, c, h);
      kww.add_prod(c, c);
      ahw = fma2(h, c, ahw);
      kzw.add_prod(zp, c);
      kzz.add_prod(zp, zp);
      if constexpr (HIST) {
        const float2 sc = qs[iz];
        float2 fx, fy, fz;
        second_diffs<R>(sc, lds2(&g.s[cy][cx - 2]), lds2(&g.s[cy][cx + 2]), lds2(&g.s[cy - 1][cx]),
                        lds2(&g.s[cy + 1][cx]), R == 2 ? lds2(&g.s[cy - 2][cx]) : sc,
                        R == 2 ? lds2(&g.s[cy + 2][cx]) : sc, qs[(iz + S - 1) % S], qs[(iz + 1) % S],
                        qs[(iz + S - 2) % S], qs[(iz + 2) % S], fx, fy, fz);
        float2 hs;
        if (CUBIC)
          hs = fma2(vv, sc, mul2(cxk, add2(add2(fx, fy), fz)));
        else
          hs = fma2(vv, sc, fma2(cxk, fx, fma2(cyk, fy, mul2(czk, fz))));
        hs = add2(hs, lds2(&g.dv[ly][2 * lx]));  // + (V - V') w'
        if constexpr (NLT) hs = add2(hs, lds2(&g.nls[ly][2 * lx]));
        const float2 b = fma2(nsig, sc, hs);      // (hw - hw') - sigma' s
        ass = fma2(sc, sc, ass);
        asb = fma2(sc, b, asb);
        asw = fma2(sc, c, asw);
        abb = fma2(b, b, abb);
        abw = fma2(b, c, abw);
      }
    }
  }
  cp_wait<0>();

  if (a.tilepart == nullptr) return;
  const int lane = tid & 31, warp = tid >> 5;
  double fin[NPT];
  auto dsum = [](float2 v) { return (double)v.x + (double)v.y; };
  fin[P_WW] = kww.value();
  fin[P_HW] = dsum(ahw);
  fin[P_ZW] = kzw.value();
  fin[P_ZZ] = kzz.value();
  fin[P_KX] = kkx.value();
  fin[P_KY] = CUBIC ? 0.0 : kky.value();
  fin[P_KZ] = CUBIC ? 0.0 : kkz.value();
  fin[P_SS] = dsum(ass);
  fin[P_SB] = dsum(asb);
  fin[P_SW] = dsum(asw);
  fin[P_BB] = dsum(abb);
  fin[P_BW] = dsum(abw);
#pragma unroll
  for (int k = 0; k < NPT; ++k) {
    double v = fin[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[warp][k] = v;
  }
  __syncthreads();
  if (tid < NPT) {
    double v = 0.0;
#pragma unroll
    for (int wi = 0; wi < NTP / 32; ++wi) v += red[wi][tid];
    const int ntile = gridDim.x * gridDim.y;
    const int tile = blockIdx.y * gridDim.x + blockIdx.x;
    a.tilepart[((i64)orb * ntile + tile) * NPT + tid] = v;
  }
}

template <int R, bool HIST, bool NLT>
size_t smem_bytes() {
  return sizeof(Stage<R, HIST, NLT>) * (size_t)(R + 2 + PFP);
}

}  // namespace pk

template <typename T, int R>
size_t apply_pair_smem() {
  return sizeof(PStage<T, R>) * (size_t)(R + 2 + PPF);
}

template <typename T, int R>
size_t apply_smem() {
  return sizeof(Stage<T, R>) * (size_t)(R + 2 + PF);
}

}  // namespace

void configure_apply_h() {
#define POU_PK_CFG(R_, H_, C_, N_)                                                                     \
  cudaFuncSetAttribute(pk::k_apply_h_pk<R_, H_, C_, N_>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                       (int)pk::smem_bytes<R_, H_, N_>())
  POU_PK_CFG(1, false, false, false);
  POU_PK_CFG(1, false, true, false);
  POU_PK_CFG(1, true, false, false);
  POU_PK_CFG(1, true, true, false);
  POU_PK_CFG(2, false, false, false);
  POU_PK_CFG(2, false, true, false);
  POU_PK_CFG(2, true, false, false);
  POU_PK_CFG(2, true, true, false);
  POU_PK_CFG(1, false, false, true);
  POU_PK_CFG(1, false, true, true);
  POU_PK_CFG(1, true, false, true);
  POU_PK_CFG(1, true, true, true);
  POU_PK_CFG(2, false, false, true);
  POU_PK_CFG(2, false, true, true);
  POU_PK_CFG(2, true, false, true);
  POU_PK_CFG(2, true, true, true);
#undef POU_PK_CFG
  cudaFuncSetAttribute(k_apply_h_pair<float, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)apply_pair_smem<float, 1>());
  cudaFuncSetAttribute(k_apply_h_pair<float, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)apply_pair_smem<float, 2>());
  cudaFuncSetAttribute(k_apply_h_pair<double, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)apply_pair_smem<double, 1>());
  cudaFuncSetAttribute(k_apply_h_pair<double, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)apply_pair_smem<double, 2>());
  cudaFuncSetAttribute(k_apply_h<float, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)apply_smem<float, 1>());
  cudaFuncSetAttribute(k_apply_h<float, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)apply_smem<float, 2>());
  cudaFuncSetAttribute(k_apply_h<double, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)apply_smem<double, 1>());
  cudaFuncSetAttribute(k_apply_h<double, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)apply_smem<double, 2>());
}

// Tile of a launch: the pk kernel for FP32 with even nx (32 x 16 points,
// 16 x 16 threads), the paired kernel for FP64 with even nx (64 x 8 points),
// the scalar kernel for odd nx (32 x 8 points).
enum TileKind { TILE_SCALAR = 0, TILE_PAIR = 1, TILE_PACKED = 2 };
struct TileShape {
  int kind, tw, th, bx, by;
};
static TileShape tile_shape(int nx, int elem_bytes, int align) {
  if (nx % 4 == 0 && elem_bytes == 4 && align >= 2) return {TILE_PACKED, pk::PW, pk::TYP, pk::TXP, pk::TYP};
  if (nx % 2 == 0 && align >= 1) return {TILE_PAIR, PTX, TY, TX, TY};
  return {TILE_SCALAR, TX, TY, TX, TY};
}

int apply_h_ntile(int nx, int ny, int nz, int N, int elem_bytes, int* nzc_out, int align) {
  const TileShape ts = tile_shape(nx, elem_bytes, align);
  const int ntx = (nx + ts.tw - 1) / ts.tw, nty = (ny + ts.th - 1) / ts.th;
  const long long base = (long long)ntx * nty * N;
  int nzc = 1;
  // enough CTAs to fill the GPU several times, with z sweeps of >= 8 planes
  while (base * nzc < 4LL * num_sms() * 8 && nz / (nzc * 2) >= 8) nzc *= 2;
  if (nzc_out) *nzc_out = nzc;
  return ntx * nty * nzc;
}

// Alignment of a launch's blocks (a caller's block need not be aligned):
// 2 when every block read starts on a 16-byte boundary and the output on a
// boundary of two elements (the FP32 kernel: 16-byte copies, pair stores);
// 1 when every block, read or written, starts on a boundary of two elements
// (the paired kernel copies and stores two elements at a time); 0 otherwise
// (the scalar kernel: one element per access).
template <typename T>
static int block_alignment(const ApplyArgs<T>& a) {
  auto on = [](const void* q, uintptr_t m) { return reinterpret_cast<uintptr_t>(q) % m == 0; };
  const void* blk[9] = {a.W[0], a.W[1], a.V[0], a.V[1], a.dV, a.nl, a.nls, a.HW[0], a.HW[1]};
  for (const void* q : blk)
    if (!on(q, 2 * sizeof(T))) return 0;
  for (int k = 0; k < 7; ++k)  // the blocks read
    if (!on(blk[k], 16)) return 1;
  return 2;
}

template <typename T>
void launch_apply_h(const ApplyArgs<T>& a0, int order, cudaStream_t s, int* ntile_out) {
  ApplyArgs<T> a = a0;
  const int align = block_alignment(a);
  int nzc = 1;
  const int ntile = apply_h_ntile(a.nx, a.ny, a.nz, a.N, (int)sizeof(T), &nzc, align);
  a.nzc = nzc;
  const TileShape ts = tile_shape(a.nx, (int)sizeof(T), align);
  const int ntx = (a.nx + ts.tw - 1) / ts.tw, nty = (a.ny + ts.th - 1) / ts.th;
  dim3 grid(ntx * nty, nzc, a.N), block(ts.bx, ts.by);
  prof_begin("apply_h", s);
  if constexpr (sizeof(T) == 4) {
    if (ts.kind == TILE_PACKED) {
      const bool hist = a.mode == 0;
      const bool cubic = a.cubic != 0;
#define POU_PK(R_, H_, C_, N_) \
  pk::k_apply_h_pk<R_, H_, C_, N_><<<grid, block, pk::smem_bytes<R_, H_, N_>(), s>>>(a)
#define POU_PK_N(R_, H_, C_)           \
  do {                                 \
    if (nlt)                           \
      POU_PK(R_, H_, C_, true);        \
    else                               \
      POU_PK(R_, H_, C_, false);       \
  } while (0)
      const bool nlt = a.nl != nullptr;
      if (order == 2) {
        if (hist) {
          if (cubic) POU_PK_N(1, true, true); else POU_PK_N(1, true, false);
        } else {
          if (cubic) POU_PK_N(1, false, true); else POU_PK_N(1, false, false);
        }
      } else {
        if (hist) {
          if (cubic) POU_PK_N(2, true, true); else POU_PK_N(2, true, false);
        } else {
          if (cubic) POU_PK_N(2, false, true); else POU_PK_N(2, false, false);
        }
      }
#undef POU_PK_N
#undef POU_PK
      prof_end(s);
      if (ntile_out) *ntile_out = ntile;
      return;
    }
  }
  if (ts.kind == TILE_PAIR) {
    if (order == 2)
      k_apply_h_pair<T, 1><<<grid, block, apply_pair_smem<T, 1>(), s>>>(a);
    else
      k_apply_h_pair<T, 2><<<grid, block, apply_pair_smem<T, 2>(), s>>>(a);
  } else if (order == 2) {
    k_apply_h<T, 1><<<grid, block, apply_smem<T, 1>(), s>>>(a);
  } else {
    k_apply_h<T, 2><<<grid, block, apply_smem<T, 2>(), s>>>(a);
  }
  prof_end(s);
  if (ntile_out) *ntile_out = ntile;
}

template void launch_apply_h<float>(const ApplyArgs<float>&, int, cudaStream_t, int*);
template void launch_apply_h<double>(const ApplyArgs<double>&, int, cudaStream_t, int*);

}  // namespace pou
