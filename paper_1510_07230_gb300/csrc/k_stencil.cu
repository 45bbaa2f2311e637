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
  const int cur = a.st ? a.st->cur : 0;
  const int t = (a.mode == 2) ? 0 : (a.mode == 3 ? cur : 1 - cur);
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
    const T h = kin + vv * c;
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
      const T hs = T(-0.5) * (ihx2 * fx + ihy2 * fy + ihz2 * fz) + vv * sc + dvv * qp[R];
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
  const int cur = a.st ? a.st->cur : 0;
  const int t = (a.mode == 2) ? 0 : (a.mode == 3 ? cur : 1 - cur);
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
          const T hsv = T(-0.5) * (ihx2 * fx + ihy2 * fy + ihz2 * fz) + vv * sc + dvv * wpc;
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

// tile width in x: paired kernel (two points per thread) for even nx
static int tile_w(int nx) { return (nx % 2 == 0) ? PTX : TX; }

int apply_h_ntile(int nx, int ny, int nz, int N, int* nzc_out) {
  const int ntx = (nx + tile_w(nx) - 1) / tile_w(nx), nty = (ny + TY - 1) / TY;
  const long long base = (long long)ntx * nty * N;
  int nzc = 1;
  // enough CTAs to fill the GPU several times, with z sweeps of >= 8 planes
  while (base * nzc < 4LL * num_sms() * 8 && nz / (nzc * 2) >= 8) nzc *= 2;
  if (nzc_out) *nzc_out = nzc;
  return ntx * nty * nzc;
}

template <typename T>
void launch_apply_h(const ApplyArgs<T>& a0, int order, cudaStream_t s, int* ntile_out) {
  ApplyArgs<T> a = a0;
  int nzc = 1;
  const int ntile = apply_h_ntile(a.nx, a.ny, a.nz, a.N, &nzc);
  a.nzc = nzc;
  const int tw = tile_w(a.nx);
  const int ntx = (a.nx + tw - 1) / tw, nty = (a.ny + TY - 1) / TY;
  dim3 grid(ntx * nty, nzc, a.N), block(TX, TY);
  prof_begin("apply_h", s);
  if (tw == PTX) {
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
