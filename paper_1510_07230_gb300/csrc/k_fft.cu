// Hartree potential by an FFT Poisson solve on the periodic grid, and the
// local potential / energy terms (Sec. 2.1, Eq. energy):
//   V_H_hat(G) = 4 pi rho_hat(G) / |G|^2,  V_H_hat(0) = 0  (neutralising background)
//   V = Vext + V_H + v_x(rho),  v_x = -(3/pi)^(1/3) rho^(1/3)
//   sums: rho*Vext, rho*V_H, eps_x(rho)*rho with eps_x = -3/4 (3/pi)^(1/3) rho^(1/3)
//
// The 3-D transform is three passes of batched 1-D transforms, one per axis,
// each staging a batch of lines in shared memory and running a mixed-radix
// (4, 2, 3, 5) self-sorting Stockham FFT there, all in FP64:
//   x-forward (reads real rho) -> y-forward -> [z-forward, Poisson scaling,
//   z-inverse in one pass] -> y-inverse -> x-inverse fused with the potential
//   and energy epilogue.
// rho and V_H are real, so only the nx/2 + 1 non-negative x frequencies are
// kept (the others are their complex conjugates): the x passes transform two
// real lines a, b as one complex line z = a + i b and separate the spectra,
//   A(k) = (Z(k) + conj Z(n-k)) / 2,  B(k) = (Z(k) - conj Z(n-k)) / (2 i),
// (and the inverse merges them back, Z = A + i B with Z(n-k) = conj A(k) +
// i conj B(k)), and the y and z passes run on nx/2 + 1 columns only.
#include "pou_internal.cuh"

#include <cmath>
#include <cstdio>
#include <vector>

namespace pou {

namespace {

constexpr int FNT = 256;
constexpr double CX = 0.98474502184269641;  // (3/pi)^(1/3)

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
// multiply by -i (forward) or +i (inverse)
__device__ __forceinline__ double2 mul_mi(double2 a, bool inv) {
  return inv ? make_double2(-a.y, a.x) : make_double2(a.y, -a.x);
}

// DFT of length r on u[] in place, exponent sign -1 (forward) or +1 (inverse).
__device__ __forceinline__ void dft_small(double2* u, int r, bool inv) {
  if (r == 2) {
    const double2 a = u[0], b = u[1];
    u[0] = cadd(a, b);
    u[1] = csub(a, b);
  } else if (r == 4) {
    const double2 s02 = cadd(u[0], u[2]), d02 = csub(u[0], u[2]);
    const double2 s13 = cadd(u[1], u[3]), d13 = mul_mi(csub(u[1], u[3]), inv);
    u[0] = cadd(s02, s13);
    u[2] = csub(s02, s13);
    u[1] = cadd(d02, d13);
    u[3] = csub(d02, d13);
  } else if (r == 3) {
    const double s3 = 0.86602540378443864676;  // sin(2 pi / 3)
    const double2 s = cadd(u[1], u[2]);
    const double2 t = make_double2(u[0].x - 0.5 * s.x, u[0].y - 0.5 * s.y);
    double2 v = csub(u[1], u[2]);
    v = mul_mi(make_double2(s3 * v.x, s3 * v.y), inv);
    u[0] = cadd(u[0], s);
    u[1] = cadd(t, v);
    u[2] = csub(t, v);
  } else {  // r == 5
    const double c1 = 0.30901699437494742410, c2 = -0.80901699437494742410;  // cos(2pi/5), cos(4pi/5)
    const double s1 = 0.95105651629515357212, s2 = 0.58778525229247312917;   // sin(2pi/5), sin(4pi/5)
    const double2 a1 = cadd(u[1], u[4]), b1 = csub(u[1], u[4]);
    const double2 a2 = cadd(u[2], u[3]), b2 = csub(u[2], u[3]);
    const double2 u0 = u[0];
    const double2 t1 = make_double2(u0.x + c1 * a1.x + c2 * a2.x, u0.y + c1 * a1.y + c2 * a2.y);
    const double2 t2 = make_double2(u0.x + c2 * a1.x + c1 * a2.x, u0.y + c2 * a1.y + c1 * a2.y);
    // forward: y1 = t1 - i (s1 b1 + s2 b2), y2 = t2 - i (s2 b1 - s1 b2)
    const double2 v1 = mul_mi(make_double2(s1 * b1.x + s2 * b2.x, s1 * b1.y + s2 * b2.y), inv);
    const double2 v2 = mul_mi(make_double2(s2 * b1.x - s1 * b2.x, s2 * b1.y - s1 * b2.y), inv);
    u[0] = make_double2(u0.x + a1.x + a2.x, u0.y + a1.y + a2.y);
    u[1] = cadd(t1, v1);
    u[4] = csub(t1, v1);
    u[2] = cadd(t2, v2);
    u[3] = csub(t2, v2);
  }
}

struct AxisDesc {
  int n, nst;
  int radix[8];
  const double2* tw;
};

// Self-sorting Stockham FFT of `nl` lines of length n stored in src (line
// stride ls), result left in the returned buffer.
__device__ double2* fft_lines(double2* src, double2* dst, int nl, int ls, const AxisDesc& ax, bool inv) {
  const int n = ax.n;
  int p = 1;
  for (int s = 0; s < ax.nst; ++s) {
    const int r = ax.radix[s];
    const int m = n / r;
    const int tstep = n / (p * r);
    for (int idx = threadIdx.x; idx < nl * m; idx += blockDim.x) {
      const int line = idx / m, i = idx % m;
      const int k = i % p;
      const double2* x = src + line * ls;
      double2* y = dst + line * ls;
      double2 u[5];
      for (int q = 0; q < r; ++q) u[q] = x[i + q * m];
      for (int q = 1; q < r; ++q) {
        double2 w = ax.tw[(q * k * tstep) % n];
        if (inv) w.y = -w.y;
        u[q] = cmul(u[q], w);
      }
      dft_small(u, r, inv);
      const int o = (i - k) * r + k;
      for (int q = 0; q < r; ++q) y[o + q * p] = u[q];
    }
    __syncthreads();
    double2* t = src;
    src = dst;
    dst = t;
    p *= r;
  }
  return src;
}

struct FftArgs {
  AxisDesc ax;
  int nx, ny, nz;
  int nxh;               // stored x frequencies: nx / 2 + 1
  int lb;
  double2* work;
  const double* rho_in;  // mode 0 source
  const double* g2x;
  const double* g2y;
  const double* g2z;
  double scale;          // 4 pi / Ng
  // potential epilogue (mode 4)
  const double* rho;
  const double* vext;
  double* V64;
  float* V32;
  double* V64out;        // (FP64 typed V when T = double)
  double* vh_out;
  double* epart;
  int hartree, exchange;
  const State* st;
  const double* rho_sel[2];
  double* V64_sel[2];
  float* V32_sel[2];
  double* Vd_sel[2];
  float* dv32;           // iteration mode: V_new - V64[cur] (working type float)
  double* dv64;          // (working type double)
};

// MODE: 0 x-forward from real rho, 1 y-forward, 2 z-forward+scale+inverse,
// 3 y-inverse, 4 x-inverse + potential epilogue.
template <int MODE>
__global__ void __launch_bounds__(FNT) k_fft(FftArgs a) {
  extern __shared__ double2 sm[];
  if (a.st && a.st->done) return;
  const int n = a.ax.n;
  const int ls = n + 1;
  const int lb = a.lb;
  double2* b0 = sm;
  double2* b1 = sm + lb * ls;
  const int nx = a.nx, ny = a.ny, nz = a.nz, nxh = a.nxh;
  const i64 plh = (i64)nxh * ny;  // one z plane of the half spectrum
  const bool xaxis = (MODE == 0 || MODE == 4);
  // line geometry: x passes take nl real lines (rows r0 .. r0 + nl) as
  // np = ceil(nl / 2) complex lines; y and z passes take nl columns of the
  // half spectrum
  i64 base = 0;  // offset of element 0 of line 0 (y, z passes)
  i64 estr = 0;  // element stride (y, z passes)
  int nl;        // lines in this block
  int r0 = 0, x0 = 0, yz = 0;
  if (xaxis) {
    r0 = blockIdx.x * lb;
    nl = min(lb, nz * ny - r0);
  } else {
    const int nxb = (nxh + lb - 1) / lb;
    x0 = (blockIdx.x % nxb) * lb;
    yz = blockIdx.x / nxb;  // z for the y-axis pass, y for the z-axis pass
    nl = min(lb, nxh - x0);
    base = (MODE == 2) ? (i64)yz * nxh + x0 : (i64)yz * plh + x0;
    estr = (MODE == 2) ? plh : nxh;
  }
  const int ncl = xaxis ? (nl + 1) / 2 : nl;  // complex lines transformed
  const double* rho_src = a.rho_in;
  if (MODE == 0 && a.st) rho_src = a.rho_sel[1 - a.st->cur];

  // load
  if (MODE == 0) {
    for (int idx = threadIdx.x; idx < ncl * n; idx += blockDim.x) {
      const int c = idx / n, e = idx % n;
      const int la = 2 * c, lbb = 2 * c + 1;
      const double va = rho_src[(i64)(r0 + la) * nx + e];
      const double vb = lbb < nl ? rho_src[(i64)(r0 + lbb) * nx + e] : 0.0;
      b0[c * ls + e] = make_double2(va, vb);
    }
  } else if (MODE == 4) {
    for (int idx = threadIdx.x; idx < ncl * n; idx += blockDim.x) {
      const int c = idx / n, k = idx % n;
      const int la = 2 * c, lbb = 2 * c + 1;
      const bool lo = k < nxh;
      const int kk = lo ? k : n - k;
      double2 fa = a.work[(i64)(r0 + la) * nxh + kk];
      double2 fb = lbb < nl ? a.work[(i64)(r0 + lbb) * nxh + kk] : make_double2(0.0, 0.0);
      if (!lo) {
        fa.y = -fa.y;
        fb.y = -fb.y;
      }
      b0[c * ls + k] = make_double2(fa.x - fb.y, fa.y + fb.x);  // A + i B
    }
  } else {
    for (int idx = threadIdx.x; idx < nl * n; idx += blockDim.x) {
      const int line = idx % nl, e = idx / nl;
      b0[line * ls + e] = a.work[base + (i64)e * estr + line];
    }
  }
  __syncthreads();
  const bool inv = (MODE >= 3);
  double2* res = fft_lines(b0, b1, ncl, ls, a.ax, inv);
  if (MODE == 2) {
    // Poisson kernel 4 pi / |G|^2 (and 1 / Ng of the inverse), G = 0 -> 0
    const int y = yz;
    for (int idx = threadIdx.x; idx < nl * n; idx += blockDim.x) {
      const int line = idx / n, z = idx % n;
      const double g2 = a.g2x[x0 + line] + a.g2y[y] + a.g2z[z];
      const double f = g2 > 0.0 ? a.scale / g2 : 0.0;
      double2 v = res[line * ls + z];
      res[line * ls + z] = make_double2(v.x * f, v.y * f);
    }
    __syncthreads();
    double2* other = (res == b0) ? b1 : b0;
    res = fft_lines(res, other, nl, ls, a.ax, true);
  }
  if (MODE == 0) {
    // separate the spectra of the two real lines, keep k = 0 .. nxh - 1
    for (int idx = threadIdx.x; idx < ncl * nxh; idx += blockDim.x) {
      const int c = idx / nxh, k = idx % nxh;
      const int la = 2 * c, lbb = 2 * c + 1;
      const double2 zk = res[c * ls + k];
      const double2 zn = res[c * ls + (k == 0 ? 0 : n - k)];
      // A = (Z(k) + conj Z(n-k)) / 2,  B = -i (Z(k) - conj Z(n-k)) / 2
      a.work[(i64)(r0 + la) * nxh + k] = make_double2(0.5 * (zk.x + zn.x), 0.5 * (zk.y - zn.y));
      if (lbb < nl) a.work[(i64)(r0 + lbb) * nxh + k] = make_double2(0.5 * (zk.y + zn.y), -0.5 * (zk.x - zn.x));
    }
    return;
  }
  if (MODE != 4) {
    for (int idx = threadIdx.x; idx < nl * n; idx += blockDim.x) {
      const int line = idx % nl, e = idx / nl;
      a.work[base + (i64)e * estr + line] = res[line * ls + e];
    }
    return;
  }
  // MODE 4: potential epilogue on rows r0 .. r0 + nl
  const double* rho = a.rho;
  double* V64 = a.V64;
  float* V32 = a.V32;
  if (a.st) {
    const int t = 1 - a.st->cur;
    rho = a.rho_sel[t];
    V64 = a.V64_sel[t];
    V32 = a.V32_sel[t];
  }
  double s_ext = 0.0, s_h = 0.0, s_x = 0.0;
  for (int idx = threadIdx.x; idx < nl * n; idx += blockDim.x) {
    const int line = idx / n, e = idx % n;
    const i64 g = (i64)(r0 + line) * nx + e;
    const double2 zv = res[(line >> 1) * ls + e];
    const double vh = (line & 1) ? zv.y : zv.x;
    if (a.vh_out) {
      a.vh_out[g] = vh;
      continue;
    }
    const double r = rho[g];
    double vx = 0.0, ex = 0.0;
    if (a.exchange) {
      const double c = cbrt(r);
      vx = -CX * c;
      ex = -0.75 * CX * c * r;
    }
    const double ve = a.vext[g];
    const double V = ve + (a.hartree ? vh : 0.0) + vx;
    V64[g] = V;
    if (V32) V32[g] = (float)V;
    if (a.st) {
      const double d = V - a.V64_sel[a.st->cur][g];
      if (a.dv32) a.dv32[g] = (float)d;
      if (a.dv64) a.dv64[g] = d;
    }
    s_ext += r * ve;
    s_h += r * vh;
    s_x += ex;
  }
  if (a.vh_out || a.epart == nullptr) return;
  __shared__ double red[FNT / 32][NE];
  for (int o = 16; o > 0; o >>= 1) {
    s_ext += __shfl_xor_sync(0xffffffffu, s_ext, o);
    s_h += __shfl_xor_sync(0xffffffffu, s_h, o);
    s_x += __shfl_xor_sync(0xffffffffu, s_x, o);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
    red[warp][E_EXT] = s_ext;
    red[warp][E_H] = s_h;
    red[warp][E_X] = s_x;
  }
  __syncthreads();
  if (threadIdx.x < NE) {
    double v = 0.0;
    for (int w = 0; w < FNT / 32; ++w) v += red[w][threadIdx.x];
    a.epart[(i64)blockIdx.x * NE + threadIdx.x] = v;
  }
}

// Potential without the Hartree term (hartree = 0): V = Vext + v_x.
template <typename T>
__global__ void __launch_bounds__(FNT) k_potential_local(FftArgs a, i64 ng) {
  if (a.st && a.st->done) return;
  const double* rho = a.rho;
  double* V64 = a.V64;
  float* V32 = a.V32;
  if (a.st) {
    const int t = 1 - a.st->cur;
    rho = a.rho_sel[t];
    V64 = a.V64_sel[t];
    V32 = a.V32_sel[t];
  }
  double s_ext = 0.0, s_x = 0.0;
  for (i64 g = (i64)blockIdx.x * blockDim.x + threadIdx.x; g < ng; g += (i64)gridDim.x * blockDim.x) {
    const double r = rho[g];
    double vx = 0.0, ex = 0.0;
    if (a.exchange) {
      const double c = cbrt(r);
      vx = -CX * c;
      ex = -0.75 * CX * c * r;
    }
    const double ve = a.vext[g];
    const double V = ve + vx;
    V64[g] = V;
    if (V32) V32[g] = (float)V;
    if (a.st) {
      const double d = V - a.V64_sel[a.st->cur][g];
      if (a.dv32) a.dv32[g] = (float)d;
      if (a.dv64) a.dv64[g] = d;
    }
    s_ext += r * ve;
    s_x += ex;
  }
  __shared__ double red[FNT / 32][2];
  for (int o = 16; o > 0; o >>= 1) {
    s_ext += __shfl_xor_sync(0xffffffffu, s_ext, o);
    s_x += __shfl_xor_sync(0xffffffffu, s_x, o);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
    red[warp][0] = s_ext;
    red[warp][1] = s_x;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double e = 0.0, x = 0.0;
    for (int w = 0; w < FNT / 32; ++w) {
      e += red[w][0];
      x += red[w][1];
    }
    a.epart[(i64)blockIdx.x * NE + E_EXT] = e;
    a.epart[(i64)blockIdx.x * NE + E_H] = 0.0;
    a.epart[(i64)blockIdx.x * NE + E_X] = x;
  }
}

int factorize(int n, int* radix) {
  int k = 0;
  while (n % 4 == 0) { radix[k++] = 4; n /= 4; }
  while (n % 2 == 0) { radix[k++] = 2; n /= 2; }
  while (n % 3 == 0) { radix[k++] = 3; n /= 3; }
  while (n % 5 == 0) { radix[k++] = 5; n /= 5; }
  if (n != 1 || k > 8) return -1;
  return k;
}

template <int MODE>
void launch_axis(const FftPlan& p, int axis, FftArgs a, int grid, cudaStream_t s) {
  a.ax.n = p.n[axis];
  a.ax.nst = p.nst[axis];
  for (int i = 0; i < 8; ++i) a.ax.radix[i] = p.radix[axis][i];
  a.ax.tw = p.tw[axis];
  a.lb = p.lb[axis];
  const size_t smem = sizeof(double2) * 2 * (size_t)a.lb * (a.ax.n + 1);
  static const char* names[5] = {"fft_x_fwd", "fft_y_fwd", "fft_z_poisson", "fft_y_inv", "fft_x_inv_potential"};
  prof_begin(names[MODE], s);
  k_fft<MODE><<<grid, FNT, smem, s>>>(a);
  prof_end(s);
}

}  // namespace

void configure_fft() {
  cudaFuncSetAttribute(k_fft<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  cudaFuncSetAttribute(k_fft<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  cudaFuncSetAttribute(k_fft<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  cudaFuncSetAttribute(k_fft<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  cudaFuncSetAttribute(k_fft<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
}

bool fft_supported(int n) {
  int r[16];
  return n >= 1 && factorize(n, r) >= 0;
}

int fft_plan_create(FftPlan* p, const int n[3], const double L[3]) {
  size_t total = 0;
  for (int a = 0; a < 3; ++a) {
    p->n[a] = n[a];
    p->nst[a] = factorize(n[a], p->radix[a]);
    if (p->nst[a] < 0) return -1;
    // per axis: n complex twiddles (2n doubles) then n values of g^2, each
    // table starting on a 16-byte boundary (twiddles are read as double2)
    total += 2 * (size_t)n[a] + (((size_t)n[a] + 1) & ~(size_t)1);
    // lines per block: keep two buffers within ~96 KB
    int lb = 16;
    while (lb > 1 && 2 * (size_t)lb * (n[a] + 1) * sizeof(double2) > 96 * 1024) lb /= 2;
    p->lb[a] = lb;
  }
  std::vector<double> host(total);
  size_t off = 0;
  size_t offs_tw[3], offs_g[3];
  for (int a = 0; a < 3; ++a) {
    offs_tw[a] = off;
    for (int k = 0; k < n[a]; ++k) {
      const double ang = -2.0 * M_PI * (double)k / (double)n[a];
      host[off + 2 * k] = cos(ang);
      host[off + 2 * k + 1] = sin(ang);
    }
    off += 2 * (size_t)n[a];
    offs_g[a] = off;
    for (int k = 0; k < n[a]; ++k) {
      const int m = (k <= n[a] / 2) ? k : k - n[a];
      const double g = 2.0 * M_PI * (double)m / L[a];
      host[off + k] = g * g;
    }
    off += ((size_t)n[a] + 1) & ~(size_t)1;
  }
  for (int a = 0; a < 3; ++a)
    if (offs_tw[a] % 2 != 0) return -4;  // a double2 table must be 16-byte aligned
  if (cudaMalloc(&p->mem, total * sizeof(double)) != cudaSuccess) return -2;
  if (cudaMemcpy(p->mem, host.data(), total * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess)
    return -3;
  for (int a = 0; a < 3; ++a) {
    p->tw[a] = reinterpret_cast<double2*>(p->mem + offs_tw[a]);
    p->g2[a] = p->mem + offs_g[a];
  }
  return 0;
}

void fft_plan_destroy(FftPlan* p) {
  if (p->mem) cudaFree(p->mem);
  p->mem = nullptr;
}

template <typename T>
int launch_potential(const FftPlan& p, const PotArgs<T>& pa, cudaStream_t s) {
  const int nx = p.n[0], ny = p.n[1], nz = p.n[2];
  const i64 ng = (i64)nx * ny * nz;
  FftArgs a{};
  a.nx = nx;
  a.ny = ny;
  a.nz = nz;
  a.nxh = nx / 2 + 1;
  a.work = pa.work;
  a.rho_in = pa.rho_x;
  a.g2x = p.g2[0];
  a.g2y = p.g2[1];
  a.g2z = p.g2[2];
  a.scale = 4.0 * M_PI / (double)ng;
  a.rho = pa.rho_x;
  a.vext = pa.vext;
  a.vh_out = pa.vh_out;
  a.epart = pa.epart;
  a.hartree = pa.hartree;
  a.exchange = pa.exchange;
  a.st = pa.st;
  for (int t = 0; t < 2; ++t) {
    a.rho_sel[t] = pa.rho[t];
    a.V64_sel[t] = pa.V64[t];
    a.V32_sel[t] = (sizeof(T) == 4) ? reinterpret_cast<float*>(pa.V[t]) : nullptr;
  }
  a.V64 = pa.V64_x;
  a.V32 = (sizeof(T) == 4) ? reinterpret_cast<float*>(pa.V_x) : nullptr;
  // when T = double the FP64 potential is the working potential
  if (sizeof(T) == 8) {
    for (int t = 0; t < 2; ++t)
      if (pa.V[t]) a.V64_sel[t] = reinterpret_cast<double*>(pa.V[t]);
    if (pa.V_x) a.V64 = reinterpret_cast<double*>(pa.V_x);
    a.dv64 = reinterpret_cast<double*>(pa.dv_out);
  } else {
    a.dv32 = reinterpret_cast<float*>(pa.dv_out);
  }
  if (!pa.hartree && !pa.vh_out) {
    const int nblk = num_sms() * 4;
    prof_begin("potential_local", s);
    k_potential_local<T><<<nblk, FNT, 0, s>>>(a, ng);
    prof_end(s);
    return nblk;
  }
  const int lbx = p.lb[0], lby = p.lb[1], lbz = p.lb[2];
  const int gx = (nz * ny + lbx - 1) / lbx;
  const int nxh = nx / 2 + 1;
  const int gy = ((nxh + lby - 1) / lby) * nz;
  const int gz = ((nxh + lbz - 1) / lbz) * ny;
  launch_axis<0>(p, 0, a, gx, s);
  launch_axis<1>(p, 1, a, gy, s);
  launch_axis<2>(p, 2, a, gz, s);
  launch_axis<3>(p, 1, a, gy, s);
  launch_axis<4>(p, 0, a, gx, s);
  return gx;
}
template int launch_potential<float>(const FftPlan&, const PotArgs<float>&, cudaStream_t);
template int launch_potential<double>(const FftPlan&, const PotArgs<double>&, cudaStream_t);

}  // namespace pou
