// Nonlocal part of the pseudopotential (Sec. 2.1): V_nloc u = sum_p <xi_p, u> xi_p.
// The projectors are Gaussians in product form, xi_p(x, y, z) =
// gx_p[x] gy_p[y] gz_p[z] (the amplitude folded into gx_p; each per-axis
// table sums the 27 nearest periodic images), with a window per axis outside
// which a table is below 1e-14 of its largest value.
//
// k_nl_project + k_nl_reduce: C_ip = dV sum_r xi_p(r) x_i(r).  One CTA per
//   (orbital, z plane, 32 rows) stages the rows and, for every projector
//   whose windows meet them, the row weights gy; one warp per projector forms
//   the column sums sum_y gy[y] x[y][x] over its x window (lanes over x, so
//   that the staged rows are read without bank conflicts), weighted by gx and
//   reduced over the lanes in FP64; a second kernel weights the planes by gz
//   and sums them in a fixed order.
// k_nl_apply: NL_i(r) = sum_p xi_p(r) C_ip and, for a trial block, the
//   nonlocal part of H applied to the step, NLS_i(r) = sum_p xi_p(r)
//   (C_ip - C'_ip) with the current iterate's C' (its two terms are then
//   formed from the step, like the local part).  One CTA per (orbital, 32 x
//   32 tile, run of NL_PLANES z planes): the projectors whose x and y windows
//   meet the tile are listed once in a fixed order (ballot and prefix counts)
//   with their column tables gx and row coefficients gy C, gy (C - C')
//   staged; on each plane their gz (zero outside the z window) is staged and
//   every thread forms 4 columns of one row.
// The H-apply adds NL to H w and NLS to H s; the controller adds the
// nonlocal energy f sum C_ip^2 to the external term.
#include "pou_internal.cuh"

namespace pou {

namespace {

constexpr int PNT = 256;
constexpr int PROWS = 32;  // rows of a projection block
constexpr int ATX = 32;    // apply tile: columns (4 per thread)
constexpr int ATY = PNT / (ATX / 4);  // apply tile: rows (32)
constexpr int NL_PLANES = 8;          // apply: z planes per CTA

template <typename T>
__device__ __forceinline__ const T* tab_x(const NlTables& t, int p);
template <>
__device__ __forceinline__ const double* tab_x<double>(const NlTables& t, int p) {
  return t.gx + (i64)p * t.nx;
}
template <>
__device__ __forceinline__ const float* tab_x<float>(const NlTables& t, int p) {
  return t.gxf + (i64)p * t.nx;
}
template <typename T>
__device__ __forceinline__ T tab_y(const NlTables& t, int p, int y) {
  return sizeof(T) == 8 ? (T)t.gy[(i64)p * t.ny + y] : (T)t.gyf[(i64)p * t.ny + y];
}
template <typename T>
__device__ __forceinline__ T tab_z(const NlTables& t, int p, int z) {
  return sizeof(T) == 8 ? (T)t.gz[(i64)p * t.nz + z] : (T)t.gzf[(i64)p * t.nz + z];
}

template <typename T>
__device__ __forceinline__ int nl_slot(const NlArgs<T>& a) {
  if (a.sel == 0) return 0;
  const int cur = a.st->cur;
  return a.sel == 1 ? 1 - cur : cur;
}

// Window test on one axis: does [a, a + len) meet the window [w0, w0 + wl)
// (all modulo n)?
__device__ __forceinline__ bool meets(int a, int len, int w0, int wl, int n) {
  if (wl >= n) return true;
  const int d = (a - w0 + n) % n;
  return d < wl || d + len > n;
}

// Projectors of one tile (plane z, rows [y0, y0 + ry), columns [x0, x0 + rx);
// z < 0: any plane), listed in index order (ballot and prefix counts).
// Returns the count.
__device__ __forceinline__ int list_tile(const NlTables& t, int z, int y0, int ry, int x0, int rx, int* list,
                                         int* wcount) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  bool take = false;
  if (tid < t.P) {
    const int* w = t.win + tid * 6;
    take = (z < 0 || meets(z, 1, w[4], w[5], t.nz)) && meets(y0, ry, w[2], w[3], t.ny) &&
           meets(x0, rx, w[0], w[1], t.nx);
  }
  const unsigned m = __ballot_sync(0xffffffffu, take);
  if (lane == 0) wcount[warp] = __popc(m);
  __syncthreads();
  int off = 0, cnt = 0;
  for (int k = 0; k < PNT / 32; ++k) {
    if (k < warp) off += wcount[k];
    cnt += wcount[k];
  }
  if (take) list[off + __popc(m & ((1u << lane) - 1u))] = tid;
  __syncthreads();
  return cnt;
}

// Projections, first stage: for one plane and PROWS rows of one orbital,
// sum_x gx_p[x] sum_y gy_p[y] w[y][x] for every projector (zero for those not
// listed), into part[i][z][row block][p].
template <typename T>
__global__ void __launch_bounds__(PNT) k_nl_project(NlArgs<T> a, double* part) {
  if (a.st && (a.st->done || !gate_open(a.st, a.gate))) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const NlTables& t = a.tab;
  const int nx = t.nx, ny = t.ny, nz = t.nz, P = t.P;
  T* ws = reinterpret_cast<T*>(smem_raw);                 // [PROWS][nx]
  T* gys = ws + (size_t)PROWS * nx;                        // [P][PROWS] gy of the listed projectors
  double* res = reinterpret_cast<double*>(gys + (size_t)P * PROWS);  // [P]
  int* list = reinterpret_cast<int*>(res + P);
  __shared__ int wcount[PNT / 32];
  const int nyb = (ny + PROWS - 1) / PROWS;
  const int yb = blockIdx.x, z = blockIdx.y, i = blockIdx.z;
  const int y0 = yb * PROWS, ry = min(PROWS, ny - y0);
  const int slot = nl_slot(a);
  const T* x = a.X[slot] + (i64)i * nx * ny * nz + (i64)z * nx * ny + (i64)y0 * nx;
  for (int e = threadIdx.x; e < ry * nx; e += PNT) ws[e] = x[e];
  for (int p = threadIdx.x; p < P; p += PNT) res[p] = 0.0;
  const int cnt = list_tile(t, z, y0, ry, 0, nx, list, wcount);
  for (int e = threadIdx.x; e < cnt * PROWS; e += PNT) {
    const int k = e / PROWS, r = e - k * PROWS;
    gys[e] = r < ry ? tab_y<T>(t, list[k], y0 + r) : T(0);
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int k = warp; k < cnt; k += PNT / 32) {
    const int p = list[k];
    const int* w = t.win + p * 6;
    const int w0 = w[0], wl = w[1];
    const T* gxp = tab_x<T>(t, p);
    const T* gyk = gys + k * PROWS;
    T acc = T(0);
    for (int j = lane; j < wl; j += 32) {
      int xx = w0 + j;
      if (xx >= nx) xx -= nx;
      T col = T(0);
      for (int r = 0; r < ry; ++r) col += gyk[r] * ws[r * nx + xx];
      acc += gxp[xx] * col;
    }
    double v = (double)acc;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) res[p] = v;
  }
  __syncthreads();
  double* out = part + (((i64)i * nz + z) * nyb + yb) * P;
  for (int p = threadIdx.x; p < P; p += PNT) out[p] = res[p];
}

// Projections, second stage: C_ip = dV sum_z gz_p[z] sum_blocks part, in a fixed order.
template <typename T>
__global__ void __launch_bounds__(PNT) k_nl_reduce(NlArgs<T> a, const double* part) {
  if (a.st && (a.st->done || !gate_open(a.st, a.gate))) return;
  const NlTables& t = a.tab;
  const int i = blockIdx.x, P = t.P, nz = t.nz;
  const int nyb = (t.ny + PROWS - 1) / PROWS;
  const int slot = nl_slot(a);
  for (int p = threadIdx.x; p < P; p += PNT) {
    double c = 0.0;
    for (int z = 0; z < nz; ++z) {
      double sz = 0.0;
      for (int b = 0; b < nyb; ++b) sz += part[(((i64)i * nz + z) * nyb + b) * P + p];
      c += t.gz[(i64)p * nz + z] * sz;
    }
    a.C[slot][(i64)i * P + p] = a.dV * c;
  }
}

// NL_i = sum_p xi_p C_ip (and NLS_i with C - C') on a tile of ATY rows x ATX
// columns for a run of planes: the projectors whose x and y windows meet the
// tile are listed once, with their column tables gx and row coefficients
// gy C (and gy (C - C')) staged; on each plane their gz (zero outside the z
// window) is staged and each thread forms 4 columns of one row, in list
// order.
template <typename T>
__global__ void __launch_bounds__(PNT) k_nl_apply(NlArgs<T> a) {
  if (a.st && (a.st->done || !gate_open(a.st, a.gate))) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const NlTables& t = a.tab;
  const int nx = t.nx, ny = t.ny, nz = t.nz, P = t.P;
  T* gxs = reinterpret_cast<T*>(smem_raw);  // [P][ATX]
  T* q = gxs + (size_t)P * ATX;              // [P][ATY]: gy C
  T* qs = q + (size_t)P * ATY;               // [P][ATY]: gy (C - C')
  T* gzs = qs + (size_t)P * ATY;             // [P]: gz of the plane
  int* list = reinterpret_cast<int*>(gzs + P);
  __shared__ int wcount[PNT / 32];
  const int ntx = (nx + ATX - 1) / ATX;
  const int x0 = (blockIdx.x % ntx) * ATX, y0 = (blockIdx.x / ntx) * ATY;
  const int za = blockIdx.y * NL_PLANES, zb = min(nz, za + NL_PLANES);
  const int i = blockIdx.z;
  const int rx = min(ATX, nx - x0), ry = min(ATY, ny - y0);
  const int slot = nl_slot(a);
  const double* C = a.C[slot] + (i64)i * P;
  const double* Cp = a.nls ? a.C[a.st->cur] + (i64)i * P : nullptr;  // the trial's previous iterate
  // projectors meeting the tile in x and y (the z window is applied per plane)
  const int cnt = list_tile(t, -1, y0, ry, x0, rx, list, wcount);
  for (int e = threadIdx.x; e < cnt * ATX; e += PNT) {
    const int k = e / ATX, c = e - k * ATX;
    gxs[e] = c < rx ? tab_x<T>(t, list[k])[x0 + c] : T(0);
  }
  for (int e = threadIdx.x; e < cnt * ATY; e += PNT) {
    const int k = e / ATY, r = e - k * ATY;
    const int p = list[k];
    const T gy = r < ry ? tab_y<T>(t, p, y0 + r) : T(0);
    q[e] = gy * (T)C[p];
    qs[e] = Cp ? gy * (T)(C[p] - Cp[p]) : T(0);
  }
  const int tx = threadIdx.x % (ATX / 4), r = threadIdx.x / (ATX / 4);
  for (int z = za; z < zb; ++z) {
    if ((int)threadIdx.x < cnt) {
      const int p = list[threadIdx.x];
      const int* w = t.win + p * 6;
      gzs[threadIdx.x] = meets(z, 1, w[4], w[5], nz) ? tab_z<T>(t, p, z) : T(0);
    }
    __syncthreads();
    T v[4] = {0, 0, 0, 0}, vs[4] = {0, 0, 0, 0};
    for (int k = 0; k < cnt; ++k) {
      const T gz = gzs[k];
      if (gz == T(0)) continue;  // outside the z window: uniform over the CTA
      const T qk = q[k * ATY + r] * gz, qsk = qs[k * ATY + r] * gz;
      const T* g = gxs + k * ATX + 4 * tx;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        v[j] += g[j] * qk;
        vs[j] += g[j] * qsk;
      }
    }
    if (r < ry) {
      const i64 o = (i64)i * nx * ny * nz + (i64)z * nx * ny + (i64)(y0 + r) * nx + x0 + 4 * tx;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        if (4 * tx + j < rx) {
          a.nl[o + j] = v[j];
          if (a.nls) a.nls[o + j] = vs[j];
        }
      }
    }
    __syncthreads();  // gzs is restaged for the next plane
  }
}

template <typename T>
size_t nl_apply_smem(int P) {
  return (size_t)P * (ATX + 2 * ATY + 1) * sizeof(T) + (size_t)P * sizeof(int);
}
template <typename T>
size_t nl_project_smem(int P, int nx) {
  return (size_t)(PROWS * nx + P * PROWS) * sizeof(T) + (size_t)P * (sizeof(double) + sizeof(int));
}

}  // namespace

template <typename T>
void launch_nl_project(const NlArgs<T>& a, double* part, cudaStream_t s) {
  const int nyb = (a.tab.ny + PROWS - 1) / PROWS;
  prof_begin("nl_project", s);
  k_nl_project<T><<<dim3(nyb, a.tab.nz, a.N), PNT, nl_project_smem<T>(a.tab.P, a.tab.nx), s>>>(a, part);
  prof_end(s);
  prof_begin("nl_reduce", s);
  k_nl_reduce<T><<<a.N, PNT, 0, s>>>(a, part);
  prof_end(s);
}
template <typename T>
void launch_nl_apply(const NlArgs<T>& a, cudaStream_t s) {
  const int tiles = ((a.tab.nx + ATX - 1) / ATX) * ((a.tab.ny + ATY - 1) / ATY);
  prof_begin("nl_apply", s);
  const int runs = (a.tab.nz + NL_PLANES - 1) / NL_PLANES;
  k_nl_apply<T><<<dim3(tiles, runs, a.N), PNT, nl_apply_smem<T>(a.tab.P), s>>>(a);
  prof_end(s);
}

size_t nl_part_bytes(int N, int P, const int n[3]) {
  return sizeof(double) * (size_t)N * n[2] * ((n[1] + PROWS - 1) / PROWS) * P;
}

void configure_nonlocal() {
  cudaFuncSetAttribute(k_nl_apply<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)nl_apply_smem<float>(kMaxProj));
  cudaFuncSetAttribute(k_nl_apply<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)nl_apply_smem<double>(kMaxProj));
  cudaFuncSetAttribute(k_nl_project<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)nl_project_smem<float>(kMaxProj, kMaxProjGrid));
  cudaFuncSetAttribute(k_nl_project<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)nl_project_smem<double>(kMaxProj, kMaxProjGrid));
}

template void launch_nl_project<float>(const NlArgs<float>&, double*, cudaStream_t);
template void launch_nl_project<double>(const NlArgs<double>&, double*, cudaStream_t);
template void launch_nl_apply<float>(const NlArgs<float>&, cudaStream_t);
template void launch_nl_apply<double>(const NlArgs<double>&, cudaStream_t);

}  // namespace pou
