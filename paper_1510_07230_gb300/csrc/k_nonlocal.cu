// Nonlocal part of the pseudopotential (Sec. 2.1): V_nloc u = sum_p <xi_p, u> xi_p.
// The projectors are Gaussians in product form, xi_p(x, y, z) =
// gx_p[x] gy_p[y] gz_p[z] (the amplitude folded into gx_p; each per-axis
// table sums the 27 nearest periodic images), with a window per axis outside
// which a table is below 1e-14 of its largest value.
//
// k_nl_project: C_ip = dV sum_r xi_p(r) x_i(r) over the window box of
//   projector p, one CTA per (projector, orbital): 32 threads along each
//   window row, row sums weighted by gy, plane sums weighted by gz and
//   promoted to FP64 once per plane.
// k_nl_apply: NL_i(r) = sum_p xi_p(r) C_ip and, for a trial block, the
//   nonlocal part of H applied to the step, NLS_i(r) = sum_p xi_p(r)
//   (C_ip - C'_ip) with the current iterate's C' (its two terms are then
//   formed from the step, like the local part).  One CTA per (orbital, z
//   plane, 32 rows): the projectors whose z and y windows meet the tile are
//   listed in a fixed order (ballot and prefix counts), their row
//   coefficients gy gz C formed once, and every point sums over the list.
// The H-apply adds NL to H w and NLS to H s; the controller adds the
// nonlocal energy f sum C_ip^2 to the external term.
#include "pou_internal.cuh"

namespace pou {

namespace {

constexpr int PNT = 256;
constexpr int AROWS = 32;

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

template <typename T>
__global__ void __launch_bounds__(PNT) k_nl_project(NlArgs<T> a) {
  if (a.st && (a.st->done || !gate_open(a.st, a.gate))) return;
  __shared__ double red[PNT / 32];
  const NlTables& t = a.tab;
  const int p = blockIdx.x, i = blockIdx.y;
  const int slot = nl_slot(a);
  const int nx = t.nx, ny = t.ny, nz = t.nz;
  const T* x = a.X[slot] + (i64)i * nx * ny * nz;
  const int* w = t.win + p * 6;
  const int x0 = w[0], wx = w[1], y0 = w[2], wy = w[3], z0 = w[4], wz = w[5];
  const T* gxp = tab_x<T>(t, p);
  // 32 threads along a window row (coalesced), 8 rows at a time
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  double acc = 0.0;
  for (int kz = 0; kz < wz; ++kz) {
    int zz = z0 + kz;
    if (zz >= nz) zz -= nz;
    const T gzv = tab_z<T>(t, p, zz);
    T plane = T(0);  // this thread's share of the plane, promoted once per plane
    for (int ky = ty; ky < wy; ky += PNT / 32) {
      int yy = y0 + ky;
      if (yy >= ny) yy -= ny;
      const T* row = x + ((i64)zz * ny + yy) * nx;
      T rs = T(0);
      for (int kx = tx; kx < wx; kx += 32) {
        int xx = x0 + kx;
        if (xx >= nx) xx -= nx;
        rs += gxp[xx] * row[xx];
      }
      plane += tab_y<T>(t, p, yy) * rs;
    }
    acc += (double)(gzv * plane);
  }
  double v = acc;
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int k = 0; k < PNT / 32; ++k) s += red[k];
    a.C[slot][(i64)i * t.P + p] = a.dV * s;
  }
}

template <typename T>
__global__ void __launch_bounds__(PNT) k_nl_apply(NlArgs<T> a) {
  if (a.st && (a.st->done || !gate_open(a.st, a.gate))) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const NlTables& t = a.tab;
  const int nx = t.nx, ny = t.ny, nz = t.nz, P = t.P;
  T* q = reinterpret_cast<T*>(smem_raw);   // [P][AROWS]: gy gz C of the listed projectors
  T* qs = q + (size_t)P * AROWS;           // [P][AROWS]: gy gz (C - C')
  int* list = reinterpret_cast<int*>(qs + (size_t)P * AROWS);
  __shared__ int wcount[PNT / 32];
  const int i = blockIdx.z, z = blockIdx.y, y0 = blockIdx.x * AROWS;
  const int slot = nl_slot(a);
  const double* C = a.C[slot] + (i64)i * P;
  const double* Cp = a.nls ? a.C[a.st->cur] + (i64)i * P : nullptr;  // the trial's previous iterate
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // projectors whose z window holds this plane and whose y window meets the rows
  bool take = false;
  if (tid < P) {
    const int* w = t.win + tid * 6;
    const int dz = (z - w[4] + nz) % nz;
    const int dy = (y0 - w[2] + ny) % ny;  // rows y0 .. y0 + AROWS - 1 meet [w2, w2 + w3) (mod ny)
    const int rows = min(AROWS, ny - y0);
    take = dz < w[5] && (dy < w[3] || dy + rows > ny || w[3] >= ny);
    if (!take && dz < w[5]) {
      for (int r = 0; r < rows && !take; ++r) take = ((y0 + r - w[2] + ny) % ny) < w[3];
    }
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
  for (int e = tid; e < cnt * AROWS; e += PNT) {
    const int k = e / AROWS, r = e - k * AROWS;
    const int p = list[k], y = y0 + r;
    T g = T(0);
    if (y < ny) g = tab_y<T>(t, p, y) * tab_z<T>(t, p, z);
    q[e] = g * (T)C[p];
    qs[e] = Cp ? g * (T)(C[p] - Cp[p]) : T(0);
  }
  __syncthreads();
  const i64 base = (i64)i * nx * ny * nz + (i64)z * nx * ny;
  const int rows = min(AROWS, ny - y0);
  for (int e = tid; e < nx * rows; e += PNT) {
    const int r = e / nx, xx = e - r * nx, y = y0 + r;
    T v = T(0), vs = T(0);
    for (int k = 0; k < cnt; ++k) {
      const T g = tab_x<T>(t, list[k])[xx];
      v += g * q[k * AROWS + r];
      vs += g * qs[k * AROWS + r];
    }
    const i64 o = base + (i64)y * nx + xx;
    a.nl[o] = v;
    if (a.nls) a.nls[o] = vs;
  }
}

template <typename T>
size_t nl_apply_smem(int P) {
  return (size_t)2 * P * AROWS * sizeof(T) + (size_t)P * sizeof(int);
}

}  // namespace

template <typename T>
void launch_nl_project(const NlArgs<T>& a, cudaStream_t s) {
  prof_begin("nl_project", s);
  k_nl_project<T><<<dim3(a.tab.P, a.N), PNT, 0, s>>>(a);
  prof_end(s);
}
template <typename T>
void launch_nl_apply(const NlArgs<T>& a, cudaStream_t s) {
  prof_begin("nl_apply", s);
  k_nl_apply<T><<<dim3((a.tab.ny + AROWS - 1) / AROWS, a.tab.nz, a.N), PNT, nl_apply_smem<T>(a.tab.P), s>>>(a);
  prof_end(s);
}

void configure_nonlocal() {
  cudaFuncSetAttribute(k_nl_apply<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)nl_apply_smem<float>(kMaxProj));
  cudaFuncSetAttribute(k_nl_apply<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)nl_apply_smem<double>(kMaxProj));
}
template void launch_nl_project<float>(const NlArgs<float>&, cudaStream_t);
template void launch_nl_project<double>(const NlArgs<double>&, cudaStream_t);
template void launch_nl_apply<float>(const NlArgs<float>&, cudaStream_t);
template void launch_nl_apply<double>(const NlArgs<double>&, cudaStream_t);

}  // namespace pou
