// H-apply pass: HW = -1/2 Lap_h W + V W on a uniform periodic grid, fused
// with the per-orbital sums the iteration needs (Sec. 3.2):
//   sigma_ii = <H w_i, w_i>, the kinetic energy f <w_i, -1/2 Lap_h w_i>
//   (Eq. energy), ||z_i||^2 and the Barzilai-Borwein traces against the
//   current iterate (S = W - W', Y = Z - Z').
//
// Layout: one orbital after another, [nz][ny][nx] each, x fastest.
// One CTA = one orbital x a 32x8 tile in (x, y) x a chunk of z planes.  The
// CTA sweeps z: each thread keeps its column's z-neighbours in a register
// queue; the current plane plus an x/y halo of width R is staged in shared
// memory (double-buffered, one barrier per plane).  Halo cells wrap
// periodically.  Second differences are formed as sums of neighbour
// differences, (u[+d] - u) + (u[-d] - u), which are exact in floating point
// for smooth fields, so the FP32 form keeps the kinetic energy accurate.
#include "pou_internal.cuh"

namespace pou {

long long g_launches = 0;
thread_local ProfRecorder* g_prof = nullptr;

namespace {

constexpr int TX = 32;
constexpr int TY = 8;
constexpr int NT = TX * TY;

__device__ __forceinline__ int wrapi(int v, int n) {
  v %= n;
  return v < 0 ? v + n : v;
}

template <typename T, int R>
__global__ void __launch_bounds__(NT) k_apply_h(ApplyArgs<T> a) {
  __shared__ T plane[2][TY + 2 * R][TX + 2 * R];
  __shared__ double red[NT / 32][NP];

  if (a.st && a.st->done) return;
  const int cur = a.st ? a.st->cur : 0;
  const int t = (a.mode == 2) ? 0 : 1 - cur;
  const bool prev = (a.mode == 0);
  const int nx = a.nx, ny = a.ny, nz = a.nz;
  const i64 ng = (i64)nx * ny * nz;
  const int orb = blockIdx.z;
  const T* w = a.W[t] + (i64)orb * ng;
  T* hw = a.HW[t] ? a.HW[t] + (i64)orb * ng : nullptr;
  const T* V = a.V[t];
  const T* wp = prev ? a.W[cur] + (i64)orb * ng : nullptr;
  const T* hp = prev ? a.HW[cur] + (i64)orb * ng : nullptr;
  const T sigp = prev ? (T)a.sigma[cur][orb] : T(0);

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
  const int xw = wrapi(x, nx), yw = wrapi(y, ny);
  const i64 col = (i64)yw * nx + xw;
  const i64 pl = (i64)nx * ny;

  // halo cell owned by this thread (80*R cells per plane)
  int hx = -1, hy = -1, sx = 0, sy = 0;
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

  T q[2 * R + 1];
#pragma unroll
  for (int j = 0; j < 2 * R; ++j) q[j] = w[(i64)wrapi(z0 - R + j, nz) * pl + col];

  T acc[NP];
#pragma unroll
  for (int k = 0; k < NP; ++k) acc[k] = T(0);

  const T c1 = (R == 1) ? T(1) : T(16) / T(12);
  const T c2 = (R == 1) ? T(0) : T(-1) / T(12);

  for (int z = z0; z < z1; ++z) {
    q[2 * R] = w[(i64)wrapi(z + R, nz) * pl + col];
    const T c = q[R];
    T(*buf)[TX + 2 * R] = plane[z & 1];
    buf[ly + R][lx + R] = c;
    if (hx >= 0) buf[sy][sx] = w[(i64)z * pl + hcol];
    __syncthreads();
    if (act) {
      const int cx = lx + R, cy = ly + R;
      T dx1 = (buf[cy][cx + 1] - c) + (buf[cy][cx - 1] - c);
      T dy1 = (buf[cy + 1][cx] - c) + (buf[cy - 1][cx] - c);
      T dz1 = (q[R + 1] - c) + (q[R - 1] - c);
      T lap;
      if (R == 1) {
        lap = a.ihx2 * dx1 + a.ihy2 * dy1 + a.ihz2 * dz1;
      } else {
        T dx2 = (buf[cy][cx + 2] - c) + (buf[cy][cx - 2] - c);
        T dy2 = (buf[cy + 2][cx] - c) + (buf[cy - 2][cx] - c);
        T dz2 = (q[R + 2] - c) + (q[R - 2] - c);
        lap = a.ihx2 * (c1 * dx1 + c2 * dx2) + a.ihy2 * (c1 * dy1 + c2 * dy2) +
              a.ihz2 * (c1 * dz1 + c2 * dz2);
      }
      const i64 idx = (i64)z * pl + col;
      const T kin = T(-0.5) * lap;
      const T h = kin + V[idx] * c;
      if (hw) hw[idx] = a.out_scale * h;
      acc[P_WW] += c * c;
      acc[P_HW] += h * c;
      acc[P_HH] += h * h;
      acc[P_KIN] += c * kin;
      if (prev) {
        const T s = c - wp[idx];
        const T b = (h - hp[idx]) - sigp * s;
        acc[P_SS] += s * s;
        acc[P_SB] += s * b;
        acc[P_SW] += s * c;
        acc[P_BB] += b * b;
        acc[P_BW] += b * c;
      }
    }
#pragma unroll
    for (int j = 0; j < 2 * R; ++j) q[j] = q[j + 1];
  }

  if (a.tilepart == nullptr) return;
  // block reduction of the sums, promoted to FP64 before combining threads
  const int lane = tid & 31, warp = tid >> 5;
#pragma unroll
  for (int k = 0; k < NP; ++k) {
    double v = (double)acc[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[warp][k] = v;
  }
  __syncthreads();
  if (tid < NP) {
    double v = 0.0;
#pragma unroll
    for (int wi = 0; wi < NT / 32; ++wi) v += red[wi][tid];
    const int ntile = gridDim.x * gridDim.y;
    const int tile = blockIdx.y * gridDim.x + blockIdx.x;
    a.tilepart[((i64)orb * ntile + tile) * NP + tid] = v;
  }
}

}  // namespace

int apply_h_ntile(int nx, int ny, int nz, int N, int* nzc_out) {
  const int ntx = (nx + TX - 1) / TX, nty = (ny + TY - 1) / TY;
  const long long base = (long long)ntx * nty * N;
  int nzc = 1;
  // enough CTAs to fill the GPU several times, with z sweeps of >= 8 planes
  while (base * nzc < 4 * 152 * 8 && nz / (nzc * 2) >= 8) nzc *= 2;
  if (nzc_out) *nzc_out = nzc;
  return ntx * nty * nzc;
}

template <typename T>
void launch_apply_h(const ApplyArgs<T>& a0, int order, cudaStream_t s, int* ntile_out) {
  ApplyArgs<T> a = a0;
  int nzc = 1;
  const int ntile = apply_h_ntile(a.nx, a.ny, a.nz, a.N, &nzc);
  a.nzc = nzc;
  const int ntx = (a.nx + TX - 1) / TX, nty = (a.ny + TY - 1) / TY;
  dim3 grid(ntx * nty, nzc, a.N), block(TX, TY);
  prof_begin("apply_h", s);
  if (order == 2)
    k_apply_h<T, 1><<<grid, block, 0, s>>>(a);
  else
    k_apply_h<T, 2><<<grid, block, 0, s>>>(a);
  prof_end(s);
  if (ntile_out) *ntile_out = ntile;
}

template void launch_apply_h<float>(const ApplyArgs<float>&, int, cudaStream_t, int*);
template void launch_apply_h<double>(const ApplyArgs<double>&, int, cudaStream_t, int*);

}  // namespace pou
