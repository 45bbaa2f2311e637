// Gaussian-well external potential and its derivatives (local
// pseudopotential of Sec. 2.1):
//   Vext(r) = -sum_I Z_I sum_n exp(-|r - R_I - nL|^2 / (2 w^2)),
// n over the 27 nearest images of R_I folded into [0, L).  The image sum of
// a Gaussian factorises per axis, so each atom is described by three 1-D
// tables g_a(k) = sum_{m=-1,0,1} exp(-(k h_a - X_a - m L_a)^2 / (2 w^2)) and
// their derivatives dg_a(k) = d g_a / d X_a; then
//   Vext = -sum_I Z_I gx gy gz,
//   dE/dX_I = -dV Z_I sum_r rho dgx gy gz (same for Y, Z),
//   dE/dZ_I = -dV sum_r rho gx gy gz.
// The force sums run over a window of +-8 w around each atom per axis
// (terms outside are below exp(-32) of the peak).
#include "pou_internal.cuh"

namespace pou {

namespace {

__global__ void k_atom_tables(const double* R, int M, double width, int nx, int ny, int nz, double Lx,
                              double Ly, double Lz, AtomTables t) {
  const int I = blockIdx.x;
  if (I >= M) return;
  const int n[3] = {nx, ny, nz};
  const double L[3] = {Lx, Ly, Lz};
  double* g[3] = {t.gx, t.gy, t.gz};
  double* dg[3] = {t.dgx, t.dgy, t.dgz};
  const double two_s2 = 2.0 * width * width, s2 = width * width;
  const double cut = 8.0 * width;
  for (int ax = 0; ax < 3; ++ax) {
    const double h = L[ax] / n[ax];
    double X = R[I * 3 + ax];
    X -= L[ax] * floor(X / L[ax]);
    for (int k = threadIdx.x; k < n[ax]; k += blockDim.x) {
      double sg = 0.0, sd = 0.0;
      for (int m = -1; m <= 1; ++m) {
        const double d = k * h - X - m * L[ax];
        const double e = exp(-d * d / two_s2);
        sg += e;
        sd += e * d / s2;
      }
      g[ax][(i64)I * n[ax] + k] = sg;
      dg[ax][(i64)I * n[ax] + k] = sd;
    }
    if (threadIdx.x == 0) {
      int start, len;
      if (2.0 * cut >= L[ax]) {
        start = 0;
        len = n[ax];
      } else {
        start = (int)ceil((X - cut) / h);
        const int stop = (int)floor((X + cut) / h);
        len = stop - start + 1;
        if (len > n[ax]) {
          start = 0;
          len = n[ax];
        }
      }
      t.win[I * 6 + ax * 2] = start;
      t.win[I * 6 + ax * 2 + 1] = len;
    }
  }
}

__global__ void k_vext(const double* Z, int M, int nx, int ny, int nz, AtomTables t, double* vext) {
  const i64 ng = (i64)nx * ny * nz;
  for (i64 p = (i64)blockIdx.x * blockDim.x + threadIdx.x; p < ng; p += (i64)gridDim.x * blockDim.x) {
    const int x = (int)(p % nx);
    const int y = (int)((p / nx) % ny);
    const int z = (int)(p / ((i64)nx * ny));
    double v = 0.0;
    for (int I = 0; I < M; ++I)
      v -= Z[I] * t.gx[(i64)I * nx + x] * t.gy[(i64)I * ny + y] * t.gz[(i64)I * nz + z];
    vext[p] = v;
  }
}

constexpr int FZS = 8;  // z splits per atom

__global__ void k_forces(const double* rho, int M, int nx, int ny, int nz, AtomTables t, double* fpart) {
  const int I = blockIdx.x;
  const int split = blockIdx.y;
  const int* w = t.win + I * 6;
  const int sx = w[0], lx = w[1], sy = w[2], ly = w[3], sz = w[4], lz = w[5];
  const int zb = (int)(((i64)split * lz) / FZS), ze = (int)(((i64)(split + 1) * lz) / FZS);
  const double* gx = t.gx + (i64)I * nx;
  const double* gy = t.gy + (i64)I * ny;
  const double* gz = t.gz + (i64)I * nz;
  const double* dgx = t.dgx + (i64)I * nx;
  const double* dgy = t.dgy + (i64)I * ny;
  const double* dgz = t.dgz + (i64)I * nz;
  double fx = 0.0, fy = 0.0, fz = 0.0, fg = 0.0;
  const i64 cnt = (i64)(ze - zb) * ly * lx;
  for (i64 q = threadIdx.x; q < cnt; q += blockDim.x) {
    const int ix = (int)(q % lx);
    const int iy = (int)((q / lx) % ly);
    const int iz = zb + (int)(q / ((i64)lx * ly));
    int x = (sx + ix) % nx;
    if (x < 0) x += nx;
    int y = (sy + iy) % ny;
    if (y < 0) y += ny;
    int z = (sz + iz) % nz;
    if (z < 0) z += nz;
    const double r = rho[((i64)z * ny + y) * nx + x];
    const double a = r * gy[y] * gz[z];
    fg += a * gx[x];
    fx += a * dgx[x];
    const double b = r * gx[x];
    fy += b * dgy[y] * gz[z];
    fz += b * gy[y] * dgz[z];
  }
  __shared__ double red[8][4];
  for (int o = 16; o > 0; o >>= 1) {
    fx += __shfl_xor_sync(0xffffffffu, fx, o);
    fy += __shfl_xor_sync(0xffffffffu, fy, o);
    fz += __shfl_xor_sync(0xffffffffu, fz, o);
    fg += __shfl_xor_sync(0xffffffffu, fg, o);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
    red[warp][0] = fx;
    red[warp][1] = fy;
    red[warp][2] = fz;
    red[warp][3] = fg;
  }
  __syncthreads();
  if (threadIdx.x < 4) {
    double v = 0.0;
    for (int k = 0; k < (int)(blockDim.x / 32); ++k) v += red[k][threadIdx.x];
    fpart[((i64)I * FZS + split) * 4 + threadIdx.x] = v;
  }
}

}  // namespace

void launch_atom_tables(const double* R, const double* Z, int M, double width, const int n[3],
                        const double L[3], const AtomTables& t, cudaStream_t s) {
  (void)Z;
  prof_begin("atom_tables", s);
  k_atom_tables<<<M, 128, 0, s>>>(R, M, width, n[0], n[1], n[2], L[0], L[1], L[2], t);
  prof_end(s);
}

void launch_vext(const double* Z, int M, const int n[3], const AtomTables& t, double* vext, cudaStream_t s) {
  prof_begin("vext", s);
  k_vext<<<num_sms() * 8, 256, 0, s>>>(Z, M, n[0], n[1], n[2], t, vext);
  prof_end(s);
}

int launch_forces(const double* rho, const double* Z, int M, const int n[3], const AtomTables& t,
                  double* fpart, cudaStream_t s) {
  (void)Z;
  dim3 grid(M, FZS);
  prof_begin("forces", s);
  k_forces<<<grid, 256, 0, s>>>(rho, M, n[0], n[1], n[2], t, fpart);
  prof_end(s);
  return FZS;
}

}  // namespace pou
