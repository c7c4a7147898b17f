// Outer residual (Section 4 stopping rule), mass rescale (eq. (32)) and the multigrid
// transfer operators (eq. (30)). All reductions are fixed-order (per-cell partials, then a
// per-instance sum in cell order) so results are run-to-run deterministic.
#include "common.cuh"
#include "kernels.h"

namespace sgs {

// Block sum of one double; result valid in thread 0.
__device__ inline double block_sum(double x, double* sh /*[32]*/) {
  double v[1] = {x};
  warp_allsum<1>(v);
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) sh[wid] = v[0];
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int k = 0; k < (int)(blockDim.x >> 5); k++) t += sh[k];
  __syncthreads();
  return t;
}

// Outgoing mass flux of each wall: side 0 sums w v1 f_0 over v1 < 0, side 1 sums w v1
// f_{J-1} over v1 > 0. flux[2 q + side].
__global__ void __launch_bounds__(256) k_wall_flux(const InstDev* inst, const double* __restrict__ f, int N,
                                                    double dv, double* flux) {
  __shared__ double sh[32];
  int q = blockIdx.x >> 1, side = blockIdx.x & 1;
  const InstDev& I = inst[q];
  int K = N * N * N;
  const double* fa = f + I.f_off + (long long)(side ? I.J - 1 : 0) * K;
  double acc = 0.0;
  for (int e = threadIdx.x; e < K; e += blockDim.x) {
    double v1 = node(e / (N * N), N, dv);
    if ((side == 0 && v1 < 0.0) || (side == 1 && v1 > 0.0)) acc += v1 * fa[e];
  }
  double t = block_sum(acc, sh);
  if (threadIdx.x == 0) flux[blockIdx.x] = dv * dv * dv * t;
}

// Per-cell sum of w R^2, R = (v1^+ (f_j - f_{j-1}) + v1^- (f_{j+1} - f_j))/dx - Q_j/eps - b_j,
// with wall ghosts rho_w * Mhat built from the same f. Optionally stores R.
__global__ void __launch_bounds__(256) k_residual_cells(AuxArgs a, const double* __restrict__ f,
                                                         const double* __restrict__ Q, const double* __restrict__ rhs,
                                                         const double* flux, double* part, double* Rout) {
  __shared__ double sh[32];
  int c = blockIdx.x;
  int q = a.cell_inst[c];
  const InstDev& I = a.inst[q];
  int N = a.N, K = N * N * N;
  long long base = a.cell_off[c];
  int j = (int)((base - I.f_off) / K);
  double w = a.dv * a.dv * a.dv;
  double inv_dx = 1.0 / I.dx, inv_eps = 1.0 / I.eps;
  double rho_l = I.bc_kind[0] == SGS_INFLOW ? I.bc_rho[0] : -flux[2 * q] / I.wall_denom[0];
  double rho_r = I.bc_kind[1] == SGS_INFLOW ? I.bc_rho[1] : -flux[2 * q + 1] / I.wall_denom[1];
  double acc = 0.0;
  for (int e = threadIdx.x; e < K; e += blockDim.x) {
    int i1 = e / (N * N), i2 = (e / N) % N, i3 = e % N;
    double v1 = node(i1, N, a.dv);
    double fj = f[base + e];
    double fl = j == 0 ? rho_l * I.wall[0][0][i1] * I.wall[0][1][i2] * I.wall[0][2][i3] : f[base - K + e];
    double fr = j == I.J - 1 ? rho_r * I.wall[1][0][i1] * I.wall[1][1][i2] * I.wall[1][2][i3] : f[base + K + e];
    double R = (fmax(v1, 0.0) * (fj - fl) + fmin(v1, 0.0) * (fr - fj)) * inv_dx - Q[base + e] * inv_eps;
    if (rhs) R -= rhs[base + e];
    if (Rout) Rout[base + e] = R;
    acc += R * R;
  }
  double t = block_sum(acc, sh);
  if (threadIdx.x == 0) part[c] = w * t;
}

__global__ void k_residual_final(const InstDev* inst, int n_inst, const double* part, double* res) {
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n_inst) return;
  const InstDev& I = inst[q];
  double s = 0.0;
  for (int j = 0; j < I.J; j++) s += part[I.cell0 + j];
  res[q] = sqrt(I.dx * I.dy * s);
}

// ---------------------------------------------------------------------------------------
// 2-D residual (one instance, nx x ny cells, row by row): face index of the boundary faces
// x_lo: j, x_hi: ny + j, y_lo: 2 ny + i, y_hi: 2 ny + nx + i. flux = w sum of (v.n) f over the
// velocities leaving the domain through the face.
// ---------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_wall_flux2d(AuxArgs a, const double* __restrict__ f, double* flux) {
  __shared__ double sh[32];
  const InstDev& I = a.inst[0];
  const int nx = a.nx, ny = a.ny, N = a.N, K = N * N * N;
  int face = blockIdx.x, side, cell;
  if (face < ny) {
    side = 0;
    cell = face * nx;
  } else if (face < 2 * ny) {
    side = 1;
    cell = (face - ny) * nx + nx - 1;
  } else if (face < 2 * ny + nx) {
    side = 2;
    cell = face - 2 * ny;
  } else {
    side = 3;
    cell = (ny - 1) * nx + (face - 2 * ny - nx);
  }
  const double* fc = f + I.f_off + (long long)cell * K;
  double acc = 0.0;
  for (int e = threadIdx.x; e < K; e += blockDim.x) {
    double vn = node(side < 2 ? e / (N * N) : (e / N) % N, N, a.dv);
    bool out = side % 2 == 0 ? vn < 0.0 : vn > 0.0;
    if (out) acc += vn * fc[e];
  }
  double t = block_sum(acc, sh);
  if (threadIdx.x == 0) flux[face] = a.dv * a.dv * a.dv * t;
}

__global__ void __launch_bounds__(256) k_residual_cells2d(AuxArgs a, const double* __restrict__ f,
                                                           const double* __restrict__ Q,
                                                           const double* __restrict__ rhs, const double* flux,
                                                           double* part, double* Rout) {
  __shared__ double sh[32];
  const InstDev& I = a.inst[0];
  const int nx = a.nx, ny = a.ny, N = a.N, K = N * N * N;
  const int c = blockIdx.x, ci = c % nx, cj = c / nx;
  const long long base = I.f_off + (long long)c * K;
  const double w = a.dv * a.dv * a.dv, inv_dx = 1.0 / I.dx, inv_dy = 1.0 / I.dy, inv_eps = 1.0 / I.eps;
  double rw[4];
  const int fidx[4] = {cj, ny + cj, 2 * ny + ci, 2 * ny + nx + ci};
  for (int s = 0; s < 4; s++) rw[s] = I.bc_kind[s] == SGS_INFLOW ? I.bc_rho[s] : -flux[fidx[s]] / I.wall_denom[s];
  double acc = 0.0;
  for (int e = threadIdx.x; e < K; e += blockDim.x) {
    int i1 = e / (N * N), i2 = (e / N) % N, i3 = e % N;
    double v1 = node(i1, N, a.dv), v2 = node(i2, N, a.dv);
    double fc = f[base + e];
    double gh[4];
    for (int s = 0; s < 4; s++) gh[s] = rw[s] * I.wall[s][0][i1] * I.wall[s][1][i2] * I.wall[s][2][i3];
    double fw = ci == 0 ? gh[0] : f[base - K + e];
    double fe = ci == nx - 1 ? gh[1] : f[base + K + e];
    double fs = cj == 0 ? gh[2] : f[base - (long long)nx * K + e];
    double fn = cj == ny - 1 ? gh[3] : f[base + (long long)nx * K + e];
    double R = (fmax(v1, 0.0) * (fc - fw) + fmin(v1, 0.0) * (fe - fc)) * inv_dx +
               (fmax(v2, 0.0) * (fc - fs) + fmin(v2, 0.0) * (fn - fc)) * inv_dy - Q[base + e] * inv_eps;
    if (rhs) R -= rhs[base + e];
    if (Rout) Rout[base + e] = R;
    acc += R * R;
  }
  double t = block_sum(acc, sh);
  if (threadIdx.x == 0) part[c] = w * t;
}

// ---------------------------------------------------------------------------------------
// Second-order scheme, 1-D (eq. (reconstruction), eq. (slope)): slopes central inside and
// one-sided in the first and last cell, faces f^-_{j+1/2} = f_j + s_j/2, f^+_{j-1/2} =
// f_j - s_j/2, zero ghost slopes; diffuse-wall densities from the outgoing face value.
// ---------------------------------------------------------------------------------------
__device__ inline double slope1d(const InstDev& I, const double* f, long long base, int j, int e, int K) {
  if (I.J < 2) return 0.0;
  if (j == 0) return f[base + K + e] - f[base + e];
  if (j == I.J - 1) return f[base + e] - f[base - K + e];
  return 0.5 * (f[base + K + e] - f[base - K + e]);
}

// sflux[2 q + side] = w sum over the outgoing velocities of v1 s at the wall cell.
__global__ void __launch_bounds__(256) k_wall_slope_flux(AuxArgs a, const double* __restrict__ f, double* sflux) {
  __shared__ double sh[32];
  int q = blockIdx.x >> 1, side = blockIdx.x & 1;
  const InstDev& I = a.inst[q];
  int N = a.N, K = N * N * N;
  int j = side ? I.J - 1 : 0;
  long long base = I.f_off + (long long)j * K;
  double acc = 0.0;
  for (int e = threadIdx.x; e < K; e += blockDim.x) {
    double v1 = node(e / (N * N), N, a.dv);
    if ((side == 0 && v1 < 0.0) || (side == 1 && v1 > 0.0)) acc += v1 * slope1d(I, f, base, j, e, K);
  }
  double t = block_sum(acc, sh);
  if (threadIdx.x == 0) sflux[blockIdx.x] = a.dv * a.dv * a.dv * t;
}

// Right-hand side of a second-order scan from the state f before it:
//   out = rhs + (v1^+ s_{j-1} - v1 s_j + v1^- s_{j+1}) / (2 dx)    (eq. (SGS_BGK), r = ... - out)
// plus, in the wall cells, the change of the lagged ghost from the cell value the scan uses
// to the face value (rho = -flux_out / wall_denom, flux_out of f_0 - s_0/2 resp. f_{J-1} +
// s_{J-1}/2): + v1^+ drho_l Mhat_l / dx in cell 0, - v1^- drho_r Mhat_r / dx in cell J-1.
__global__ void __launch_bounds__(256) k_slope_rhs(AuxArgs a, const double* __restrict__ f,
                                                   const double* __restrict__ rhs, const double* __restrict__ sflux,
                                                   double* __restrict__ out) {
  int c = blockIdx.x;
  int q = a.cell_inst[c];
  const InstDev& I = a.inst[q];
  int N = a.N, K = N * N * N;
  long long base = a.cell_off[c];
  int j = (int)((base - I.f_off) / K);
  double inv_dx = 1.0 / I.dx;
  double drho_l = (j == 0 && I.bc_kind[0] != SGS_INFLOW) ? 0.5 * sflux[2 * q] / I.wall_denom[0] : 0.0;
  double drho_r = (j == I.J - 1 && I.bc_kind[1] != SGS_INFLOW) ? -0.5 * sflux[2 * q + 1] / I.wall_denom[1] : 0.0;
  for (int e = blockIdx.y * blockDim.x + threadIdx.x; e < K; e += gridDim.y * blockDim.x) {
    int i1 = e / (N * N), i2 = (e / N) % N, i3 = e % N;
    double v1 = node(i1, N, a.dv);
    double sj = slope1d(I, f, base, j, e, K);
    double sm = j > 0 ? slope1d(I, f, base - K, j - 1, e, K) : 0.0;
    double sp = j < I.J - 1 ? slope1d(I, f, base + K, j + 1, e, K) : 0.0;
    double b = (rhs ? rhs[base + e] : 0.0) + (fmax(v1, 0.0) * sm - v1 * sj + fmin(v1, 0.0) * sp) * (0.5 * inv_dx);
    if (drho_l != 0.0) b += fmax(v1, 0.0) * drho_l * I.wall[0][0][i1] * I.wall[0][1][i2] * I.wall[0][2][i3] * inv_dx;
    if (drho_r != 0.0) b -= fmin(v1, 0.0) * drho_r * I.wall[1][0][i1] * I.wall[1][1][i2] * I.wall[1][2][i3] * inv_dx;
    out[base + e] = b;
  }
}

cudaError_t launch_slope_rhs(const AuxArgs& a, const double* f, const double* rhs, double* out, cudaStream_t st) {
  k_wall_slope_flux<<<2 * a.n_inst, 256, 0, st>>>(a, f, a.sflux);
  k_slope_rhs<<<dim3(a.C, 4), 256, 0, st>>>(a, f, rhs, a.sflux, out);
  return cudaGetLastError();
}

// Second-order residual per cell: R = (v1^+ (f^-_{j+1/2} - f^-_{j-1/2}) + v1^- (f^+_{j+1/2} -
// f^+_{j-1/2}))/dx - Q_j/eps - b_j (eq. (upwind)), ghosts from the face values of the same f.
__global__ void __launch_bounds__(256) k_residual_cells_o2(AuxArgs a, const double* __restrict__ f,
                                                            const double* __restrict__ Q,
                                                            const double* __restrict__ rhs, const double* flux,
                                                            const double* sflux, double* part, double* Rout) {
  __shared__ double sh[32];
  int c = blockIdx.x;
  int q = a.cell_inst[c];
  const InstDev& I = a.inst[q];
  int N = a.N, K = N * N * N;
  long long base = a.cell_off[c];
  int j = (int)((base - I.f_off) / K);
  double w = a.dv * a.dv * a.dv;
  double inv_dx = 1.0 / I.dx, inv_eps = 1.0 / I.eps;
  double rho_l = I.bc_kind[0] == SGS_INFLOW ? I.bc_rho[0] : -(flux[2 * q] - 0.5 * sflux[2 * q]) / I.wall_denom[0];
  double rho_r =
      I.bc_kind[1] == SGS_INFLOW ? I.bc_rho[1] : -(flux[2 * q + 1] + 0.5 * sflux[2 * q + 1]) / I.wall_denom[1];
  double acc = 0.0;
  for (int e = threadIdx.x; e < K; e += blockDim.x) {
    int i1 = e / (N * N), i2 = (e / N) % N, i3 = e % N;
    double v1 = node(i1, N, a.dv);
    double fj = f[base + e];
    double sj = slope1d(I, f, base, j, e, K);
    double mr = fj + 0.5 * sj, pl = fj - 0.5 * sj;
    double ml = j == 0 ? rho_l * I.wall[0][0][i1] * I.wall[0][1][i2] * I.wall[0][2][i3]
                       : f[base - K + e] + 0.5 * slope1d(I, f, base - K, j - 1, e, K);
    double pr = j == I.J - 1 ? rho_r * I.wall[1][0][i1] * I.wall[1][1][i2] * I.wall[1][2][i3]
                             : f[base + K + e] - 0.5 * slope1d(I, f, base + K, j + 1, e, K);
    double R = (fmax(v1, 0.0) * (mr - ml) + fmin(v1, 0.0) * (pr - pl)) * inv_dx - Q[base + e] * inv_eps;
    if (rhs) R -= rhs[base + e];
    if (Rout) Rout[base + e] = R;
    acc += R * R;
  }
  double t = block_sum(acc, sh);
  if (threadIdx.x == 0) part[c] = w * t;
}

// ---------------------------------------------------------------------------------------
// Second-order scheme, 2-D: the slopes of eq. (slope) along x within each row and along y
// within each column (central inside, one-sided in the end cells, zero when the grid has a
// single cell in that direction), zero ghost slopes, wall ghosts from the outgoing face
// value f -/+ s/2 of the slope normal to the side. Cells (i, j) at j nx + i.
// ---------------------------------------------------------------------------------------
__device__ inline double slope_x2d(const double* f, long long base, int ci, int nx, int e, int K) {
  if (nx < 2) return 0.0;
  if (ci == 0) return f[base + K + e] - f[base + e];
  if (ci == nx - 1) return f[base + e] - f[base - K + e];
  return 0.5 * (f[base + K + e] - f[base - K + e]);
}
__device__ inline double slope_y2d(const double* f, long long base, int cj, int nx, int ny, int e, int K) {
  if (ny < 2) return 0.0;
  const long long r = (long long)nx * K;
  if (cj == 0) return f[base + r + e] - f[base + e];
  if (cj == ny - 1) return f[base + e] - f[base - r + e];
  return 0.5 * (f[base + r + e] - f[base - r + e]);
}

// Boundary face of index `face` (numbering of k_wall_flux2d): its side and cell.
__device__ inline void face_cell2d(int face, int nx, int ny, int& side, int& cell) {
  if (face < ny) {
    side = 0;
    cell = face * nx;
  } else if (face < 2 * ny) {
    side = 1;
    cell = (face - ny) * nx + nx - 1;
  } else if (face < 2 * ny + nx) {
    side = 2;
    cell = face - 2 * ny;
  } else {
    side = 3;
    cell = (ny - 1) * nx + (face - 2 * ny - nx);
  }
}

// sflux[face] = w sum over the velocities leaving the domain through the face of (v.n) s_n,
// s_n the slope normal to the face's side in its cell.
__global__ void __launch_bounds__(256) k_wall_slope_flux2d(AuxArgs a, const double* __restrict__ f, double* sflux) {
  __shared__ double sh[32];
  const InstDev& I = a.inst[0];
  const int nx = a.nx, ny = a.ny, N = a.N, K = N * N * N;
  int side, cell;
  face_cell2d(blockIdx.x, nx, ny, side, cell);
  const int ci = cell % nx, cj = cell / nx;
  const long long base = I.f_off + (long long)cell * K;
  double acc = 0.0;
  for (int e = threadIdx.x; e < K; e += blockDim.x) {
    double vn = node(side < 2 ? e / (N * N) : (e / N) % N, N, a.dv);
    bool out = side % 2 == 0 ? vn < 0.0 : vn > 0.0;
    if (out) acc += vn * (side < 2 ? slope_x2d(f, base, ci, nx, e, K) : slope_y2d(f, base, cj, nx, ny, e, K));
  }
  double t = block_sum(acc, sh);
  if (threadIdx.x == 0) sflux[blockIdx.x] = a.dv * a.dv * a.dv * t;
}

// Right-hand side of a second-order 2-D scan ordering from the state f before it (r = ... - out):
//   out = rhs + (v1^+ sx_W - v1 sx + v1^- sx_E) / (2 dx) + (v2^+ sy_S - v2 sy + v2^- sy_N) / (2 dy)
// (zero slopes beyond the walls), plus in the wall cells the change of each lagged ghost from
// the cell value the scan uses to the face value: rho_face - rho_cell = +0.5 sflux / denom on
// the x_lo / y_lo sides (face f - s/2), -0.5 sflux / denom on the x_hi / y_hi sides; the
// scan's r holds -v1^+ ghost_W / dx, +v1^- ghost_E / dx, -v2^+ ghost_S / dy, +v2^- ghost_N / dy.
__global__ void __launch_bounds__(256) k_slope_rhs2d(AuxArgs a, const double* __restrict__ f,
                                                     const double* __restrict__ rhs,
                                                     const double* __restrict__ sflux, double* __restrict__ out) {
  const InstDev& I = a.inst[0];
  const int nx = a.nx, ny = a.ny, N = a.N, K = N * N * N;
  const int c = blockIdx.x, ci = c % nx, cj = c / nx;
  const long long base = I.f_off + (long long)c * K;
  const double inv_dx = 1.0 / I.dx, inv_dy = 1.0 / I.dy;
  const int fidx[4] = {cj, ny + cj, 2 * ny + ci, 2 * ny + nx + ci};
  const bool at[4] = {ci == 0, ci == nx - 1, cj == 0, cj == ny - 1};
  double drho[4];
  for (int s = 0; s < 4; s++)
    drho[s] = (at[s] && I.bc_kind[s] != SGS_INFLOW) ? (s % 2 == 0 ? 0.5 : -0.5) * sflux[fidx[s]] / I.wall_denom[s]
                                                    : 0.0;
  for (int e = blockIdx.y * blockDim.x + threadIdx.x; e < K; e += gridDim.y * blockDim.x) {
    int i1 = e / (N * N), i2 = (e / N) % N, i3 = e % N;
    double v1 = node(i1, N, a.dv), v2 = node(i2, N, a.dv);
    double sx = slope_x2d(f, base, ci, nx, e, K), sy = slope_y2d(f, base, cj, nx, ny, e, K);
    double sw = ci > 0 ? slope_x2d(f, base - K, ci - 1, nx, e, K) : 0.0;
    double se = ci < nx - 1 ? slope_x2d(f, base + K, ci + 1, nx, e, K) : 0.0;
    const long long r = (long long)nx * K;
    double ss = cj > 0 ? slope_y2d(f, base - r, cj - 1, nx, ny, e, K) : 0.0;
    double sn = cj < ny - 1 ? slope_y2d(f, base + r, cj + 1, nx, ny, e, K) : 0.0;
    double b = (rhs ? rhs[base + e] : 0.0) + (fmax(v1, 0.0) * sw - v1 * sx + fmin(v1, 0.0) * se) * (0.5 * inv_dx) +
               (fmax(v2, 0.0) * ss - v2 * sy + fmin(v2, 0.0) * sn) * (0.5 * inv_dy);
    double Mh[4];
    for (int s = 0; s < 4; s++) Mh[s] = drho[s] != 0.0 ? drho[s] * I.wall[s][0][i1] * I.wall[s][1][i2] * I.wall[s][2][i3] : 0.0;
    b += fmax(v1, 0.0) * Mh[0] * inv_dx - fmin(v1, 0.0) * Mh[1] * inv_dx + fmax(v2, 0.0) * Mh[2] * inv_dy -
         fmin(v2, 0.0) * Mh[3] * inv_dy;
    out[base + e] = b;
  }
}

cudaError_t launch_slope_rhs2d(const AuxArgs& a, const double* f, const double* rhs, double* out, cudaStream_t st) {
  k_wall_slope_flux2d<<<2 * (a.nx + a.ny), 256, 0, st>>>(a, f, a.sflux);
  k_slope_rhs2d<<<dim3(a.C, 4), 256, 0, st>>>(a, f, rhs, a.sflux, out);
  return cudaGetLastError();
}

// Second-order 2-D residual per cell: the upwind differences of the face values in x and y
// (eq. (upwind) in each direction), R = (v1^+ ((f + sx/2) - (f_W + sx_W/2)) + v1^- ((f_E - sx_E/2)
// - (f - sx/2))) / dx + (the same in y) / dy - Q/eps - b, ghosts from the face values of the
// same f with zero ghost slopes.
__global__ void __launch_bounds__(256) k_residual_cells2d_o2(AuxArgs a, const double* __restrict__ f,
                                                              const double* __restrict__ Q,
                                                              const double* __restrict__ rhs, const double* flux,
                                                              const double* sflux, double* part, double* Rout) {
  __shared__ double sh[32];
  const InstDev& I = a.inst[0];
  const int nx = a.nx, ny = a.ny, N = a.N, K = N * N * N;
  const int c = blockIdx.x, ci = c % nx, cj = c / nx;
  const long long base = I.f_off + (long long)c * K, r = (long long)nx * K;
  const double w = a.dv * a.dv * a.dv, inv_dx = 1.0 / I.dx, inv_dy = 1.0 / I.dy, inv_eps = 1.0 / I.eps;
  double rw[4];
  const int fidx[4] = {cj, ny + cj, 2 * ny + ci, 2 * ny + nx + ci};
  for (int s = 0; s < 4; s++)
    rw[s] = I.bc_kind[s] == SGS_INFLOW ? I.bc_rho[s]
                                       : -(flux[fidx[s]] + (s % 2 == 0 ? -0.5 : 0.5) * sflux[fidx[s]]) / I.wall_denom[s];
  double acc = 0.0;
  for (int e = threadIdx.x; e < K; e += blockDim.x) {
    int i1 = e / (N * N), i2 = (e / N) % N, i3 = e % N;
    double v1 = node(i1, N, a.dv), v2 = node(i2, N, a.dv);
    double fc = f[base + e];
    double hx = 0.5 * slope_x2d(f, base, ci, nx, e, K), hy = 0.5 * slope_y2d(f, base, cj, nx, ny, e, K);
    double gh[4];
    for (int s = 0; s < 4; s++) gh[s] = rw[s] * I.wall[s][0][i1] * I.wall[s][1][i2] * I.wall[s][2][i3];
    double xw = ci == 0 ? gh[0] : f[base - K + e] + 0.5 * slope_x2d(f, base - K, ci - 1, nx, e, K);
    double xe = ci == nx - 1 ? gh[1] : f[base + K + e] - 0.5 * slope_x2d(f, base + K, ci + 1, nx, e, K);
    double ys = cj == 0 ? gh[2] : f[base - r + e] + 0.5 * slope_y2d(f, base - r, cj - 1, nx, ny, e, K);
    double yn = cj == ny - 1 ? gh[3] : f[base + r + e] - 0.5 * slope_y2d(f, base + r, cj + 1, nx, ny, e, K);
    double R = (fmax(v1, 0.0) * ((fc + hx) - xw) + fmin(v1, 0.0) * (xe - (fc - hx))) * inv_dx +
               (fmax(v2, 0.0) * ((fc + hy) - ys) + fmin(v2, 0.0) * (yn - (fc - hy))) * inv_dy - Q[base + e] * inv_eps;
    if (rhs) R -= rhs[base + e];
    if (Rout) Rout[base + e] = R;
    acc += R * R;
  }
  double t = block_sum(acc, sh);
  if (threadIdx.x == 0) part[c] = w * t;
}

cudaError_t launch_residual_impl(const AuxArgs& a, const double* f, const double* Q, const double* rhs, double* res,
                                 double* R, cudaStream_t st) {
  double* flux = a.scratch;                  // [2 n_inst]
  double* part = a.scratch + 2 * a.n_inst;   // [C]
  if (a.two_d) {
    double* flux2 = a.scratch + 2 * a.n_inst + 2 * a.C;  // [2 (nx + ny)], after the mass slots
    k_wall_flux2d<<<2 * (a.nx + a.ny), 256, 0, st>>>(a, f, flux2);
    if (a.sflux) {  // second-order scheme
      k_wall_slope_flux2d<<<2 * (a.nx + a.ny), 256, 0, st>>>(a, f, a.sflux);
      k_residual_cells2d_o2<<<a.C, 256, 0, st>>>(a, f, Q, rhs, flux2, a.sflux, part, R);
    } else {
      k_residual_cells2d<<<a.C, 256, 0, st>>>(a, f, Q, rhs, flux2, part, R);
    }
    if (res) k_residual_final<<<1, 32, 0, st>>>(a.inst, 1, part, res);
    return cudaGetLastError();
  }
  k_wall_flux<<<2 * a.n_inst, 256, 0, st>>>(a.inst, f, a.N, a.dv, flux);
  if (a.sflux) {  // second-order scheme
    k_wall_slope_flux<<<2 * a.n_inst, 256, 0, st>>>(a, f, a.sflux);
    k_residual_cells_o2<<<a.C, 256, 0, st>>>(a, f, Q, rhs, flux, a.sflux, part, R);
  } else {
    k_residual_cells<<<a.C, 256, 0, st>>>(a, f, Q, rhs, flux, part, R);
  }
  if (res) k_residual_final<<<(a.n_inst + 127) / 128, 128, 0, st>>>(a.inst, a.n_inst, part, res);
  return cudaGetLastError();
}

// Source iteration (eq. (SI)) with the lagged BGK-penalty source (eq. (28)): for every
// velocity node of every instance,
//   (|v1|/dx + nu_j/eps) f_j = (|v1|/dx) f_upwind + P_j/eps + (nu_j/eps) M_j + b_j,
// marched from the node's inflow side, with P, nu and the Maxwellian factors (efac) of the
// previous iterate and its wall fluxes (flux) for the diffuse-wall ghosts. One thread per
// (node, instance): nodes are independent, cells are visited in order.
__global__ void __launch_bounds__(256) k_si_transport(AuxArgs a, double* f, const double* __restrict__ P,
                                                      const double* __restrict__ rhs,
                                                      const double* __restrict__ efac,
                                                      const double* __restrict__ nu,
                                                      const double* __restrict__ flux) {
  const int q = blockIdx.y;
  if (a.active && !a.active[q]) return;
  const InstDev& I = a.inst[q];
  const int N = a.N, K = N * N * N;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= K) return;
  const int i1 = e / (N * N), i2 = (e / N) % N, i3 = e % N;
  const double v1 = node(i1, N, a.dv);
  const double c = fabs(v1) / I.dx, inv_eps = 1.0 / I.eps;
  const int side = v1 > 0.0 ? 0 : 1;  // the node's inflow side (v1 = 0 needs none: c = 0)
  const double rho_w = I.bc_kind[side] == SGS_INFLOW ? I.bc_rho[side] : -flux[2 * q + side] / I.wall_denom[side];
  double up = rho_w * I.wall[side][0][i1] * I.wall[side][1][i2] * I.wall[side][2][i3];
  for (int s = 0; s < I.J; s++) {
    const int j = v1 < 0.0 ? I.J - 1 - s : s;
    const int cell = I.cell0 + j;
    const long long o = I.f_off + (long long)j * K + e;
    const double* ef = efac + (long long)cell * 3 * kMaxN;
    const double M = ef[i1] * ef[kMaxN + i2] * ef[2 * kMaxN + i3];
    const double A = nu[cell] * inv_eps;
    double src = P[o] * inv_eps + A * M;
    if (rhs) src += rhs[o];
    const double x = (c * up + src) / (c + A);
    f[o] = x;
    up = x;
  }
}

cudaError_t launch_si_transport(const AuxArgs& a, double* f, const double* P, const double* rhs, const double* efac,
                                const double* nu, cudaStream_t st) {
  double* flux = a.scratch;  // [2 n_inst], the walls' outgoing fluxes of the previous iterate
  k_wall_flux<<<2 * a.n_inst, 256, 0, st>>>(a.inst, f, a.N, a.dv, flux);
  const int K = a.N * a.N * a.N;
  k_si_transport<<<dim3((K + 255) / 256, a.n_inst), 256, 0, st>>>(a, f, P, rhs, efac, nu, flux);
  return cudaGetLastError();
}

cudaError_t launch_residual(const AuxArgs& a, const double* f, const double* Q, const double* rhs, double* res,
                            cudaStream_t st) {
  return launch_residual_impl(a, f, Q, rhs, res, nullptr, st);
}

cudaError_t launch_residual_field(const AuxArgs& a, const double* f, const double* Q, const double* rhs, double* R,
                                  cudaStream_t st) {
  return launch_residual_impl(a, f, Q, rhs, nullptr, R, st);
}

// ---------------------------------------------------------------------------------------
// Mass rescale: mass[c] = w sum f, then f *= C / (dx sum_j mass[j]) per instance.
// ---------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_cell_mass(AuxArgs a, const double* __restrict__ f, double* mass) {
  __shared__ double sh[32];
  int c = blockIdx.x;
  int K = a.N * a.N * a.N;
  const double* fc = f + a.cell_off[c];
  double acc = 0.0;
  for (int e = threadIdx.x; e < K; e += blockDim.x) acc += fc[e];
  double t = block_sum(acc, sh);
  if (threadIdx.x == 0) mass[c] = a.dv * a.dv * a.dv * t;
}

__global__ void __launch_bounds__(256) k_rescale_apply(AuxArgs a, double* f, const double* mass) {
  __shared__ double lam_s;
  int c = blockIdx.x;
  int q = a.cell_inst[c];
  const InstDev& I = a.inst[q];
  if (!(I.total_mass > 0.0) || (a.active && !a.active[q])) return;
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int j = 0; j < I.J; j++) s += mass[I.cell0 + j];
    lam_s = I.total_mass / (I.dx * I.dy * s);
  }
  __syncthreads();
  double lam = lam_s;
  int K = a.N * a.N * a.N;
  double* fc = f + a.cell_off[c];
  for (int e = blockIdx.y * blockDim.x + threadIdx.x; e < K; e += gridDim.y * blockDim.x) fc[e] *= lam;
}

// Macroscopic quantities of every cell: rho, U and T as the moments define them (d = 3) and
// the heat flux q = 1/2 sum w (v - U)|v - U|^2 f of the lid-driven cavity study (Section
// 4.2.2). out[8 c ..] = (rho, U1, U2, U3, T, q1, q2, q3). Raw sums give rho and U, a second
// pass over the cell's nodes (from L2) forms the central sums about U, so T and q carry no
// cancellation between raw moments.
__global__ void __launch_bounds__(256) k_macroscopic(AuxArgs a, const double* __restrict__ f, double* __restrict__ out) {
  __shared__ double sh[4][32];
  __shared__ double tot[4];
  const int c = blockIdx.x, N = a.N, K = N * N * N;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const double* fc = f + a.cell_off[c];
  const double dv = a.dv, w = dv * dv * dv;
  auto block_sums = [&](double (&x)[4]) {
    warp_allsum<4>(x);
    if (lane == 0)
      for (int k = 0; k < 4; k++) sh[k][wid] = x[k];
    __syncthreads();
    if (threadIdx.x < 4) {
      double t = 0.0;
      for (int k = 0; k < nw; k++) t += sh[threadIdx.x][k];
      tot[threadIdx.x] = t;
    }
    __syncthreads();
  };
  double x[4] = {0.0, 0.0, 0.0, 0.0};
  for (int e = threadIdx.x; e < K; e += blockDim.x) {
    const double fe = fc[e];
    x[0] += fe;
    x[1] += node(e / (N * N), N, dv) * fe;
    x[2] += node((e / N) % N, N, dv) * fe;
    x[3] += node(e % N, N, dv) * fe;
  }
  block_sums(x);
  const double s0 = tot[0], U1 = tot[1] / s0, U2 = tot[2] / s0, U3 = tot[3] / s0;
  __syncthreads();
  double y[4] = {0.0, 0.0, 0.0, 0.0};
  for (int e = threadIdx.x; e < K; e += blockDim.x) {
    const double fe = fc[e];
    const double c1 = node(e / (N * N), N, dv) - U1, c2 = node((e / N) % N, N, dv) - U2, c3 = node(e % N, N, dv) - U3;
    const double cc = c1 * c1 + c2 * c2 + c3 * c3, fcc = fe * cc;
    y[0] += fcc;
    y[1] += c1 * fcc;
    y[2] += c2 * fcc;
    y[3] += c3 * fcc;
  }
  block_sums(y);
  if (threadIdx.x == 0) {
    double* o = out + 8 * (long long)c;
    o[0] = w * s0;
    o[1] = U1;
    o[2] = U2;
    o[3] = U3;
    o[4] = tot[0] / (3.0 * s0);
    o[5] = 0.5 * w * tot[1];
    o[6] = 0.5 * w * tot[2];
    o[7] = 0.5 * w * tot[3];
  }
}

cudaError_t launch_macroscopic(const AuxArgs& a, const double* f, double* out, cudaStream_t st) {
  if (a.C <= 0) return cudaSuccess;
  k_macroscopic<<<a.C, 256, 0, st>>>(a, f, out);
  return cudaGetLastError();
}

cudaError_t launch_rescale(const AuxArgs& a, double* f, cudaStream_t st) {
  double* mass = a.scratch + 2 * a.n_inst + a.C;  // [C]
  k_cell_mass<<<a.C, 256, 0, st>>>(a, f, mass);
  k_rescale_apply<<<dim3(a.C, 4), 256, 0, st>>>(a, f, mass);
  return cudaGetLastError();
}

// Collision results of cells evaluated before the rescale, carried over to the rescaled
// state: with f -> lam f, Q and P = Q - nu (M - f) scale by lam^2 (Q is quadratic, nu linear
// and M homogeneous of degree 1 in f), nu by lam and the Maxwellian's exp(alpha) by lam. lam
// is formed exactly as k_rescale_apply forms it, from the same per-cell masses. Cells
// [c_lo, c_lo + gridDim.x).
__global__ void __launch_bounds__(256) k_rescale_fixup(AuxArgs a, const double* mass, int c_lo, double* Q, double* P,
                                                       double* nu, double* theta) {
  __shared__ double lam_s;
  int c = c_lo + blockIdx.x;
  int q = a.cell_inst[c];
  const InstDev& I = a.inst[q];
  if (!(I.total_mass > 0.0) || (a.active && !a.active[q])) return;
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int j = 0; j < I.J; j++) s += mass[I.cell0 + j];
    lam_s = I.total_mass / (I.dx * I.dy * s);
  }
  __syncthreads();
  const double lam = lam_s, lam2 = lam * lam;
  const int K = a.N * a.N * a.N;
  const long long off = a.cell_off[c];
  for (int e = blockIdx.y * blockDim.x + threadIdx.x; e < K; e += gridDim.y * blockDim.x) {
    if (Q) Q[off + e] *= lam2;
    if (P) P[off + e] *= lam2;
  }
  if (blockIdx.y == 0 && threadIdx.x == 0) {
    nu[c] *= lam;
    theta[5 * (long long)c] += log(lam);
  }
}

cudaError_t launch_rescale_fixup(const AuxArgs& a, int c_lo, int c_hi, double* Q, double* P, double* nu,
                                 double* theta, cudaStream_t st) {
  if (c_hi <= c_lo) return cudaSuccess;
  const double* mass = a.scratch + 2 * a.n_inst + a.C;  // written by launch_rescale
  k_rescale_fixup<<<dim3(c_hi - c_lo, 4), 256, 0, st>>>(a, mass, c_lo, Q, P, nu, theta);
  return cudaGetLastError();
}

// Defect-correction right-hand side b = (Q_hi - Q_lo) / eps, in place over Q_lo.
__global__ void __launch_bounds__(256) k_dc_rhs(AuxArgs a, const double* __restrict__ Qhi, double* Qlo_b) {
  int c = blockIdx.x;
  const InstDev& I = a.inst[a.cell_inst[c]];
  double inv_eps = 1.0 / I.eps;
  int K = a.N * a.N * a.N;
  long long base = a.cell_off[c];
  for (int e = blockIdx.y * blockDim.x + threadIdx.x; e < K; e += gridDim.y * blockDim.x)
    Qlo_b[base + e] = (Qhi[base + e] - Qlo_b[base + e]) * inv_eps;
}

cudaError_t launch_dc_rhs(const AuxArgs& a, const double* Qhi, double* Qlo_b, cudaStream_t st) {
  k_dc_rhs<<<dim3(a.C, 4), 256, 0, st>>>(a, Qhi, Qlo_b);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------
// Multigrid transfers on one instance's contiguous cells (K doubles per cell).
// ---------------------------------------------------------------------------------------
__global__ void k_restrict(const double* __restrict__ fine, double* __restrict__ coarse, long long K, long long n) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  for (; i < n; i += (long long)gridDim.x * blockDim.x) {
    long long jc = i / K, k = i % K;
    coarse[i] = 0.5 * (fine[(2 * jc) * K + k] + fine[(2 * jc + 1) * K + k]);
  }
}

__global__ void k_prolong_add(double* __restrict__ fine, const double* __restrict__ fc, const double* __restrict__ fc0,
                              long long K, long long n) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  for (; i < n; i += (long long)gridDim.x * blockDim.x) {
    long long jc = i / K, k = i % K;
    double d = fc[i] - fc0[i];
    fine[(2 * jc) * K + k] += d;
    fine[(2 * jc + 1) * K + k] += d;
  }
}

__global__ void k_restrict2d(const double* __restrict__ fine, double* __restrict__ coarse, long long K, int nx,
                             long long n) {
  const int cx = nx / 2;
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  for (; i < n; i += (long long)gridDim.x * blockDim.x) {
    long long c = i / K, k = i % K;
    long long ic = c % cx, jc = c / cx;
    long long f00 = (2 * jc) * nx + 2 * ic;
    coarse[i] = 0.25 * (fine[f00 * K + k] + fine[(f00 + 1) * K + k] + fine[(f00 + nx) * K + k] +
                        fine[(f00 + nx + 1) * K + k]);
  }
}

__global__ void k_prolong_add2d(double* __restrict__ fine, const double* __restrict__ fc,
                                const double* __restrict__ fc0, long long K, int nx, long long n) {
  const int cx = nx / 2;
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  for (; i < n; i += (long long)gridDim.x * blockDim.x) {
    long long c = i / K, k = i % K;
    long long ic = c % cx, jc = c / cx;
    long long f00 = (2 * jc) * nx + 2 * ic;
    double d = fc[i] - fc0[i];
    fine[f00 * K + k] += d;
    fine[(f00 + 1) * K + k] += d;
    fine[(f00 + nx) * K + k] += d;
    fine[(f00 + nx + 1) * K + k] += d;
  }
}

__global__ void k_axpby(double* __restrict__ y, const double* __restrict__ x, double a, double b, long long n) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  for (; i < n; i += (long long)gridDim.x * blockDim.x) y[i] = a * y[i] + b * x[i];
}

static int blocks_for(long long n) {
  long long b = (n + 255) / 256;
  return (int)(b < 152 * 16 ? b : 152 * 16);
}

cudaError_t launch_restrict(const double* fine, double* coarse, long long K, int Jc, cudaStream_t st) {
  long long n = K * Jc;
  k_restrict<<<blocks_for(n), 256, 0, st>>>(fine, coarse, K, n);
  return cudaGetLastError();
}

cudaError_t launch_prolong_add(double* fine, const double* fc, const double* fc0, long long K, int Jc, cudaStream_t st) {
  long long n = K * Jc;
  k_prolong_add<<<blocks_for(n), 256, 0, st>>>(fine, fc, fc0, K, n);
  return cudaGetLastError();
}

cudaError_t launch_restrict2d(const double* fine, double* coarse, long long K, int nx, int ny, cudaStream_t st) {
  long long n = K * (nx / 2) * (ny / 2);
  k_restrict2d<<<blocks_for(n), 256, 0, st>>>(fine, coarse, K, nx, n);
  return cudaGetLastError();
}

cudaError_t launch_prolong_add2d(double* fine, const double* fc, const double* fc0, long long K, int nx, int ny,
                                 cudaStream_t st) {
  long long n = K * (nx / 2) * (ny / 2);
  k_prolong_add2d<<<blocks_for(n), 256, 0, st>>>(fine, fc, fc0, K, nx, n);
  return cudaGetLastError();
}

cudaError_t launch_axpby(double* y, const double* x, double a, double b, long long n, cudaStream_t st) {
  k_axpby<<<blocks_for(n), 256, 0, st>>>(y, x, a, b, n);
  return cudaGetLastError();
}


// ---------------------------------------------------------------------------------------
// Per-instance activity flags of a batch: an instance whose residual is below tol is
// converged and its scans are skipped (a non-finite residual keeps it active).
// ---------------------------------------------------------------------------------------
__global__ void k_update_active(const double* res, int n, double tol, int* active) {
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q < n) active[q] = res[q] < tol ? 0 : 1;
}

__global__ void k_fill_int(int* p, int n, int v) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = v;
}

cudaError_t launch_update_active(const double* res, int n, double tol, int* active, cudaStream_t st) {
  k_update_active<<<(n + 127) / 128, 128, 0, st>>>(res, n, tol, active);
  return cudaGetLastError();
}

cudaError_t launch_fill_int(int* p, int n, int value, cudaStream_t st) {
  k_fill_int<<<(n + 127) / 128, 128, 0, st>>>(p, n, value);
  return cudaGetLastError();
}

}  // namespace sgs
