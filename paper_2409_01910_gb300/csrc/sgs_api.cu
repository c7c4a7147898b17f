// Host side of the C ABI declared in include/sgs.h: problem validation, velocity-grid and
// Fourier-weight tables, work planning of the spectral sum, workspace layout and the
// enqueueing of kernels on the caller's stream.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "common.cuh"
#include "kernels.h"

using namespace sgs;

namespace {

constexpr size_t kAlign = 256;
size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

// ---------------------------------------------------------------------------------------
// Fourier weight of the collision integral, closed form of
//   G(a, b) = 16 pi^2 int_0^{2R} rho^2 B(rho) sinc(c a rho) sinc(c b rho) drho,  c = pi/(2L),
// for B = b0 (Maxwell molecules) and B = b0 rho (hard spheres); a, b given by their
// squares (integers). Products of sines integrate in closed form.
// ---------------------------------------------------------------------------------------
double radial_I0(double om, double R) {  // int_0^R cos(om x) dx
  return om == 0.0 ? R : std::sin(om * R) / om;
}
double radial_I1(double om, double R) {  // int_0^R x cos(om x) dx
  if (om == 0.0) return 0.5 * R * R;
  double s = std::sin(0.5 * om * R);
  return R * std::sin(om * R) / om - 2.0 * s * s / (om * om);
}
double radial_sin2(double A, double R) {  // int_0^R x^2 sin(A x) / A dx  (A > 0): the b = 0 case, Maxwell
  return (std::sin(A * R) / (A * A) - R * std::cos(A * R) / A) / A;
}
double radial_sin3(double A, double R) {  // int_0^R x^2 sin(A x) / A dx (A > 0): the b = 0 case, hard spheres
  double AR = A * R, hh = std::sin(0.5 * AR);
  return (-R * R * std::cos(AR) / A + 2.0 * R * std::sin(AR) / (A * A) - 4.0 * hh * hh / (A * A * A)) / A;
}

double weight_G(int N, double L, int collision, double b0, long long a2, long long b2) {
  (void)N;
  const double pi = kPi;
  double R2 = 2.0 * (2.0 * L / (3.0 * std::sqrt(2.0) + 1.0));
  double c = pi / (2.0 * L);
  double Kc = 16.0 * pi * pi * b0;
  double a = std::sqrt((double)a2), b = std::sqrt((double)b2);
  bool hs = collision == SGS_HARD_SPHERE;
  if (a2 == 0 && b2 == 0) return hs ? Kc * std::pow(R2, 4) / 4.0 : Kc * R2 * R2 * R2 / 3.0;
  if (a2 == 0 || b2 == 0) {
    double A = c * (a2 == 0 ? b : a);
    return hs ? Kc * radial_sin3(A, R2) : Kc * radial_sin2(A, R2);
  }
  double A = c * a, B = c * b;
  // sinc(A x) sinc(B x) = [cos((A-B)x) - cos((A+B)x)] / (2 A B x^2)
  if (hs) return Kc / (2.0 * A * B) * (radial_I1(A - B, R2) - radial_I1(A + B, R2));
  return Kc / (2.0 * A * B) * (radial_I0(A - B, R2) - radial_I0(A + B, R2));
}

bool valid_nv(int N) { return N >= 8 && N <= 32 && N % 4 == 0; }

// Decompositions of the spectral sum: about kSumBlocks blocks of NW warps (NW lane groups) by
// default; the autotuner tries every NW in 1, 2, 4 with each block count of kSumBlockChoices.
constexpr int kSumBlocks = 3000;
constexpr int kSumBlockChoices[3] = {1500, 3000, 6000};
constexpr int kSumMaxWarps = 4;

struct Unit {
  int k1, k2, m1lo, m1hi;
  long long step0;
  int steps;
  int row;
};

}  // namespace

struct sgs_handle {
  int n_inst = 0, N = 0, n = 0, H = 0, precision = SGS_FP64;
  int C = 0, G = 0;
  double L = 0.0, dv = 0.0;
  long long field = 0;
  bool spectral = true;  // false when every instance uses BGK
  std::vector<sgs_problem> prob;
  std::vector<InstDev> inst;
  std::vector<long long> cell_off;
  std::vector<int> cell_inst;
  // spectral-sum plan
  std::vector<Unit> units;  // launch order
  std::vector<int2> row_k;
  std::vector<int> row_start, row_units;
  long long steps = 0;
  int NW = 1, PW64 = 0, PW32 = 0;
  long long sum_total = 0;  // steps of the whole sum
  int U_cap = 0;            // largest unit count of any decomposition (sizes the partial buffers)
  int sum_blocks = 0;       // block count the current decomposition was planned for
  // tables
  std::vector<double> tw_cos, tw_sin, Gtab, Lo;
  long long na = 0, nb = 0;
  // workspace
  size_t ws_bytes = 0;
  char* ws = nullptr;
  struct {
    size_t inst, cell_off, cell_inst, cnt, theta, nu, scratch, tw_cos, tw_sin, G, Lo, units, step0, row_k, row_start,
        row_units, W64, W32, st1a, st1b, st2a, st2b, ahat, bhat, qhat, partial, partial2, f_ref, Q_ref, theta_ref,
        ahat_ref, active, W32lo, tw_cos32, tw_sin32, efac, efac_ref, cproj_A, mom, sflux, o2rhs, end;
  } off;
  int cproj = 0;  // conservation projection of Q after every spectral collision step (mode 1 or 2)
  bool order2 = false;  // second-order reconstruction (1-D)
  bool dc_ref = false;  // FP32 collisions use the increment form against the stored reference
  int dc_prec = SGS_DF64;  // arithmetic of the high-precision evaluation in sgs_dc_step
  bool two_d = false;      // 2-D space: one instance, wavefront scans, four orderings
  // multigrid levels: lev[0] is the bound grid (tables at off.inst, off.cell_off, off.cell_inst);
  // level l has every instance's cell count halved l times and its own tables and fields
  struct Level {
    int C = 0, G = 0;
    size_t inst = 0, cell_off = 0, cell_inst = 0, f = 0, f0 = 0, b = 0, Q = 0, P = 0, R = 0;
    // increment-form reference of this level (f_ref, Q_ref, theta_ref, ahat_ref); on coarse
    // levels the restricted iterate I f and its FP32 collision operator
    size_t rf = 0, rQ = 0, rth = 0, rah = 0;
    bool ref = false;
    InstDev hinst0;  // host copy of instance 0 on this level (2-D grid sizes)
    std::vector<InstDev> hinst;
    std::vector<long long> hcell_off;
    std::vector<int> hcell_inst;
  };
  std::vector<Level> lev;
  SweepShape sweep{8, 1, 256};
  int sweep_arith = kSweepF64;
  // profiling: per-class CUDA-event pairs recorded on the launching stream
  bool prof = false;
  struct Rec {
    int cls;
    cudaEvent_t a, b;
    double work;  // cells the bracketed launches evaluated (sums) or visited (scans)
  };
  std::vector<Rec> recs;
  std::vector<cudaEvent_t> pool;
  unsigned long long launches = 0;
  long long spin_max = 1LL << 26;
  // pipelined iterations: the scans run on a high-priority stream of the handle while the
  // collision steps of the groups the scan has left run on the caller's stream
  bool overlap = true;
  cudaStream_t scan_st = nullptr;
  std::vector<cudaEvent_t> ov_ev;

  template <typename T>
  T* at(size_t o) const {
    return reinterpret_cast<T*>(ws + o);
  }
};

namespace {

// Inverse of the Gram matrix A = sum_k phi(v_k) phi(v_k)^T, phi = (1, v1, v2, v3, |v|^2), over
// the N^3 velocity nodes (conservation projection), by Gauss-Jordan elimination with
// partial pivoting in FP64. False if A is singular.
bool gram_inverse(int N, double dv, double* Ainv) {
  double A[5][10];
  memset(A, 0, sizeof(A));
  for (int i1 = 0; i1 < N; i1++)
    for (int i2 = 0; i2 < N; i2++)
      for (int i3 = 0; i3 < N; i3++) {
        double v1 = (i1 - N / 2 + 1) * dv, v2 = (i2 - N / 2 + 1) * dv, v3 = (i3 - N / 2 + 1) * dv;
        double ph[5] = {1.0, v1, v2, v3, v1 * v1 + v2 * v2 + v3 * v3};
        for (int a = 0; a < 5; a++)
          for (int b = 0; b < 5; b++) A[a][b] += ph[a] * ph[b];
      }
  for (int a = 0; a < 5; a++) A[a][5 + a] = 1.0;
  for (int col = 0; col < 5; col++) {
    int piv = col;
    for (int r = col + 1; r < 5; r++)
      if (std::fabs(A[r][col]) > std::fabs(A[piv][col])) piv = r;
    if (!(std::fabs(A[piv][col]) > 0.0)) return false;
    if (piv != col)
      for (int k = 0; k < 10; k++) std::swap(A[piv][k], A[col][k]);
    double d = A[col][col];
    for (int k = 0; k < 10; k++) A[col][k] /= d;
    for (int r = 0; r < 5; r++) {
      if (r == col) continue;
      double m = A[r][col];
      for (int k = 0; k < 10; k++) A[r][k] -= m * A[col][k];
    }
  }
  for (int a = 0; a < 5; a++)
    for (int b = 0; b < 5; b++) Ainv[a * 5 + b] = A[a][5 + b];
  return true;
}

// Work units of the spectral sum: each row (k1, k2) of the Hermitian half split into m1
// ranges of about `cap` steps. The steps are numbered row by row and m1 by m1 whatever the
// split, so the weight blocks (built per step) stay valid for every decomposition.
long long sum_target(const sgs_handle* h, int nw, int blocks) {
  int blocks_y = (h->G + nw - 1) / nw;
  return std::max(1LL, (long long)blocks / blocks_y);
}

int plan_units(sgs_handle* h, long long target_units) {
  const int n = h->n, H = h->H;
  const int n_rows = (int)h->row_k.size();
  long long cap = std::max<long long>(n, h->sum_total / target_units);
  std::vector<Unit> u;
  long long step = 0;
  for (int r = 0; r < n_rows; r++) {
    int k1 = h->row_k[r].x, k2 = h->row_k[r].y;
    int m1lo = std::max(-H, k1 - H), m1hi = std::min(H, k1 + H);
    int nm2 = n - std::abs(k2);
    int per = (int)std::max(1LL, cap / nm2);
    for (int m = m1lo; m <= m1hi; m += per) {
      Unit x;
      x.k1 = k1;
      x.k2 = k2;
      x.m1lo = m;
      x.m1hi = std::min(m1hi, m + per - 1);
      x.steps = (x.m1hi - x.m1lo + 1) * nm2;
      x.step0 = step;
      x.row = r;
      step += x.steps;
      u.push_back(x);
    }
  }
  h->steps = step;
  // longest units first
  std::stable_sort(u.begin(), u.end(), [](const Unit& a, const Unit& b) { return a.steps > b.steps; });
  h->units = u;
  h->row_start.assign(n_rows + 1, 0);
  for (auto& x : u) h->row_start[x.row + 1]++;
  for (int r = 0; r < n_rows; r++) h->row_start[r + 1] += h->row_start[r];
  h->row_units.assign(u.size(), 0);
  std::vector<int> fill(h->row_start.begin(), h->row_start.end() - 1);
  // within a row, partials are summed in m1 order
  std::vector<int> order(u.size());
  for (size_t i = 0; i < u.size(); i++) order[i] = (int)i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    return u[a].row != u[b].row ? u[a].row < u[b].row : u[a].m1lo < u[b].m1lo;
  });
  for (int i : order) h->row_units[fill[u[i].row]++] = i;
  return (int)u.size();
}

int plan(sgs_handle* h) {
  int N = h->N, n = N - 1, H = N / 2 - 1;
  h->n = n;
  h->H = H;
  h->G = (h->C + kLanes - 1) / kLanes;
  h->NW = h->G >= 2 ? 2 : 1;
  h->PW64 = sum_pad(H, 8);
  h->PW32 = sum_pad(H, 4);
  // twiddles: angle 2 pi ((k j) mod N) / N, k in [-H, H], j = i - N/2 + 1
  h->tw_cos.assign((size_t)n * N, 0.0);
  h->tw_sin.assign((size_t)n * N, 0.0);
  for (int k = -H; k <= H; k++)
    for (int i = 0; i < N; i++) {
      long long kj = ((long long)k * (i - N / 2 + 1)) % N;
      if (kj < 0) kj += N;
      double ang = 2.0 * kPi * (double)kj / N;
      h->tw_cos[(size_t)(k + H) * N + i] = std::cos(ang);
      h->tw_sin[(size_t)(k + H) * N + i] = std::sin(ang);
    }
  if (!h->spectral) return SGS_OK;
  const sgs_problem& p0 = h->prob[0];
  h->na = 3LL * H * H + 1;
  h->nb = 12LL * H * H + 1;
  h->Gtab.resize((size_t)(h->na * h->nb));
  h->Lo.resize((size_t)h->na);
  for (long long a2 = 0; a2 < h->na; a2++) {
    for (long long b2 = 0; b2 < h->nb; b2++)
      h->Gtab[(size_t)(a2 * h->nb + b2)] = weight_G(N, p0.v_max, p0.collision, p0.b0, a2, b2);
    h->Lo[(size_t)a2] = weight_G(N, p0.v_max, p0.collision, p0.b0, 4 * a2, 0);
  }
  // rows of the Hermitian half: k1 > 0, or k1 == 0 and k2 >= 0
  long long total = 0;
  for (int k1 = 0; k1 <= H; k1++)
    for (int k2 = -H; k2 <= H; k2++) {
      if (k1 == 0 && k2 < 0) continue;
      int m1lo = std::max(-H, k1 - H), m1hi = std::min(H, k1 + H);
      int nm2 = n - std::abs(k2);
      total += (long long)(m1hi - m1lo + 1) * nm2;
      h->row_k.push_back(make_int2(k1, k2));
    }
  h->sum_total = total;
  // default decomposition: about kSumBlocks blocks in the launch; the partial buffers are sized
  // for the largest unit count the autotuner may try
  h->U_cap = 0;
  for (int nw = 1; nw <= kSumMaxWarps; nw *= 2)
    for (int bl : kSumBlockChoices) h->U_cap = std::max(h->U_cap, plan_units(h, sum_target(h, nw, bl)));
  h->NW = h->G >= 2 ? 2 : 1;
  h->sum_blocks = kSumBlocks;
  plan_units(h, sum_target(h, h->NW, h->sum_blocks));
  h->U_cap = std::max(h->U_cap, (int)h->units.size());
  return SGS_OK;
}

void layout(sgs_handle* h) {
  size_t o = 0;
  auto take = [&](size_t bytes) {
    size_t r = o;
    o = align_up(o + bytes);
    return r;
  };
  int N = h->N, n = h->n, C = h->C, G = h->G;
  auto& f = h->off;
  f.inst = take(sizeof(InstDev) * h->n_inst);
  f.cell_off = take(sizeof(long long) * C);
  f.cell_inst = take(sizeof(int) * C);
  f.cnt = take(sizeof(Counters) * h->n_inst);
  f.active = take(sizeof(int) * h->n_inst);
  f.theta = take(sizeof(double) * 5 * C);
  f.nu = take(sizeof(double) * C);
  // per instance: 2 wall fluxes; per cell: residual partial and mass; 2-D: one outgoing
  // flux per boundary face
  f.scratch = take(sizeof(double) * (2 * h->n_inst + 2 * C + 2 * (h->inst[0].nx + h->inst[0].ny) + 64));
  f.tw_cos = take(sizeof(double) * n * N);
  f.tw_sin = take(sizeof(double) * n * N);
  f.tw_cos32 = take(sizeof(float) * n * N);
  f.tw_sin32 = take(sizeof(float) * n * N);
  f.efac = take(sizeof(double) * 3 * kMaxN * C);      // per-cell Maxwellian factors (finest level
  f.efac_ref = take(sizeof(double) * 3 * kMaxN * C);  // is the largest) and those of the reference
  f.cproj_A = take(h->cproj == 1 ? sizeof(double) * 25 : 0);  // inverse Gram matrix of (1, v, |v|^2)
  f.mom = take(h->cproj ? sizeof(double) * 5 * (size_t)C * N : 0);  // moments of Q per (cell, i1) slab
  f.sflux = take(h->order2 ? sizeof(double) * (h->two_d ? 2 * (h->inst[0].nx + h->inst[0].ny) : 2 * h->n_inst)
                           : 0);                                     // second order: wall slope fluxes
  f.o2rhs = take(h->order2 ? sizeof(double) * h->field : 0);         // second order: scan right-hand side
  bool sp = h->spectral;
  size_t U = (size_t)std::max<int>(h->U_cap, (int)h->units.size());
  f.G = take(sp ? sizeof(double) * h->na * h->nb : 0);
  f.Lo = take(sp ? sizeof(double) * h->na : 0);
  f.units = take(sizeof(int4) * U);
  f.step0 = take(sizeof(long long) * U);
  f.row_k = take(sizeof(int2) * h->row_k.size());
  f.row_start = take(sizeof(int) * h->row_start.size());
  f.row_units = take(sizeof(int) * U);
  f.W64 = take(sp ? sizeof(double) * h->steps * h->PW64 : 0);
  f.W32 = take(sp && h->precision == SGS_FP32 ? sizeof(float) * h->steps * h->PW32 : 0);
  size_t cpl = sizeof(double2);
  size_t spec = sp ? (size_t)G * n * n * n * kLanes * cpl : 0;
  f.st1a = take(sp ? (size_t)C * N * N * n * cpl : 0);
  f.st1b = take(sp ? (size_t)C * N * N * n * cpl : 0);
  f.st2a = take(sp ? (size_t)C * N * n * n * cpl : 0);
  f.st2b = take(sp ? (size_t)C * N * n * n * cpl : 0);
  f.ahat = take(spec);
  f.bhat = take(spec);
  f.qhat = take(spec);
  f.partial = take(sp ? U * G * n * kLanes * cpl : 0);
  // defect-correction reference state (mixed precision only)
  bool dc = sp && h->precision == SGS_FP32;
  f.partial2 = take(dc ? U * G * n * kLanes * sizeof(float2) : 0);
  f.f_ref = take(dc ? sizeof(double) * h->field : 0);
  f.Q_ref = take(dc ? sizeof(double) * h->field : 0);
  f.theta_ref = take(dc ? sizeof(double) * 5 * C : 0);
  f.ahat_ref = take(dc ? (size_t)G * n * n * n * kLanes * sizeof(float2) : 0);
  f.W32lo = take(dc ? sizeof(float) * h->steps * h->PW32 : 0);
  size_t K = (size_t)N * N * N;
  int nl = (int)h->lev.size();
  for (int l = 0; l < nl; l++) {
    auto& L = h->lev[l];
    if (l == 0) {
      L.inst = f.inst;
      L.cell_off = f.cell_off;
      L.cell_inst = f.cell_inst;
    } else {
      L.inst = take(sizeof(InstDev) * h->n_inst);
      L.cell_off = take(sizeof(long long) * L.C);
      L.cell_inst = take(sizeof(int) * L.C);
      L.f = take(sizeof(double) * K * L.C);
      L.f0 = take(sizeof(double) * K * L.C);
      L.b = take(sizeof(double) * K * L.C);
      L.Q = take(sizeof(double) * K * L.C);
      L.P = take(sizeof(double) * K * L.C);
    }
    if (l == 0) {
      L.rf = f.f_ref;
      L.rQ = f.Q_ref;
      L.rth = f.theta_ref;
      L.rah = f.ahat_ref;
    } else {
      L.rf = L.f0;
      L.rQ = take(dc ? sizeof(double) * K * L.C : 0);
      L.rth = take(dc ? sizeof(double) * 5 * L.C : 0);
      L.rah = take(dc ? (size_t)L.G * n * n * n * kLanes * sizeof(float2) : 0);
    }
    if (l + 1 < nl) L.R = take(sizeof(double) * K * L.C);
  }
  f.end = o;
  h->ws_bytes = o;
}

}  // namespace

// Problem validation shared by every entry point that takes a problem description.
int sgs::check_problem(const sgs_problem& p) {
  if (p.space_dim != 1 && p.space_dim != 2) return SGS_ERR_ARG;
  if (p.nx < 1 || !(p.x_hi > p.x_lo)) return SGS_ERR_ARG;
  if (p.space_dim == 2) {
    if (p.ny < 1 || !(p.y_hi > p.y_lo)) return SGS_ERR_ARG;
    for (int s = 2; s < 4; s++) {
      if (p.bc[s].kind != SGS_DIFFUSE && p.bc[s].kind != SGS_INFLOW) return SGS_ERR_ARG;
      if (!(p.bc[s].T > 0.0)) return SGS_ERR_ARG;
      if (p.bc[s].kind == SGS_INFLOW && !(p.bc[s].rho > 0.0)) return SGS_ERR_ARG;
      if (p.bc[s].kind == SGS_DIFFUSE && p.bc[s].u[1] != 0.0) return SGS_ERR_UNSUPPORTED;  // tangential walls
    }
  }
  if (!valid_nv(p.nv) || !(p.v_max > 0.0)) return SGS_ERR_ARG;
  if (p.collision < SGS_MAXWELL || p.collision > SGS_BGK) return SGS_ERR_ARG;
  if (!(p.b0 > 0.0) || !(p.eps > 0.0)) return SGS_ERR_ARG;
  if (p.precision != SGS_FP64 && p.precision != SGS_FP32) return SGS_ERR_ARG;
  if (p.inner_method != SGS_PFP && p.inner_method != SGS_FP && p.inner_method != SGS_PFP_RELAX) return SGS_ERR_ARG;
  if (p.inner_max < 0 || p.inner_fixed < 0 || p.newton_max < 1) return SGS_ERR_ARG;
  if (p.conserve_proj < 0 || p.conserve_proj > 2) return SGS_ERR_ARG;
  if (p.order < 0 || p.order > 2) return SGS_ERR_ARG;
  for (int s = 0; s < 2; s++) {
    if (p.bc[s].kind != SGS_DIFFUSE && p.bc[s].kind != SGS_INFLOW) return SGS_ERR_ARG;
    if (!(p.bc[s].T > 0.0)) return SGS_ERR_ARG;
    if (p.bc[s].kind == SGS_INFLOW && !(p.bc[s].rho > 0.0)) return SGS_ERR_ARG;
    if (p.bc[s].kind == SGS_DIFFUSE && p.bc[s].u[0] != 0.0) return SGS_ERR_UNSUPPORTED;  // tangential walls only
  }
  return SGS_OK;
}

// Device description of one instance: cell sizes, solver controls and the unit wall
// Maxwellians with their discrete zero-mass-flux normalisation.
void sgs::fill_inst(const sgs_problem& p, int N, double dv, InstDev& I) {
  memset(&I, 0, sizeof(I));
  const bool two_d = p.space_dim == 2;
  I.space_dim = two_d ? 2 : 1;
  I.nx = p.nx;
  I.ny = two_d ? p.ny : 1;
  I.J = I.nx * I.ny;
  I.collision = p.collision;
  I.dx = (p.x_hi - p.x_lo) / p.nx;
  I.dy = two_d ? (p.y_hi - p.y_lo) / p.ny : 1.0;
  I.eps = p.eps;
  I.b0 = p.b0;
  I.total_mass = p.total_mass;
  I.inner_tol = p.inner_tol;
  I.inner_max = p.inner_max;
  I.inner_fixed = p.inner_fixed;
  I.inner_method = p.inner_method;
  I.newton_max = p.newton_max;
  I.newton_tol = p.newton_tol;
  double w = dv * dv * dv;
  for (int s = 0; s < (two_d ? 4 : 2); s++) {
    const sgs_bc& b = p.bc[s];
    const int dn = s < 2 ? 0 : 1;  // normal velocity component of the side
    I.bc_kind[s] = b.kind;
    I.bc_rho[s] = b.rho;
    double T = b.T;
    double norm = 1.0 / (2.0 * kPi * T * std::sqrt(2.0 * kPi * T));
    for (int d = 0; d < 3; d++)
      for (int i = 0; i < N; i++) {
        double v = node(i, N, dv);
        double x = std::exp(-(v - b.u[d]) * (v - b.u[d]) / (2.0 * T));
        if (d == 0) x *= norm;
        if (d == dn) {
          bool incoming = s % 2 == 0 ? v > 0.0 : v < 0.0;
          x = incoming ? x : 0.0;
        }
        I.wall[s][d][i] = x;
      }
    // sum over incoming v of w (v.n) Mhat with the normal component n of the side
    double sd[3] = {0.0, 0.0, 0.0};
    for (int d = 0; d < 3; d++)
      for (int i = 0; i < N; i++) sd[d] += (d == dn ? node(i, N, dv) : 1.0) * I.wall[s][d][i];
    I.wall_denom[s] = w * sd[0] * sd[1] * sd[2];
  }
}

namespace {

cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

int cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return SGS_OK;
  fprintf(stderr, "sgs: CUDA error: %s\n", cudaGetErrorString(e));
  return SGS_ERR_CUDA;
}

cudaEvent_t take_event(sgs_handle* h) {
  if (!h->pool.empty()) {
    cudaEvent_t e = h->pool.back();
    h->pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

// Counts the kernels a host call enqueues and, when profiling is on, brackets them with
// CUDA events on the same stream.
struct Scope {
  sgs_handle* h;
  int cls;
  cudaStream_t st;
  cudaEvent_t a = nullptr, b = nullptr;
  double work;
  Scope(sgs_handle* h_, int cls_, cudaStream_t st_, int n_launch, double work_ = 0.0)
      : h(h_), cls(cls_), st(st_), work(work_) {
    h->launches += n_launch;
    // launches captured into a CUDA graph are not timed: an event recorded during capture
    // becomes a graph node, not a timestamp
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (h->prof && cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusNone) {
      a = take_event(h);
      b = take_event(h);
      if (a && b) cudaEventRecord(a, st);
    }
  }
  ~Scope() {
    if (a && b) {
      cudaEventRecord(b, st);
      h->recs.push_back({cls, a, b, work});
    }
  }
};

AuxArgs aux_args(const sgs_handle* h, int l = 0) {
  const auto& L = h->lev[l];
  AuxArgs a;
  a.inst = h->at<InstDev>(L.inst);
  a.n_inst = h->n_inst;
  a.N = h->N;
  a.C = L.C;
  a.dv = h->dv;
  a.cell_off = h->at<long long>(L.cell_off);
  a.cell_inst = h->at<int>(L.cell_inst);
  a.scratch = h->at<double>(h->off.scratch);
  a.active = h->at<int>(h->off.active);
  a.two_d = h->two_d ? 1 : 0;
  a.nx = L.hinst0.nx;
  a.ny = L.hinst0.ny;
  a.sflux = h->order2 ? h->at<double>(h->off.sflux) : nullptr;
  return a;
}

// The collision step skips the cells of converged (inactive) instances of multi-instance
// handles: their f no longer changes, so the Q and P of their last evaluation stay valid.
CellTables cell_tables(const sgs_handle* h, int l = 0) {
  const auto& L = h->lev[l];
  CellTables ct;
  ct.inst = h->at<InstDev>(L.inst);
  ct.cell_off = h->at<long long>(L.cell_off);
  ct.cell_inst = h->at<int>(L.cell_inst);
  ct.active = h->n_inst > 1 ? h->at<int>(h->off.active) : nullptr;
  return ct;
}

// Collision context of level l restricted to the lane groups [g_lo, g_hi) (g_hi < 0: all):
// every per-cell and per-group pointer starts at the range's first cell and group, so the
// kernels index cells and groups relative to the range; the partial sums keep the level's
// group stride.
template <typename T>
CollideCtx<T> collide_ctx(const sgs_handle* h, int l = 0, int g_lo = 0, int g_hi = -1) {
  typedef typename CplxOf<T>::type CT;
  const int Gl = h->lev[l].G, Cl = h->lev[l].C;
  if (g_hi < 0) g_hi = Gl;
  const int c0 = g_lo * kLanes, c1 = std::min(g_hi * kLanes, Cl);
  const int N = h->N, n = h->n;
  const size_t gsz = (size_t)n * n * n * kLanes;
  CollideCtx<T> x;
  x.N = N;
  x.C = c1 - c0;
  x.H = h->H;
  x.NW = std::min(h->NW, g_hi - g_lo);
  x.n_units = (int)h->units.size();
  x.dv = h->dv;
  x.ct = cell_tables(h, l);
  x.ct.cell_off += c0;
  x.ct.cell_inst += c0;
  x.theta = h->at<double>(h->off.theta) + 5 * (size_t)c0;
  x.nu = h->at<double>(h->off.nu) + c0;
  x.sb.tw_cos = h->at<double>(h->off.tw_cos);
  x.sb.tw_sin = h->at<double>(h->off.tw_sin);
  x.sb.twc = sizeof(T) == 8 ? h->at<T>(h->off.tw_cos) : h->at<T>(h->off.tw_cos32);
  x.sb.tws = sizeof(T) == 8 ? h->at<T>(h->off.tw_sin) : h->at<T>(h->off.tw_sin32);
  x.efac = h->at<double>(h->off.efac) + (size_t)3 * kMaxN * c0;
  x.efac_ref = h->at<double>(h->off.efac_ref) + (size_t)3 * kMaxN * c0;
  x.mom = h->cproj ? h->at<double>(h->off.mom) + (size_t)5 * N * c0 : nullptr;
  x.cproj = h->cproj == 1 ? h->at<double>(h->off.cproj_A) : nullptr;
  x.cproj_mode = h->cproj;
  x.sb.st1a = h->at<CT>(h->off.st1a) + (size_t)c0 * N * N * n;
  x.sb.st1b = h->at<CT>(h->off.st1b) + (size_t)c0 * N * N * n;
  x.sb.st2a = h->at<CT>(h->off.st2a) + (size_t)c0 * N * n * n;
  x.sb.st2b = h->at<CT>(h->off.st2b) + (size_t)c0 * N * n * n;
  x.sb.ahat = h->at<CT>(h->off.ahat) + g_lo * gsz;
  x.sb.bhat = h->at<CT>(h->off.bhat) + g_lo * gsz;
  x.sb.qhat = h->at<CT>(h->off.qhat) + g_lo * gsz;
  x.sum.units = h->at<int4>(h->off.units);
  x.sum.unit_step0 = h->at<long long>(h->off.step0);
  x.sum.W = sizeof(T) == 8 ? h->at<T>(h->off.W64) : h->at<T>(h->off.W32);
  x.sum.ahat = x.sb.ahat;
  x.sum.bhat = x.sb.bhat;
  x.sum.partial = h->at<CT>(h->off.partial) + (size_t)g_lo * n * kLanes;
  x.sum.G = g_hi - g_lo;
  x.sum.Gs = Gl;
  x.sum.cnt = h->at<Counters>(h->off.cnt);
  x.sum.spin_max = h->spin_max;
  x.sb.cell_inst = x.ct.cell_inst;
  x.sb.active = x.ct.active;
  x.sum.cell_inst = x.ct.cell_inst;
  x.sum.active = x.ct.active;
  x.sum.C = x.C;
  x.red.row_k = h->at<int2>(h->off.row_k);
  x.red.row_start = h->at<int>(h->off.row_start);
  x.red.row_units = h->at<int>(h->off.row_units);
  x.red.partial = x.sum.partial;
  x.red.qhat = x.sb.qhat;
  x.red.n = h->n;
  x.red.G = g_hi - g_lo;
  x.red.Gs = Gl;
  x.red.n_rows = (int)h->row_k.size();
  return x;
}

// Qraw (non-null only with the conservation projection): receives the unprojected operator,
// the reference of the increment form. The projection of mode 2 depends on f through M, so
// the increment form adds increments to the unprojected reference and projects the sum.
//
// [g_lo, g_hi): the lane groups (32 consecutive cells each) to evaluate; g_hi < 0 means every
// group of the level. Cells outside the range are neither read nor written.
int collide_impl(sgs_handle* h, const double* f, double* Q, double* P, int precision, cudaStream_t st, int l = 0,
                 double* Qraw = nullptr, int g_lo = 0, int g_hi = -1) {
  if (g_hi < 0) g_hi = h->lev[l].G;
  const int c0 = g_lo * kLanes;
  CellTables ct = cell_tables(h, l);
  ct.cell_off += c0;
  ct.cell_inst += c0;
  const int C = std::min(g_hi * kLanes, h->lev[l].C) - c0;
  double* theta = h->at<double>(h->off.theta) + 5 * (size_t)c0;
  double* nu = h->at<double>(h->off.nu) + c0;
  const sgs_problem& p0 = h->prob[0];
  cudaError_t e;
  {
    Scope sc(h, SGS_PROF_MOMENTS, st, 1);
    e = launch_moments(f, ct, C, h->N, h->dv, p0.newton_tol, p0.newton_max, theta, nu,
                       h->at<Counters>(h->off.cnt), st);
  }
  if (e != cudaSuccess) return cuda_status(e);
  if (!h->spectral) {
    Scope sc(h, SGS_PROF_REDUCE_IDFT, st, 1);
    return cuda_status(launch_collide_bgk(f, ct, C, h->N, h->dv, theta, nu, Q, P, st));
  }
  auto run = [&](auto x) -> int {
    cudaError_t er;
    {
      Scope sc(h, SGS_PROF_DFT, st, 4);
      er = launch_dft(f, x, DftMode{0, nullptr, nullptr}, st);
    }
    if (er != cudaSuccess) return cuda_status(er);
    {
      Scope sc(h, precision == SGS_FP64 ? SGS_PROF_SUM_FP64 : SGS_PROF_SUM, st, 1, x.C);
      er = launch_spectral_sum(x, nullptr, st);
    }
    if (er != cudaSuccess) return cuda_status(er);
    Scope sc(h, SGS_PROF_REDUCE_IDFT, st, h->cproj ? 5 : 4);
    return cuda_status(launch_reduce_idft(f, Q, P, x, nullptr, nullptr, st, Qraw));
  };
  // Increment form against the reference f_ref (defect correction): with a = f - M, b = f + M,
  //   Q(f) = Q_ref + Q_s(a - a_ref, b) + Q_s(a_ref, b - b_ref)   (exact: Q_s is bilinear),
  // both sums in FP32 on small increments, so the rounding error vanishes as f -> f_ref.
  auto run_inc = [&](CollideCtx<float> x) -> int {
    typedef float2 CT;
    const auto& Lv = h->lev[l];
    DftMode m1{1, h->at<double>(Lv.rf), h->at<double>(Lv.rth) + 5 * (size_t)c0};
    DftMode m2{2, m1.f_ref, m1.theta_ref};
    CT* part2 = h->at<CT>(h->off.partial2) + (size_t)g_lo * h->n * kLanes;
    cudaError_t er;
    {
      Scope sc(h, SGS_PROF_DFT, st, 5);
      er = launch_dft(f, x, m1, st);
    }
    if (er != cudaSuccess) return cuda_status(er);
    {
      Scope sc(h, SGS_PROF_SUM, st, 1, x.C);
      er = launch_spectral_sum(x, nullptr, st);
    }
    if (er != cudaSuccess) return cuda_status(er);
    {
      Scope sc(h, SGS_PROF_DFT, st, 5);
      er = launch_dft(f, x, m2, st);
      if (er == cudaSuccess)
        er = cudaMemcpyAsync(x.sb.ahat, h->at<CT>(Lv.rah) + (size_t)g_lo * h->n * h->n * h->n * kLanes,
                             (size_t)(g_hi - g_lo) * h->n * h->n * h->n * kLanes * sizeof(CT),
                             cudaMemcpyDeviceToDevice, st);
    }
    if (er != cudaSuccess) return cuda_status(er);
    {
      Scope sc(h, SGS_PROF_SUM, st, 1, x.C);
      er = launch_spectral_sum(x, part2, st);
    }
    if (er != cudaSuccess) return cuda_status(er);
    Scope sc(h, SGS_PROF_REDUCE_IDFT, st, h->cproj ? 5 : 4);
    return cuda_status(launch_reduce_idft(f, Q, P, x, part2, h->at<double>(Lv.rQ), st, Qraw));
  };
  if (precision == SGS_DF64) {
    if (h->precision != SGS_FP32) return SGS_ERR_ARG;  // FP32 tables not built
    CollideCtx<double> x = collide_ctx<double>(h, l, g_lo, g_hi);
    cudaError_t er;
    {
      Scope sc(h, SGS_PROF_DFT, st, 6);
      er = launch_dft(f, x, DftMode{0, nullptr, nullptr}, st);
      const long long cnt = (long long)(g_hi - g_lo) * h->n * h->n * h->n * kLanes;
      if (er == cudaSuccess) er = launch_split_spec(x.sb.ahat, cnt, st);
      if (er == cudaSuccess) er = launch_split_spec(x.sb.bhat, cnt, st);
    }
    if (er != cudaSuccess) return cuda_status(er);
    {
      Scope sc(h, SGS_PROF_SUM_DF64, st, 1, x.C);
      SumDfArgs d;
      d.units = x.sum.units;
      d.unit_step0 = x.sum.unit_step0;
      d.Whi = h->at<float>(h->off.W32);
      d.Wlo = h->at<float>(h->off.W32lo);
      d.ahat = reinterpret_cast<const float4*>(x.sb.ahat);
      d.bhat = reinterpret_cast<const float4*>(x.sb.bhat);
      d.partial = x.sum.partial;
      d.G = x.sum.G;
      d.Gs = x.sum.Gs;
      d.cnt = x.sum.cnt;
      d.cell_inst = x.sum.cell_inst;
      d.active = x.sum.active;
      d.C = x.sum.C;
      d.spin_max = x.sum.spin_max;
      er = launch_sum_df(d, h->H, x.n_units, st);
    }
    if (er != cudaSuccess) return cuda_status(er);
    Scope sc(h, SGS_PROF_REDUCE_IDFT, st, h->cproj ? 5 : 4);
    return cuda_status(launch_reduce_idft(f, Q, P, x, nullptr, nullptr, st, Qraw));
  }
  if (precision == SGS_FP32) {
    if (h->precision != SGS_FP32) return SGS_ERR_ARG;  // FP32 tables not built
    if (l == 0 ? h->dc_ref : h->lev[l].ref) return run_inc(collide_ctx<float>(h, l, g_lo, g_hi));
    return run(collide_ctx<float>(h, l, g_lo, g_hi));
  }
  return run(collide_ctx<double>(h, l, g_lo, g_hi));
}

// One scan: in 1-D dir +1 / -1 walks the cells forward / backward (ordering 0 / 1); in 2-D
// the ordering o in 0..3 is launched wavefront by wavefront.
// In 1-D, [s0, s1) limits the launch to those scan positions (a segment of the scan; first
// order only: the second-order slope terms are formed once per scan).
int sweep_impl(sgs_handle* h, double* f, const double* P, const double* rhs, int dir, cudaStream_t st, int l = 0,
               int ordering = -1, int s0 = 0, int s1 = 1 << 30) {
  SweepArgs a;
  a.s0 = s0;
  a.s1 = s1;
  a.inst = h->at<InstDev>(h->lev[l].inst);
  a.n_inst = h->n_inst;
  a.f = f;
  a.P = P;
  a.rhs = rhs;
  a.nu = h->at<double>(h->off.nu);
  a.cnt = h->at<Counters>(h->off.cnt);
  a.N = h->N;
  a.dv = h->dv;
  a.dir = dir;
  a.active = h->at<int>(h->off.active);
  a.theta = h->at<double>(h->off.theta);
  if (h->two_d) {
    const InstDev& I = h->lev[l].hinst0;
    const int o = ordering >= 0 ? ordering : (dir > 0 ? 0 : 1);
    const int nwf = I.nx + I.ny - 1;
    Scope sc(h, SGS_PROF_SWEEP, st, nwf + (h->order2 ? 2 : 0), (double)I.nx * I.ny);
    if (h->order2) {
      // second order: the slope terms and the face-value wall correction of this ordering
      // depend only on the state before it, so they join the right-hand side
      double* b2 = h->at<double>(h->off.o2rhs);
      cudaError_t e = launch_slope_rhs2d(aux_args(h, l), f, rhs, b2, st);
      if (e != cudaSuccess) return cuda_status(e);
      a.rhs = b2;
    }
    for (int wf = 0; wf < nwf; wf++) {
      int ncells = std::min(I.nx - 1, wf) - std::max(0, wf - (I.ny - 1)) + 1;
      cudaError_t e = launch_sweep2d(a, h->sweep, h->sweep_arith, o, wf, ncells, st);
      if (e != cudaSuccess) return cuda_status(e);
    }
    return SGS_OK;
  }
  double visits = 0.0;  // cells this launch visits (inactive instances included)
  for (const auto& I : h->lev[l].hinst.empty() ? h->inst : h->lev[l].hinst)
    visits += std::max(0, std::min(s1, I.J) - s0);
  Scope sc(h, SGS_PROF_SWEEP, st, h->order2 ? 3 : 1, visits);
  if (h->order2) {
    // second order: the explicit slope terms (and the face-value wall correction) of this
    // scan depend only on the state before it, so they join the right-hand side
    double* b2 = h->at<double>(h->off.o2rhs);
    cudaError_t e = launch_slope_rhs(aux_args(h, l), f, rhs, b2, st);
    if (e != cudaSuccess) return cuda_status(e);
    a.rhs = b2;
  }
  return cuda_status(launch_sweep(a, h->sweep, h->sweep_arith, st));
}

int rescale_impl(sgs_handle* h, double* f, cudaStream_t st) {
  Scope sc(h, SGS_PROF_RESCALE, st, 2);
  return cuda_status(launch_rescale(aux_args(h), f, st));
}

int residual_impl(sgs_handle* h, const double* f, const double* Q, const double* rhs, double* res, cudaStream_t st,
                  int l = 0) {
  Scope sc(h, SGS_PROF_RESIDUAL, st, res ? 3 : 2);
  return cuda_status(launch_residual(aux_args(h, l), f, Q, rhs, res, st));
}

int residual_field_impl(sgs_handle* h, const double* f, const double* Q, const double* rhs, double* R,
                        cudaStream_t st, int l) {
  Scope sc(h, SGS_PROF_RESIDUAL, st, 2);
  return cuda_status(launch_residual_field(aux_args(h, l), f, Q, rhs, R, st));
}

// Whether an SGS iteration of level l can pipeline its collision steps behind the scans: one
// 1-D instance of at least two lane groups, first order, spectral collisions, on the finest
// level, with the handle's scan stream available.
bool overlap_ok(const sgs_handle* h, int l) {
  return h->overlap && l == 0 && !h->two_d && h->n_inst == 1 && h->spectral && !h->order2 && h->lev[0].G >= 2 &&
         h->scan_st != nullptr && (int)h->ov_ev.size() >= 3 * h->lev[0].G + 2;
}

// One SGS iteration (eq. (29)) whose collision steps overlap the scans. The scans run on the
// handle's high-priority stream in segments of one lane group (32 cells), the collision
// steps on the caller's stream st, ordered by events (a fork/join pattern, also under stream
// capture):
//   - forward scan, group by group; the collision step of group g (the P^(n+1/2) the
//     backward scan needs) starts as soon as the forward scan has left group g;
//   - backward scan, groups G-1 .. 0, each segment after its group's collision step;
//   - with SGS_IT_EVAL, the collision step of the new iterate for group g >= 1 starts as
//     soon as the backward scan has left group g, and group 0 follows the mass rescale
//     (eq. (32)); the earlier groups' Q, P, nu and theta are carried over to the rescaled
//     state, whose operator they equal up to rounding (Q, P homogeneous of degree 2 in f).
// Each cell sees the same inputs as in iterate_impl's sequence of whole-grid steps.
int iterate_overlap(sgs_handle* h, double* f, double* Q, double* P, const double* rhs, int flags, double* res,
                    cudaStream_t st) {
  const int G = h->lev[0].G, J = h->inst[0].J, prec = h->precision;
  const bool eval = (flags & SGS_IT_EVAL) != 0;
  if (eval && !Q) return SGS_ERR_ARG;
  cudaStream_t ss = h->scan_st;
  int k = 0, r;
  cudaError_t e = cudaSuccess;
  // `to` waits for everything enqueued on `from` so far (either may be the legacy default
  // stream, whose handle is null)
  auto fork = [&](cudaStream_t from, cudaStream_t to) {
    cudaEvent_t x = h->ov_ev[k++];
    if (e == cudaSuccess) e = cudaEventRecord(x, from);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(to, x, 0);
  };
  if (!(flags & SGS_IT_P_VALID) && (r = collide_impl(h, f, nullptr, P, prec, st))) return r;
  fork(st, ss);
  for (int g = 0; g < G && e == cudaSuccess; g++) {
    if ((r = sweep_impl(h, f, P, rhs, +1, ss, 0, -1, g * kLanes, std::min((g + 1) * kLanes, J)))) return r;
    fork(ss, st);
    if ((r = collide_impl(h, f, nullptr, P, prec, st, 0, nullptr, g, g + 1))) return r;
  }
  for (int g = G - 1; g >= 0 && e == cudaSuccess; g--) {
    // the collision steps of groups < G-1 were enqueued earlier on st; one event covers them
    if (g == G - 1) fork(st, ss);
    const int c_lo = g * kLanes, c_hi = std::min((g + 1) * kLanes, J);
    if ((r = sweep_impl(h, f, P, rhs, -1, ss, 0, -1, J - c_hi, J - c_lo))) return r;
    if (g > 0 && eval) {
      fork(ss, st);
      if ((r = collide_impl(h, f, Q, P, prec, st, 0, nullptr, g, g + 1))) return r;
    }
  }
  fork(ss, st);  // join: every scan segment precedes what follows on st
  if (e != cudaSuccess) return cuda_status(e);
  if ((r = rescale_impl(h, f, st))) return r;
  if (eval) {
    {
      Scope sc(h, SGS_PROF_RESCALE, st, 1);
      e = launch_rescale_fixup(aux_args(h), kLanes, h->C, Q, P, h->at<double>(h->off.nu),
                               h->at<double>(h->off.theta), st);
      if (e != cudaSuccess) return cuda_status(e);
    }
    if ((r = collide_impl(h, f, Q, P, prec, st, 0, nullptr, 0, 1))) return r;
    if (res && (r = residual_impl(h, f, Q, rhs, res, st))) return r;
  }
  return SGS_OK;
}

int iterate_impl(sgs_handle* h, double* f, double* Q, double* P, const double* rhs, int flags, double* res,
                 cudaStream_t st, int l = 0) {
  if (overlap_ok(h, l)) return iterate_overlap(h, f, Q, P, rhs, flags, res, st);
  int r;
  if (!(flags & SGS_IT_P_VALID)) {
    r = collide_impl(h, f, nullptr, P, h->precision, st, l);
    if (r) return r;
  }
  if (h->two_d) {
    // the four corner-to-corner orderings, each after a collision evaluation
    for (int o = 0; o < 4; o++) {
      if (o > 0 && (r = collide_impl(h, f, nullptr, P, h->precision, st, l))) return r;
      if ((r = sweep_impl(h, f, P, rhs, 0, st, l, o))) return r;
    }
  } else {
    if ((r = sweep_impl(h, f, P, rhs, +1, st, l))) return r;
    if ((r = collide_impl(h, f, nullptr, P, h->precision, st, l))) return r;
    if ((r = sweep_impl(h, f, P, rhs, -1, st, l))) return r;
  }
  if (l == 0 && (r = rescale_impl(h, f, st))) return r;
  if (flags & SGS_IT_EVAL) {
    if (!Q) return SGS_ERR_ARG;
    if ((r = collide_impl(h, f, Q, P, h->precision, st, l))) return r;
    if (res && (r = residual_impl(h, f, Q, rhs, res, st, l))) return r;
  }
  return SGS_OK;
}

// FAS V-cycle (eq. (30)) from level l down to level levels-1; f and b are level-l fields
// (b may be null on the finest level).
int vcycle_impl(sgs_handle* h, int l, int levels, double* f, const double* b, int pre, int post, int coarse_iters,
                cudaStream_t st) {
  auto& L = h->lev[l];
  const long long K = (long long)h->N * h->N * h->N;
  double* Qs = l == 0 ? h->at<double>(h->lev[0].R) : h->at<double>(L.Q);  // scratch for P/Q of this level
  double* Ps = l == 0 ? nullptr : h->at<double>(L.P);
  int r;
  if (l == levels - 1) {
    for (int it = 0; it < coarse_iters; it++)
      if ((r = iterate_impl(h, f, nullptr, Ps ? Ps : Qs, b, 0, nullptr, st, l))) return r;
    return SGS_OK;
  }
  double* Pl = Ps ? Ps : h->at<double>(h->lev[0].R);
  for (int it = 0; it < pre; it++)
    if ((r = iterate_impl(h, f, nullptr, Pl, b, 0, nullptr, st, l))) return r;
  auto& H = h->lev[l + 1];
  double* R = h->at<double>(L.R);
  double* fH = h->at<double>(H.f);
  double* fH0 = h->at<double>(H.f0);
  double* bH = h->at<double>(H.b);
  double* QH = h->at<double>(H.Q);
  double* PH = h->at<double>(H.P);
  // residual field of the smoothed fine iterate: R_h = T(f) - Q(f)/eps - b_h
  double* Ql = l == 0 ? R : h->at<double>(L.Q);
  if ((r = collide_impl(h, f, Ql, nullptr, h->precision, st, l))) return r;
  if ((r = residual_field_impl(h, f, Ql, b, R, st, l))) return r;
  {
    Scope sc(h, SGS_PROF_RESCALE, st, 2);
    cudaError_t e;
    if (h->two_d) {
      e = launch_restrict2d(f, fH0, K, L.hinst0.nx, L.hinst0.ny, st);
      if (e == cudaSuccess) e = launch_restrict2d(R, bH, K, L.hinst0.nx, L.hinst0.ny, st);
    } else {
      e = launch_restrict(f, fH0, K, H.C, st);
      if (e == cudaSuccess) e = launch_restrict(R, bH, K, H.C, st);
    }
    if (e != cudaSuccess) return cuda_status(e);
  }
  // b_H = R_H(I f) - I(R_h), with R_H(I f) the coarse residual field of the restricted iterate
  H.ref = false;
  const bool coarse_ref = h->precision == SGS_FP32 && h->spectral;
  if ((r = collide_impl(h, fH0, QH, nullptr, h->precision, st, l + 1,
                        coarse_ref && h->cproj ? h->at<double>(H.rQ) : nullptr)))
    return r;
  if (coarse_ref) {
    // Coarse FP32 collisions in increment form against I f: the coarse operator then
    // reproduces R_H(I f) exactly at f_H = I f, so FP32 rounding of Q_H(I f) cancels in the
    // coarse correction f_H - I f instead of entering it as noise.
    CollideCtx<float> x = collide_ctx<float>(h, l + 1);
    cudaError_t e = h->cproj ? cudaSuccess  // the unprojected operator is already in rQ
                             : cudaMemcpyAsync(h->ws + H.rQ, QH, sizeof(double) * K * H.C, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(h->ws + H.rth, h->ws + h->off.theta, sizeof(double) * 5 * H.C, cudaMemcpyDeviceToDevice,
                          st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(h->ws + H.rah, x.sb.ahat, (size_t)H.G * h->n * h->n * h->n * kLanes * sizeof(float2),
                          cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return cuda_status(e);
    H.ref = true;
  }
  if ((r = residual_field_impl(h, fH0, QH, nullptr, PH, st, l + 1))) return r;
  {
    Scope sc(h, SGS_PROF_RESCALE, st, 1);
    cudaError_t e = launch_axpby(bH, PH, -1.0, 1.0, K * H.C, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(fH, fH0, sizeof(double) * K * H.C, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return cuda_status(e);
  }
  if ((r = vcycle_impl(h, l + 1, levels, fH, bH, pre, post, coarse_iters, st))) return r;
  {
    Scope sc(h, SGS_PROF_RESCALE, st, 1);
    cudaError_t e = h->two_d ? launch_prolong_add2d(f, fH, fH0, K, L.hinst0.nx, L.hinst0.ny, st)
                             : launch_prolong_add(f, fH, fH0, K, H.C, st);
    if (e != cudaSuccess) return cuda_status(e);
  }
  for (int it = 0; it < post; it++)
    if ((r = iterate_impl(h, f, nullptr, Pl, b, 0, nullptr, st, l))) return r;
  return SGS_OK;
}

}  // namespace

cudaError_t sgs::func_attr(const void* fn, cudaFuncAttribute attr, int value) {
  static std::mutex mu;
  static std::map<std::tuple<const void*, int, int>, int> done;  // (kernel, attribute, device) -> value
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  auto key = std::make_tuple(fn, (int)attr, dev);
  auto it = done.find(key);
  if (it != done.end() && it->second == value) return cudaSuccess;
  e = cudaFuncSetAttribute(fn, attr, value);
  if (e == cudaSuccess) done[key] = value;
  return e;
}

namespace {

// Uploads the work-unit tables of the current spectral-sum decomposition (synchronous).
cudaError_t upload_sum_plan(sgs_handle* h) {
  std::vector<int4> u4;
  std::vector<long long> s0;
  for (auto& x : h->units) {
    u4.push_back(make_int4(x.k1, x.k2, x.m1lo, x.m1hi));
    s0.push_back(x.step0);
  }
  cudaError_t e = cudaMemcpy(h->ws + h->off.units, u4.data(), sizeof(int4) * u4.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(h->ws + h->off.step0, s0.data(), sizeof(long long) * s0.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(h->ws + h->off.row_start, h->row_start.data(), sizeof(int) * h->row_start.size(),
                   cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(h->ws + h->off.row_units, h->row_units.data(), sizeof(int) * h->row_units.size(),
                   cudaMemcpyHostToDevice);
  return e;
}

// Times `reps` launches of the spectral sum of the handle's arithmetic over every group with
// the current decomposition (CUDA events on st, after one untimed launch). The sums read the
// transformed spectra in the workspace and write only the partial sums.
int time_sum(sgs_handle* h, int reps, cudaStream_t st, float* ms) {
  cudaEvent_t a, b;
  if (cudaEventCreate(&a) != cudaSuccess) return SGS_ERR_CUDA;
  if (cudaEventCreate(&b) != cudaSuccess) {
    cudaEventDestroy(a);
    return SGS_ERR_CUDA;
  }
  cudaError_t e = cudaSuccess;
  for (int i = 0; i <= reps && e == cudaSuccess; i++) {
    if (i == 1) e = cudaEventRecord(a, st);
    if (e != cudaSuccess) break;
    e = h->precision == SGS_FP32 ? launch_spectral_sum(collide_ctx<float>(h), nullptr, st)
                                 : launch_spectral_sum(collide_ctx<double>(h), nullptr, st);
  }
  if (e == cudaSuccess) e = cudaEventRecord(b, st);
  if (e == cudaSuccess) e = cudaEventSynchronize(b);
  if (e == cudaSuccess) e = cudaEventElapsedTime(ms, a, b);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return cuda_status(e);
}

// Times `reps` forward + backward scans of the current launch shape (CUDA events on st).
int time_sweeps(sgs_handle* h, double* f, const double* P, int reps, cudaStream_t st, float* ms) {
  cudaEvent_t a, b;
  if (cudaEventCreate(&a) != cudaSuccess) return SGS_ERR_CUDA;
  if (cudaEventCreate(&b) != cudaSuccess) {
    cudaEventDestroy(a);
    return SGS_ERR_CUDA;
  }
  int r = SGS_OK;
  cudaError_t e = cudaEventRecord(a, st);
  for (int i = 0; i < reps && r == SGS_OK && e == cudaSuccess; i++) {
    r = sweep_impl(h, f, P, nullptr, +1, st);
    if (r == SGS_OK) r = sweep_impl(h, f, P, nullptr, -1, st);
  }
  if (e == cudaSuccess) e = cudaEventRecord(b, st);
  if (e == cudaSuccess) e = cudaEventSynchronize(b);
  if (e == cudaSuccess) e = cudaEventElapsedTime(ms, a, b);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (r != SGS_OK) return r;
  return e == cudaSuccess ? SGS_OK : cuda_status(e);
}

}  // namespace

extern "C" {

int sgs_setup(const sgs_problem* problems, int n_inst, sgs_handle** out, size_t* workspace_bytes) {
  if (!problems || n_inst < 1 || !out) return SGS_ERR_ARG;
  *out = nullptr;
  for (int q = 0; q < n_inst; q++) {
    int r = check_problem(problems[q]);
    if (r != SGS_OK) return r;
    if (problems[q].nv != problems[0].nv || problems[q].v_max != problems[0].v_max ||
        problems[q].precision != problems[0].precision || problems[q].b0 != problems[0].b0 ||
        (problems[q].collision == SGS_BGK) != (problems[0].collision == SGS_BGK) ||
        (problems[q].collision != SGS_BGK && problems[q].collision != problems[0].collision) ||
        problems[q].conserve_proj != problems[0].conserve_proj ||
        (problems[q].order == 2) != (problems[0].order == 2))
      return SGS_ERR_UNSUPPORTED;
  }
  if (problems[0].space_dim == 2 && n_inst != 1) return SGS_ERR_UNSUPPORTED;  // one 2-D instance per handle
  sgs_handle* h = new (std::nothrow) sgs_handle();
  if (!h) return SGS_ERR_NOMEM;
  h->n_inst = n_inst;
  h->prob.assign(problems, problems + n_inst);
  h->N = problems[0].nv;
  h->L = problems[0].v_max;
  h->dv = 2.0 * h->L / h->N;
  h->precision = problems[0].precision;
  h->spectral = problems[0].collision != SGS_BGK;
  h->cproj = h->spectral ? problems[0].conserve_proj : 0;
  h->order2 = problems[0].order == 2;
  h->two_d = problems[0].space_dim == 2;
  long long K = (long long)h->N * h->N * h->N;
  h->inst.resize(n_inst);
  long long off = 0;
  int cell = 0;
  for (int q = 0; q < n_inst; q++) {
    fill_inst(problems[q], h->N, h->dv, h->inst[q]);
    h->inst[q].f_off = off;
    h->inst[q].cell0 = cell;
    const int Jq = h->inst[q].J;
    for (int j = 0; j < Jq; j++) {
      h->cell_off.push_back(off + j * K);
      h->cell_inst.push_back(q);
    }
    off += (long long)Jq * K;
    cell += Jq;
  }
  h->field = off;
  h->C = cell;
  {
    sgs_handle::Level L0;
    L0.C = cell;
    L0.G = (cell + kLanes - 1) / kLanes;
    L0.hinst0 = h->inst[0];
    h->lev.push_back(L0);
    for (int l = 1;; l++) {
      bool ok = true;
      for (int q = 0; q < n_inst; q++) {
        if (problems[q].nx % (1 << l) != 0) ok = false;
        if (h->two_d && problems[q].ny % (1 << l) != 0) ok = false;  // 2 x 2 coarsening
      }
      if (!ok || l > 12) break;
      sgs_handle::Level L;
      long long loff = 0;
      int lcell = 0;
      for (int q = 0; q < n_inst; q++) {
        sgs_problem pc = problems[q];
        pc.nx = problems[q].nx >> l;
        if (h->two_d) pc.ny = problems[q].ny >> l;
        pc.total_mass = 0.0;  // no rescale on coarse levels
        InstDev I;
        fill_inst(pc, h->N, h->dv, I);
        I.f_off = loff;
        I.cell0 = lcell;
        L.hinst.push_back(I);
        for (int j = 0; j < I.J; j++) {
          L.hcell_off.push_back(loff + j * K);
          L.hcell_inst.push_back(q);
        }
        loff += (long long)I.J * K;
        lcell += I.J;
      }
      L.hinst0 = L.hinst[0];
      L.C = lcell;
      L.G = (lcell + kLanes - 1) / kLanes;
      h->lev.push_back(L);
    }
  }
  int r = plan(h);
  if (r != SGS_OK) {
    delete h;
    return r;
  }
  layout(h);
  h->sweep_arith = h->precision == SGS_FP32 ? kSweepDF64 : kSweepF64;
  h->sweep = sweep_shape(h->N, h->sweep_arith);
  *out = h;
  if (workspace_bytes) *workspace_bytes = h->ws_bytes;
  return SGS_OK;
}

int sgs_bind_workspace(sgs_handle* h, void* device_ptr, size_t bytes) {
  if (!h || !device_ptr) return SGS_ERR_ARG;
  if (bytes < h->ws_bytes) return SGS_ERR_WORKSPACE;
  if (((uintptr_t)device_ptr) % kAlign) return SGS_ERR_ARG;
  h->ws = (char*)device_ptr;
  auto up = [&](size_t o, const void* src, size_t n) -> cudaError_t {
    if (n == 0) return cudaSuccess;
    return cudaMemcpy(h->ws + o, src, n, cudaMemcpyHostToDevice);
  };
  cudaError_t e = cudaSuccess;
  std::vector<int4> u4;
  std::vector<long long> s0;
  for (auto& x : h->units) {
    u4.push_back(make_int4(x.k1, x.k2, x.m1lo, x.m1hi));
    s0.push_back(x.step0);
  }
#define SGS_UP(field, vec) \
  if (e == cudaSuccess) e = up(h->off.field, vec.data(), sizeof(vec[0]) * vec.size())
  SGS_UP(inst, h->inst);
  SGS_UP(cell_off, h->cell_off);
  SGS_UP(cell_inst, h->cell_inst);
  SGS_UP(tw_cos, h->tw_cos);
  SGS_UP(tw_sin, h->tw_sin);
  std::vector<float> twc32(h->tw_cos.begin(), h->tw_cos.end()), tws32(h->tw_sin.begin(), h->tw_sin.end());
  SGS_UP(tw_cos32, twc32);
  SGS_UP(tw_sin32, tws32);
  SGS_UP(G, h->Gtab);
  SGS_UP(Lo, h->Lo);
  SGS_UP(units, u4);
  SGS_UP(step0, s0);
  SGS_UP(row_k, h->row_k);
  SGS_UP(row_start, h->row_start);
  SGS_UP(row_units, h->row_units);
#undef SGS_UP
  for (size_t l = 1; l < h->lev.size() && e == cudaSuccess; l++) {
    auto& L = h->lev[l];
    e = up(L.inst, L.hinst.data(), sizeof(InstDev) * L.hinst.size());
    if (e == cudaSuccess) e = up(L.cell_off, L.hcell_off.data(), sizeof(long long) * L.hcell_off.size());
    if (e == cudaSuccess) e = up(L.cell_inst, L.hcell_inst.data(), sizeof(int) * L.hcell_inst.size());
  }
  if (e == cudaSuccess && h->cproj == 1) {
    double Ainv[25];
    if (!gram_inverse(h->N, h->dv, Ainv)) return SGS_ERR_ARG;
    e = up(h->off.cproj_A, Ainv, sizeof(Ainv));
  }
  if (e == cudaSuccess) e = cudaMemset(h->ws + h->off.cnt, 0, sizeof(Counters) * h->n_inst);
  if (e == cudaSuccess) {
    std::vector<int> on(h->n_inst, 1);
    e = up(h->off.active, on.data(), sizeof(int) * on.size());
  }
  if (e == cudaSuccess && h->spectral) {
    // spectral lanes beyond the last cell must hold zeros
    e = cudaMemset(h->ws + h->off.ahat, 0, h->off.qhat - h->off.ahat);
    if (e == cudaSuccess)
      e = launch_build_weights<double>(h->at<int4>(h->off.units), h->at<long long>(h->off.step0), (int)h->units.size(),
                                       h->H, h->PW64, h->at<double>(h->off.G), h->nb, h->at<double>(h->off.Lo),
                                       h->at<double>(h->off.W64), 0);
    if (e == cudaSuccess && h->precision == SGS_FP32)
      e = launch_build_weights<float>(h->at<int4>(h->off.units), h->at<long long>(h->off.step0), (int)h->units.size(),
                                      h->H, h->PW32, h->at<double>(h->off.G), h->nb, h->at<double>(h->off.Lo),
                                      h->at<float>(h->off.W32), 0);
    if (e == cudaSuccess && h->precision == SGS_FP32)
      e = launch_build_weights_lo(h->at<int4>(h->off.units), h->at<long long>(h->off.step0), (int)h->units.size(),
                                  h->H, h->PW32, h->at<double>(h->off.G), h->nb, h->at<double>(h->off.Lo),
                                  h->at<float>(h->off.W32lo), 0);
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  // the scan stream (highest priority) and the events of pipelined iterations
  if (e == cudaSuccess && !h->two_d && h->n_inst == 1 && h->spectral && h->lev[0].G >= 2 && !h->scan_st) {
    int least = 0, greatest = 0;
    e = cudaDeviceGetStreamPriorityRange(&least, &greatest);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&h->scan_st, cudaStreamNonBlocking, greatest);
    for (int i = 0; e == cudaSuccess && i < 3 * h->lev[0].G + 2; i++) {
      cudaEvent_t x = nullptr;
      e = cudaEventCreateWithFlags(&x, cudaEventDisableTiming);
      if (e == cudaSuccess) h->ov_ev.push_back(x);
    }
  }
  return cuda_status(e);
}

int sgs_layout(const sgs_handle* h, int inst, size_t* f_offset, int* n_cells, int* nv) {
  if (!h || inst < 0 || inst >= h->n_inst) return SGS_ERR_ARG;
  if (f_offset) *f_offset = (size_t)h->inst[inst].f_off;
  if (n_cells) *n_cells = h->inst[inst].J;
  if (nv) *nv = h->N;
  return SGS_OK;
}

size_t sgs_field_elems(const sgs_handle* h) { return h ? (size_t)h->field : 0; }

int sgs_collide(sgs_handle* h, const double* f, double* Q, double* P, void* stream) {
  if (!h || !f) return SGS_ERR_ARG;
  if (!h->ws) return SGS_ERR_WORKSPACE;
  return collide_impl(h, f, Q, P, h->precision, as_stream(stream));
}

int sgs_collide_prec(sgs_handle* h, const double* f, double* Q, double* P, int precision, void* stream) {
  if (!h || !f || (precision != SGS_FP64 && precision != SGS_FP32 && precision != SGS_DF64)) return SGS_ERR_ARG;
  if (!h->ws) return SGS_ERR_WORKSPACE;
  if (precision != SGS_FP64 && (h->precision != SGS_FP32 || !h->spectral)) return SGS_ERR_ARG;
  return collide_impl(h, f, Q, P, precision, as_stream(stream));
}

int sgs_sweep_forward(sgs_handle* h, double* f, const double* P, const double* rhs, void* stream) {
  if (!h || !f || !P) return SGS_ERR_ARG;
  if (!h->ws) return SGS_ERR_WORKSPACE;
  return sweep_impl(h, f, P, rhs, +1, as_stream(stream));
}

int sgs_sweep_backward(sgs_handle* h, double* f, const double* P, const double* rhs, void* stream) {
  if (!h || !f || !P) return SGS_ERR_ARG;
  if (!h->ws) return SGS_ERR_WORKSPACE;
  return sweep_impl(h, f, P, rhs, -1, as_stream(stream));
}

int sgs_sweep_ordering(sgs_handle* h, double* f, const double* P, const double* rhs, int ordering, void* stream) {
  if (!h || !f || !P || ordering < 0 || ordering > (h->two_d ? 3 : 1)) return SGS_ERR_ARG;
  if (!h->ws) return SGS_ERR_WORKSPACE;
  return sweep_impl(h, f, P, rhs, ordering == 0 ? +1 : -1, as_stream(stream), 0, ordering);
}

int sgs_rescale(sgs_handle* h, double* f, void* stream) {
  if (!h || !f) return SGS_ERR_ARG;
  if (!h->ws) return SGS_ERR_WORKSPACE;
  return rescale_impl(h, f, as_stream(stream));
}

int sgs_macroscopic(const sgs_handle* h, const double* f, double* out, void* stream) {
  if (!h || !f || !out) return SGS_ERR_ARG;
  if (!h->ws) return SGS_ERR_WORKSPACE;
  return cuda_status(launch_macroscopic(aux_args(h), f, out, as_stream(stream)));
}

int sgs_si_iteration(sgs_handle* h, double* f, double* P, const double* rhs, void* stream) {
  if (!h || !f || !P) return SGS_ERR_ARG;
  if (!h->ws) return SGS_ERR_WORKSPACE;
  if (h->two_d) return SGS_ERR_UNSUPPORTED;
  cudaStream_t st = as_stream(stream);
  int r = collide_impl(h, f, nullptr, P, h->precision, st);  // P, nu, theta of the current iterate
  if (r) return r;
  {
    Scope sc(h, SGS_PROF_SWEEP, st, 3);
    double* efac = h->at<double>(h->off.efac);
    cudaError_t e = launch_factors(h->at<double>(h->off.theta), h->C, h->N, h->dv, efac, st);
    if (e == cudaSuccess) e = launch_si_transport(aux_args(h), f, P, rhs, efac, h->at<double>(h->off.nu), st);
    if (e != cudaSuccess) return cuda_status(e);
  }
  return rescale_impl(h, f, st);
}

int sgs_residual(sgs_handle* h, const double* f, const double* Q, const double* rhs, double* res, void* stream) {
  if (!h || !f || !Q || !res) return SGS_ERR_ARG;
  if (!h->ws) return SGS_ERR_WORKSPACE;
  return residual_impl(h, f, Q, rhs, res, as_stream(stream));
}

int sgs_iterate(sgs_handle* h, double* f, double* Q, double* P, const double* rhs, int flags, double* res,
                void* stream) {
  if (!h || !f || !P) return SGS_ERR_ARG;
  if (!h->ws) return SGS_ERR_WORKSPACE;
  return iterate_impl(h, f, Q, P, rhs, flags, res, as_stream(stream));
}

int sgs_dc_step(sgs_handle* h, double* f, double* Q, double* P, int lo_iters, double* res, void* stream) {
  if (!h || !f || !Q || !P || lo_iters < 0) return SGS_ERR_ARG;
  if (!h->ws) return SGS_ERR_WORKSPACE;
  if (h->precision != SGS_FP32 || !h->spectral) return SGS_ERR_ARG;
  cudaStream_t st = as_stream(stream);
  int r;
  // FP64 collision and residual of the current iterate f_k: the convergence test
  h->dc_ref = false;
  // with the conservation projection the unprojected operator goes straight to Q_ref
  if ((r = collide_impl(h, f, Q, P, h->dc_prec, st, 0, h->cproj ? h->at<double>(h->off.Q_ref) : nullptr))) return r;
  if (res && (r = residual_impl(h, f, Q, nullptr, res, st))) return r;
  // new reference: f_ref = f_k, theta_ref = theta(f_k), Q_ref = Q_FP64(f_k), ahat_ref = FP32 DFT of f_k - M_k
  cudaError_t e = cudaMemcpyAsync(h->ws + h->off.f_ref, f, sizeof(double) * h->field, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess && !h->cproj)
    e = cudaMemcpyAsync(h->ws + h->off.Q_ref, Q, sizeof(double) * h->field, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h->ws + h->off.theta_ref, h->ws + h->off.theta, sizeof(double) * 5 * h->C,
                        cudaMemcpyDeviceToDevice, st);
  if (e != cudaSuccess) return cuda_status(e);
  {
    CollideCtx<float> x = collide_ctx<float>(h);
    Scope sc(h, SGS_PROF_DFT, st, 4);
    e = launch_dft(f, x, DftMode{0, nullptr, nullptr}, st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(h->ws + h->off.ahat_ref, x.sb.ahat,
                          (size_t)h->G * h->n * h->n * h->n * kLanes * sizeof(float2), cudaMemcpyDeviceToDevice, st);
  }
  if (e != cudaSuccess) return cuda_status(e);
  h->dc_ref = true;
  // P from the FP64 collision is P of f_k in the increment form as well (zero increments)
  // Pipelined iterations also evaluate the collision step of the iterate they produce (its
  // P is the next iteration's), so every collision step overlaps a scan; otherwise the next
  // iteration evaluates it first.
  const bool ov = overlap_ok(h, 0);
  for (int it = 0; it < lo_iters; it++) {
    int fl = ov ? SGS_IT_P_VALID | SGS_IT_EVAL : (it == 0 ? SGS_IT_P_VALID : 0);
    if ((r = iterate_impl(h, f, Q, P, nullptr, fl, nullptr, st))) return r;
  }
  return SGS_OK;
}

int sgs_set_dc_precision(sgs_handle* h, int precision) {
  if (!h || (precision != SGS_FP64 && precision != SGS_DF64)) return SGS_ERR_ARG;
  h->dc_prec = precision;
  return SGS_OK;
}

int sgs_dc_clear(sgs_handle* h) {
  if (!h) return SGS_ERR_ARG;
  h->dc_ref = false;
  return SGS_OK;
}

int sgs_vcycle(sgs_handle* h, double* f, int levels, int pre, int post, int coarse_iters, void* stream) {
  if (!h || !f || levels < 2 || pre < 0 || post < 0 || coarse_iters < 0) return SGS_ERR_ARG;
  if (!h->ws) return SGS_ERR_WORKSPACE;
  if (levels > (int)h->lev.size()) return SGS_ERR_ARG;
  return vcycle_impl(h, 0, levels, f, nullptr, pre, post, coarse_iters, as_stream(stream));
}

int sgs_max_levels(const sgs_handle* h) { return h ? (int)h->lev.size() : 0; }

int sgs_set_overlap(sgs_handle* h, int enable) {
  if (!h) return SGS_ERR_ARG;
  h->overlap = enable != 0;
  return SGS_OK;
}

int sgs_get_overlap(const sgs_handle* h) { return h && h->ws ? (overlap_ok(h, 0) ? 1 : 0) : 0; }

int sgs_update_active(sgs_handle* h, const double* res, double tol, void* stream) {
  if (!h || !res || !(tol >= 0.0)) return SGS_ERR_ARG;
  if (!h->ws) return SGS_ERR_WORKSPACE;
  return cuda_status(launch_update_active(res, h->n_inst, tol, h->at<int>(h->off.active), as_stream(stream)));
}

int sgs_activate_all(sgs_handle* h, void* stream) {
  if (!h) return SGS_ERR_ARG;
  if (!h->ws) return SGS_ERR_WORKSPACE;
  return cuda_status(launch_fill_int(h->at<int>(h->off.active), h->n_inst, 1, as_stream(stream)));
}

int sgs_read_active(sgs_handle* h, int* active, void* stream) {
  if (!h || !active) return SGS_ERR_ARG;
  if (!h->ws) return SGS_ERR_WORKSPACE;
  cudaError_t e = cudaStreamSynchronize(as_stream(stream));
  if (e == cudaSuccess)
    e = cudaMemcpy(active, h->ws + h->off.active, sizeof(int) * h->n_inst, cudaMemcpyDeviceToHost);
  return cuda_status(e);
}

int sgs_get_sweep_shape(const sgs_handle* h, int* ept, int* cluster, int* threads) {
  if (!h || !ept || !cluster || !threads) return SGS_ERR_ARG;
  *ept = h->sweep.ept;
  *cluster = h->sweep.cluster;
  *threads = h->sweep.tpb;
  return SGS_OK;
}

int sgs_set_sweep_shape(sgs_handle* h, int ept, int cluster, int threads) {
  if (!h) return SGS_ERR_ARG;
  SweepShape sh{ept, cluster, threads};
  if (!sweep_ept_compiled(ept) || !sweep_shape_valid(h->N, sh)) return SGS_ERR_ARG;
  int n = 0;
  cudaError_t e = sweep_max_clusters(sh, h->sweep_arith, &n);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return SGS_ERR_UNSUPPORTED;
  }
  if (n < 1) return SGS_ERR_UNSUPPORTED;
  h->sweep = sh;
  return SGS_OK;
}

int sgs_autotune(sgs_handle* h, double* f, const double* P, int reps, sgs_tuning* out, void* stream) {
  if (!h || !f || !P || reps < 1) return SGS_ERR_ARG;
  if (!h->ws) return SGS_ERR_WORKSPACE;
  cudaStream_t st = as_stream(stream);
  const bool prof = h->prof;
  h->prof = false;
  const SweepShape start = h->sweep;
  const int K = h->N * h->N * h->N;
  SweepShape best = start;
  float best_ms = -1.0f;
  int tried = 0, r = SGS_OK;
  const int epts[] = {2, 4, 8, 12, 16, 20, 24, 28, 32};
  for (int ept : epts) {
    if (h->N % ept) continue;
    for (int cs = 1; cs <= 16; cs *= 2) {
      int per = (K + ept * cs - 1) / (ept * cs);
      int tpb = (per + 31) / 32 * 32;
      if (tpb < 160) tpb = 160;  // warps 0-4 serve the Newton evaluations
      SweepShape sh{ept, cs, tpb};
      if (!sweep_shape_valid(h->N, sh)) continue;
      if ((long long)(tpb - 32) * cs * ept >= K && tpb > 160) continue;  // a whole warp idle in every CTA
      int n = 0;
      if (sweep_max_clusters(sh, h->sweep_arith, &n) != cudaSuccess) {
        cudaGetLastError();
        continue;
      }
      if (n < 1) continue;
      h->sweep = sh;
      float ms = 0.0f;
      r = time_sweeps(h, f, P, 1, st, &ms);  // warm-up
      if (r == SGS_OK) r = time_sweeps(h, f, P, reps, st, &ms);
      if (r != SGS_OK) break;
      tried++;
      if (best_ms < 0.0f || ms < best_ms) {
        best_ms = ms;
        best = sh;
      }
    }
    if (r != SGS_OK) break;
  }
  h->sweep = r == SGS_OK ? best : start;
  if (r != SGS_OK) {
    h->prof = prof;
    return r;
  }
  // spectral-sum decomposition: warps (lane groups) per block and block count
  float sum_best = -1.0f;
  int sum_tried = 0;
  if (h->spectral) {
    const int nw0 = h->NW, bl0 = h->sum_blocks;
    int best_nw = nw0, best_bl = bl0;
    for (int nw = 1; nw <= kSumMaxWarps && r == SGS_OK; nw *= 2) {
      if (nw > 1 && (nw / 2) >= h->G) break;  // more warps than lane groups
      for (int bl : kSumBlockChoices) {
        plan_units(h, sum_target(h, nw, bl));
        if ((int)h->units.size() > h->U_cap) continue;
        h->NW = nw;
        cudaError_t e = upload_sum_plan(h);
        if (e != cudaSuccess) {
          r = cuda_status(e);
          break;
        }
        float ms = 0.0f;
        r = time_sum(h, 2, st, &ms);
        if (r != SGS_OK) break;
        sum_tried++;
        if (sum_best < 0.0f || ms < sum_best) {
          sum_best = ms;
          best_nw = nw;
          best_bl = bl;
        }
      }
    }
    h->NW = best_nw;
    h->sum_blocks = best_bl;
    plan_units(h, sum_target(h, best_nw, best_bl));
    cudaError_t e = upload_sum_plan(h);
    if (r == SGS_OK && e != cudaSuccess) r = cuda_status(e);
  }
  h->prof = prof;
  if (r != SGS_OK) return r;
  if (out) {
    out->sweep_ept = best.ept;
    out->sweep_cluster = best.cluster;
    out->sweep_threads = best.tpb;
    out->sweep_ms = best_ms / reps;
    out->candidates = tried;
    out->sum_warps = h->NW;
    out->sum_units = (int)h->units.size();
    out->sum_blocks = (int)h->units.size() * ((h->G + h->NW - 1) / h->NW);
    out->sum_ms = sum_best > 0.0f ? sum_best / 2 : 0.0f;
    out->sum_candidates = sum_tried;
  }
  return SGS_OK;
}

int sgs_probe_scan(int nv, double v_max, int precision, int cluster, int threads, int mode, int reps,
                   float* us_per_op, void* stream) {
  if (!valid_nv(nv) || !(v_max > 0.0) || (mode < 0 || mode > 2) || reps < 1 || !us_per_op) return SGS_ERR_ARG;
  if (precision != SGS_FP64 && precision != SGS_FP32) return SGS_ERR_ARG;
  const int arith = precision == SGS_FP32 ? kSweepDF64 : kSweepF64;  // the scan arithmetic of such a handle
  const double dv = 2.0 * v_max / nv;
  cudaStream_t st = as_stream(stream);
  cudaEvent_t ev[4];
  for (int i = 0; i < 4; i++)
    if (cudaEventCreate(&ev[i]) != cudaSuccess) {
      for (int k = 0; k < i; k++) cudaEventDestroy(ev[k]);
      return SGS_ERR_CUDA;
    }
  // warm-up, then an empty launch (launch and set-up cost) and the timed one
  cudaError_t e = probe_scan(nv, dv, arith, cluster, threads, mode, 1, st);
  if (e == cudaSuccess) e = cudaEventRecord(ev[0], st);
  if (e == cudaSuccess) e = probe_scan(nv, dv, arith, cluster, threads, mode, 0, st);
  if (e == cudaSuccess) e = cudaEventRecord(ev[1], st);
  if (e == cudaSuccess) e = cudaEventRecord(ev[2], st);
  if (e == cudaSuccess) e = probe_scan(nv, dv, arith, cluster, threads, mode, reps, st);
  if (e == cudaSuccess) e = cudaEventRecord(ev[3], st);
  if (e == cudaSuccess) e = cudaEventSynchronize(ev[3]);
  float t0 = 0.f, t1 = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t0, ev[0], ev[1]);
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t1, ev[2], ev[3]);
  for (int i = 0; i < 4; i++) cudaEventDestroy(ev[i]);
  if (e == cudaErrorInvalidConfiguration) {
    cudaGetLastError();
    return SGS_ERR_ARG;
  }
  if (e != cudaSuccess) return cuda_status(e);
  *us_per_op = (t1 - t0) * 1e3f / reps;
  return SGS_OK;
}

// ---------------------------------------------------------------------------------------
// The fast (Carleman-form) spectral operator, hard spheres, on the tensor cores.
// ---------------------------------------------------------------------------------------
}  // extern "C"

struct sgs_fast {
  int N = 0, n = 0, h = 0, npad = 0, P = 0, C = 0, M = 0, slots = 0, chunk = 0;
  double L = 0.0, b0 = 0.0;
  std::vector<float> wtab, wslot, bt12, bt3;
  std::vector<float2> tw;
  struct {
    size_t fhat, wtab, wslot, bt12, bt3, tw, Y1h, Y1l, Y2h, Y2l, G, T1, T2, end;
  } off;
  size_t ws_bytes = 0;
  char* ws = nullptr;
  template <typename T>
  T* at(size_t o) const {
    return reinterpret_cast<T*>(ws + o);
  }
};

namespace {

// Gauss-Legendre nodes and weights on [-1, 1] (Newton iteration on the Legendre polynomial
// from the Chebyshev-like initial guesses).
void gauss_legendre(int m, std::vector<double>& x, std::vector<double>& w) {
  x.assign(m, 0.0);
  w.assign(m, 0.0);
  for (int i = 0; i < m; i++) {
    double z = std::cos(kPi * (i + 0.75) / (m + 0.5)), dp = 0.0;
    for (int it = 0; it < 100; it++) {
      double p0 = 1.0, p1 = 0.0;
      for (int j = 1; j <= m; j++) {
        double p2 = p1;
        p1 = p0;
        p0 = ((2.0 * j - 1.0) * z * p1 - (j - 1.0) * p2) / j;
      }
      dp = m * (z * p0 - p1) / (z * z - 1.0);
      double dz = p0 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    x[i] = z;
    w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

// The radial factors of the Carleman weights with both variables truncated at T:
// phi(s) = 2 int_0^T rho cos(pi rho s / L) drho, psi(t) = 2 pi int_0^T rho J0(pi rho t / L) drho.
double fast_phi(double s, double T, double L) {
  const double a = kPi * s / L;
  if (std::fabs(a) <= 1e-12) return T * T;
  return 2.0 * (T * std::sin(a * T) / a + (std::cos(a * T) - 1.0) / (a * a));
}
double fast_psi(double t, double T, double L) {
  if (t <= 1e-12) return kPi * T * T;
  return 2.0 * T * L * std::cyl_bessel_j(1.0, kPi * T * t / L) / t;
}

}  // namespace

extern "C" {

int sgs_fast_setup(const sgs_handle* h, int m_theta, int m_phi, int chunk, sgs_fast** out, size_t* workspace_bytes) {
  if (!h || !out || m_theta < 1 || m_phi < 1 || chunk < 1 || m_theta * m_phi > 4096) return SGS_ERR_ARG;
  *out = nullptr;
  if (!h->spectral || h->prob[0].collision != SGS_HARD_SPHERE) return SGS_ERR_UNSUPPORTED;
  sgs_fast* x = new (std::nothrow) sgs_fast();
  if (!x) return SGS_ERR_NOMEM;
  x->N = h->N;
  x->n = h->n;
  x->h = h->H;
  x->npad = x->n <= 16 ? 16 : 32;
  x->P = 3 * x->h + 1 <= 32 ? 32 : 48;  // zero padding that keeps the linear convolutions free of wrap-around
  x->C = h->C;
  x->M = m_theta * m_phi;
  x->slots = x->M + 1;  // the nodes, then the loss term
  x->chunk = std::min(chunk, x->slots);
  x->L = h->L;
  x->b0 = h->prob[0].b0;
  const int n = x->n, np = x->npad, P = x->P, H = x->h;
  const double R = 2.0 * x->L / (3.0 * std::sqrt(2.0) + 1.0), T = 2.0 * R;
  // half-sphere rule: Gauss-Legendre in cos(theta) on [0, 1], uniform azimuths
  std::vector<double> gx, gw;
  gauss_legendre(m_theta, gx, gw);
  std::vector<double> e(3 * x->M), wp(x->M);
  for (int i = 0; i < m_theta; i++)
    for (int j = 0; j < m_phi; j++) {
      const double mu = 0.5 * (gx[i] + 1.0), st = std::sqrt(std::max(0.0, 1.0 - mu * mu));
      const double az = 2.0 * kPi * j / m_phi;
      const int p = i * m_phi + j;
      e[3 * p] = st * std::cos(az);
      e[3 * p + 1] = st * std::sin(az);
      e[3 * p + 2] = mu;
      wp[p] = 0.5 * gw[i] * 2.0 * kPi / m_phi;
    }
  const size_t per = (size_t)n * np * np;
  x->wtab.assign((size_t)x->slots * 2 * per, 0.0f);
  x->wslot.assign(x->slots, 0.0f);
  std::vector<double> bmm((size_t)n * n * n, 0.0);
  for (int p = 0; p < x->M; p++) {
    float* wa = &x->wtab[((size_t)p * 2) * per];
    float* wb = wa + per;
    for (int k1 = 0; k1 < n; k1++)
      for (int k2 = 0; k2 < n; k2++)
        for (int k3 = 0; k3 < n; k3++) {
          const double kv[3] = {(double)(k1 - H), (double)(k2 - H), (double)(k3 - H)};
          const double ke = kv[0] * e[3 * p] + kv[1] * e[3 * p + 1] + kv[2] * e[3 * p + 2];
          const double kk = kv[0] * kv[0] + kv[1] * kv[1] + kv[2] * kv[2];
          const double ph = fast_phi(ke, T, x->L), ps = fast_psi(std::sqrt(std::max(kk - ke * ke, 0.0)), T, x->L);
          const size_t o = ((size_t)k1 * np + k2) * np + k3;
          wa[o] = (float)ph;
          wb[o] = (float)ps;
          bmm[((size_t)k1 * n + k2) * n + k3] += wp[p] * ph * ps;
        }
    x->wslot[p] = (float)(4.0 * x->b0 * wp[p]);
  }
  {  // the loss term: -fhat * (beta(m, m) fhat) as the last slot
    float* wa = &x->wtab[((size_t)x->M * 2) * per];
    float* wb = wa + per;
    for (int k1 = 0; k1 < n; k1++)
      for (int k2 = 0; k2 < n; k2++)
        for (int k3 = 0; k3 < n; k3++) {
          const size_t o = ((size_t)k1 * np + k2) * np + k3;
          wa[o] = 1.0f;
          wb[o] = (float)(4.0 * x->b0 * bmm[((size_t)k1 * n + k2) * n + k3]);
        }
    x->wslot[x->M] = -1.0f;
  }
  // DFT matrices E[x, k] = exp(2 pi i x (k - h) / P) as real 2 x 2 blocks, K index 2 k + (re, im)
  x->bt12.assign((size_t)2 * P * 2 * np, 0.0f);
  x->bt3.assign((size_t)P * 2 * np, 0.0f);
  for (int xx = 0; xx < P; xx++)
    for (int k = 0; k < n; k++) {
      const double ang = 2.0 * kPi * (double)(((long long)xx * (k - H)) % P) / P;
      const float er = (float)std::cos(ang), ei = (float)std::sin(ang);
      float* r0 = &x->bt12[(size_t)(2 * xx) * 2 * np];
      float* r1 = &x->bt12[(size_t)(2 * xx + 1) * 2 * np];
      r0[2 * k] = er;
      r0[2 * k + 1] = -ei;
      r1[2 * k] = ei;
      r1[2 * k + 1] = er;
      float* r3 = &x->bt3[(size_t)xx * 2 * np];
      r3[2 * k] = er;
      r3[2 * k + 1] = -ei;
    }
  x->tw.resize((size_t)n * P);
  for (int k = 0; k < n; k++)
    for (int xx = 0; xx < P; xx++) {
      const double ang = -2.0 * kPi * (double)(((long long)xx * (k - H)) % P) / P;
      x->tw[(size_t)k * P + xx] = make_float2((float)std::cos(ang), (float)std::sin(ang));
    }
  // workspace
  size_t o = 0;
  auto take = [&](size_t bytes) {
    size_t r = o;
    o = align_up(o + bytes);
    return r;
  };
  const size_t Bc = (size_t)x->C * x->chunk * 2;
  x->off.fhat = take(sizeof(float) * x->C * per * 2);
  x->off.wtab = take(sizeof(float) * x->wtab.size());
  x->off.wslot = take(sizeof(float) * x->wslot.size());
  x->off.bt12 = take(sizeof(float) * x->bt12.size());
  x->off.bt3 = take(sizeof(float) * x->bt3.size());
  x->off.tw = take(sizeof(float2) * x->tw.size());
  // BF16 operand planes of 128-row tiles (K = 2 np); Y1 rows (b, k1 < np, x3), k1 padded
  const size_t tile = (size_t)128 * 2 * np;
  const size_t y1_tiles = (Bc * P * np + 127) / 128, y2_tiles = Bc * P * P / 128;
  x->off.Y1h = take(sizeof(uint16_t) * y1_tiles * tile);
  x->off.Y1l = take(sizeof(uint16_t) * y1_tiles * tile);
  x->off.Y2h = take(sizeof(uint16_t) * y2_tiles * tile);
  x->off.Y2l = take(sizeof(uint16_t) * y2_tiles * tile);
  x->off.G = take(sizeof(float) * (size_t)x->C * P * P * P);
  x->off.T1 = take(sizeof(float2) * (size_t)x->C * P * P * n);
  x->off.T2 = take(sizeof(float2) * (size_t)x->C * P * n * n);
  x->off.end = o;
  x->ws_bytes = o;
  *out = x;
  if (workspace_bytes) *workspace_bytes = o;
  return SGS_OK;
}

int sgs_fast_bind(sgs_fast* x, void* device_ptr, size_t bytes) {
  if (!x || !device_ptr) return SGS_ERR_ARG;
  if (bytes < x->ws_bytes) return SGS_ERR_WORKSPACE;
  if (((uintptr_t)device_ptr) % kAlign) return SGS_ERR_ARG;
  x->ws = (char*)device_ptr;
  cudaError_t e = cudaMemcpy(x->ws + x->off.wtab, x->wtab.data(), sizeof(float) * x->wtab.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(x->ws + x->off.wslot, x->wslot.data(), sizeof(float) * x->wslot.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(x->ws + x->off.bt12, x->bt12.data(), sizeof(float) * x->bt12.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(x->ws + x->off.bt3, x->bt3.data(), sizeof(float) * x->bt3.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(x->ws + x->off.tw, x->tw.data(), sizeof(float2) * x->tw.size(), cudaMemcpyHostToDevice);
  // the padded entries of the pass-3 operand (k1 >= n) and the rows past the last pass-2 row
  // are never written: zero them once
  if (e == cudaSuccess) e = cudaMemset(x->ws + x->off.Y1h, 0, x->off.G - x->off.Y1h);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  return cuda_status(e);
}

int sgs_fast_collide(sgs_fast* x, sgs_handle* h, const double* f, double* Q, int terms, void* stream) {
  if (!x || !h || !f || !Q || (terms != 1 && terms != 3)) return SGS_ERR_ARG;
  if (!x->ws || !h->ws) return SGS_ERR_WORKSPACE;
  if (x->N != h->N || x->C != h->C || x->L != h->L) return SGS_ERR_ARG;
  cudaStream_t st = as_stream(stream);
  // moments and discrete Maxwellians (the transforms of f - M and f + M give fhat); the
  // transforms run in FP32 (the passes take FP32 spectra and BF16 products)
  CollideCtx<float> cx = collide_ctx<float>(h);
  cudaError_t e;
  {
    Scope sc(h, SGS_PROF_MOMENTS, st, 1);
    const sgs_problem& p0 = h->prob[0];
    e = launch_moments(f, cx.ct, h->C, h->N, h->dv, p0.newton_tol, p0.newton_max, h->at<double>(h->off.theta),
                       h->at<double>(h->off.nu), h->at<Counters>(h->off.cnt), st);
  }
  if (e != cudaSuccess) return cuda_status(e);
  {
    Scope sc(h, SGS_PROF_DFT, st, 5);
    e = launch_dft(f, cx, DftMode{0, nullptr, nullptr}, st);
    if (e == cudaSuccess)
      e = launch_fast_fhat(cx.sb.ahat, cx.sb.bhat, x->C, x->n, x->npad, x->at<float>(x->off.fhat), st);
  }
  if (e != cudaSuccess) return cuda_status(e);
  {
    Scope sc(h, SGS_PROF_FAST, st, 3 * ((x->slots + x->chunk - 1) / x->chunk) + 4, (double)x->C);
    e = cudaMemsetAsync(x->ws + x->off.G, 0, sizeof(float) * (size_t)x->C * x->P * x->P * x->P, st);
    FastArgs a;
    a.n = x->n;
    a.npad = x->npad;
    a.P = x->P;
    a.C = x->C;
    a.terms = terms;
    a.fhat = x->at<float>(x->off.fhat);
    a.wtab = x->at<float>(x->off.wtab);
    a.wslot = x->at<float>(x->off.wslot);
    a.bt12 = x->at<float>(x->off.bt12);
    a.bt3 = x->at<float>(x->off.bt3);
    a.Y1h = x->at<uint16_t>(x->off.Y1h);
    a.Y1l = x->at<uint16_t>(x->off.Y1l);
    a.Y2h = x->at<uint16_t>(x->off.Y2h);
    a.Y2l = x->at<uint16_t>(x->off.Y2l);
    a.G = x->at<float>(x->off.G);
    a.spin_max = h->spin_max;
    a.status = &h->at<Counters>(h->off.cnt)[0].status;
    for (int s0 = 0; s0 < x->slots && e == cudaSuccess; s0 += x->chunk) {
      a.s0 = s0;
      a.S = std::min(x->chunk, x->slots - s0);
      for (int pass = 1; pass <= 3 && e == cudaSuccess; pass++) e = launch_fast_pass(pass, a, st);
    }
    if (e == cudaSuccess)
      e = launch_fast_final(a.G, x->at<float2>(x->off.tw), x->C, x->n, x->P, x->at<float2>(x->off.T1),
                            x->at<float2>(x->off.T2), cx.sb.qhat, st);
  }
  if (e != cudaSuccess) return cuda_status(e);
  // inverse transform of the modes to the velocity grid (no partial sums to reduce)
  Scope sc(h, SGS_PROF_REDUCE_IDFT, st, 3);
  cx.red.n_rows = 0;
  cx.mom = nullptr;
  return cuda_status(launch_reduce_idft(f, Q, nullptr, cx, nullptr, nullptr, st));
}

void sgs_fast_destroy(sgs_fast* x) { delete x; }

int sgs_read_status(sgs_handle* h, sgs_stats* out, void* stream) {
  if (!h || !out) return SGS_ERR_ARG;
  if (!h->ws) return SGS_ERR_WORKSPACE;
  cudaError_t e = cudaStreamSynchronize(as_stream(stream));
  if (e != cudaSuccess) return cuda_status(e);
  std::vector<Counters> c(h->n_inst);
  e = cudaMemcpy(c.data(), h->ws + h->off.cnt, sizeof(Counters) * h->n_inst, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_status(e);
  memset(out, 0, sizeof(*out));
  for (auto& x : c) {
    out->status |= x.status;
    out->visits += x.visits;
    out->inner_iters += x.inner_iters;
    out->newton_iters += x.newton_iters;
    out->newton_solves += x.newton_solves;
    out->fallbacks += x.fallbacks;
  }
  return SGS_OK;
}

int sgs_reset_stats(sgs_handle* h, void* stream) {
  if (!h) return SGS_ERR_ARG;
  if (!h->ws) return SGS_ERR_WORKSPACE;
  return cuda_status(cudaMemsetAsync(h->ws + h->off.cnt, 0, sizeof(Counters) * h->n_inst, as_stream(stream)));
}

int sgs_profile(sgs_handle* h, int enable) {
  if (!h) return SGS_ERR_ARG;
  h->prof = enable != 0;
  return SGS_OK;
}

int sgs_profile_read(sgs_handle* h, double* ms, unsigned long long* launches, double* work, int n_classes) {
  if (!h || n_classes < 0) return SGS_ERR_ARG;
  for (int c = 0; c < n_classes; c++) {
    if (ms) ms[c] = 0.0;
    if (launches) launches[c] = 0;
    if (work) work[c] = 0.0;
  }
  for (auto& rec : h->recs) {
    cudaError_t e = cudaEventSynchronize(rec.b);
    if (e != cudaSuccess) return cuda_status(e);
    float t = 0.f;
    cudaEventElapsedTime(&t, rec.a, rec.b);
    if (rec.cls < n_classes) {
      if (ms) ms[rec.cls] += t;
      if (launches) launches[rec.cls] += 1;
      if (work) work[rec.cls] += rec.work;
    }
    h->pool.push_back(rec.a);
    h->pool.push_back(rec.b);
  }
  h->recs.clear();
  return SGS_OK;
}

unsigned long long sgs_launch_count(const sgs_handle* h) { return h ? h->launches : 0; }

void sgs_destroy(sgs_handle* h) {
  if (!h) return;
  for (auto& rec : h->recs) {
    h->pool.push_back(rec.a);
    h->pool.push_back(rec.b);
  }
  for (auto e : h->pool) cudaEventDestroy(e);
  for (auto e : h->ov_ev) cudaEventDestroy(e);
  if (h->scan_st) cudaStreamDestroy(h->scan_st);
  delete h;
}

const char* sgs_strerror(int code) {
  switch (code) {
    case SGS_OK: return "ok";
    case SGS_ERR_ARG: return "invalid argument";
    case SGS_ERR_UNSUPPORTED: return "unsupported configuration";
    case SGS_ERR_CUDA: return "CUDA runtime error";
    case SGS_ERR_WORKSPACE: return "workspace missing or too small";
    case SGS_ERR_NOMEM: return "host allocation failed";
  }
  return "unknown error";
}

double sgs_host_weight(int nv, double v_max, int collision, double b0, long long a2, long long b2) {
  return weight_G(nv, v_max, collision, b0, a2, b2);
}

}  // extern "C"
