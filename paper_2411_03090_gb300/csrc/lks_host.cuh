// lks_host.cuh -- host helpers shared by the single-lattice and the batched C ABI:
// descriptor checks, coefficient and geometry records of a problem, the inlet
// amplitude of the pulsed inflow, the generalized-inverse edge moment maps of the
// adjoint (Sec. 2.5, App. A) and the CUDA driver entry point that encodes tensor maps.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <utility>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/lks.h"
#include "lks_kernels.cuh"

namespace lks_host {
using lks::Coef;
using lks::Geom;

// NVTX range over a scope of host code (the enqueue of a march, a segment, a
// gradient); a profiler attached to the process shows it on the host timeline and
// can restrict kernel captures to it (ncu --nvtx --nvtx-include).  Without a tool
// attached the calls return at once.
struct Range {
  explicit Range(const char* name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
  Range(const Range&) = delete;
  Range& operator=(const Range&) = delete;
};

constexpr int CXh[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
constexpr int CYh[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
constexpr double Wh[9] = {4.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};

// Multiprocessors of the current device (looked up on first use; 152 on a GB300 if
// the query fails).
inline int device_sm_count() {
  static const int sms = [] {
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        n <= 0)
      n = 152;
    return n;
  }();
  return sms;
}

// Grid of an element-wise kernel over n items: 256-thread blocks, at most eight per
// multiprocessor (the kernels loop over the rest).
inline int elementwise_blocks(size_t n) { return (int)std::min<size_t>((n + 255) / 256, (size_t)device_sm_count() * 8); }

// Any of the thermal source terms (heat source, heat-exchange objective, Boussinesq).
inline bool has_sources(const lks_problem_desc& d) {
  return d.beta_bar != 0.0 || d.kappa_Q != 0.0 || d.gb[0] != 0.0 || d.gb[1] != 0.0;
}
// Terms that only the per-step kernels carry: the thermal sources and the energy loss.
inline bool step_kernels_only(const lks_problem_desc& d) { return has_sources(d) || d.kappa_E != 0.0; }

inline lks_status check_desc(const lks_problem_desc* d, std::string* why) {
  auto bad = [&](const char* m) {
    if (why) *why = m;
    return LKS_ERR_INVALID_ARG;
  };
  if (!d) return bad("descriptor is NULL");
  if (d->version != LKS_DESC_VERSION) return bad("descriptor version mismatch");
  if (d->nx < 5 || d->ny < 5) return bad("nx and ny must be >= 5");
  if (d->lattice != LKS_LATTICE_D2Q9 && d->lattice != LKS_LATTICE_D3Q19) return bad("bad lattice");
  if (d->lattice == LKS_LATTICE_D3Q19) {
    if (d->nz < 5) return bad("D3Q19: nz must be >= 5");
    if ((int64_t)d->nx * d->ny * d->nz > (int64_t)1 << 31) return bad("lattice larger than 2^31 nodes");
    if (d->real_type != LKS_REAL_F32 && d->real_type != LKS_REAL_F64) return bad("real_type must be F32 or F64");
    if (!(d->nu > 0.0 && d->nu < 0.5)) return bad("nu must lie in (0, 0.5)");
    if (!(d->alpha_bar >= 0.0) || !(d->q_alpha > 0.0)) return bad("alpha_bar >= 0 and q_alpha > 0 required");
    if (!d->steady || d->thermal || has_sources(*d)) return bad("D3Q19: steady, non-thermal problems only");
    if (d->kappa_E != 0.0) return bad("D3Q19: kappa_E must be 0");
    if (d->n_steps < 1 || d->n_adj < 1) return bad("n_steps and n_adj must be >= 1");
    if (d->res_steps != 0) return bad("D3Q19: res_steps must be 0");
    if (d->exec_path < LKS_PATH_AUTO || d->exec_path > LKS_PATH_COLUMN) return bad("bad exec_path");
    if (!std::isfinite(d->kappa_p)) return bad("kappa_p must be finite");
    if (d->tol != 0.0) return bad("D3Q19: tol must be 0 (fixed step counts)");
    if (d->warm_start != 0) return bad("D3Q19: warm_start must be 0");
    for (int q = 0; q < 4; ++q)
      if (d->reserved[q] != 0) return bad("reserved fields must be zero");
    return LKS_OK;
  }
  if (d->nz != 0 && d->nz != 1) return bad("D2Q9: nz must be 0 or 1");
  if ((int64_t)d->nx * d->ny > (int64_t)1 << 31) return bad("lattice larger than 2^31 nodes");
  if (d->real_type != LKS_REAL_F32 && d->real_type != LKS_REAL_F64) return bad("real_type must be F32 or F64");
  if (!(d->nu > 0.0 && d->nu < 0.5)) return bad("nu must lie in (0, 0.5)");
  if (!(d->alpha_bar >= 0.0) || !(d->q_alpha > 0.0)) return bad("alpha_bar >= 0 and q_alpha > 0 required");
  if (d->in_y0 < 0 || d->in_y1 > d->ny - 1 || d->in_y1 <= d->in_y0) return bad("bad inlet span");
  // outlet span inside [1, ny-2]; out_y1 = out_y0 - 1 means no outlet (the right edge is a wall)
  if (d->out_y0 < 1 || d->out_y1 > d->ny - 2 || d->out_y1 < d->out_y0 - 1) return bad("bad outlet span");
  if (!std::isfinite(d->heat_q)) return bad("heat_q must be finite");
  if (d->n_steps < 1) return bad("n_steps must be >= 1");
  if (d->steady && d->n_adj < 1) return bad("n_adj must be >= 1 for a steady problem");
  if (d->thermal) {
    if (!(d->q_K > 0.0)) return bad("q_K must be > 0");
    for (int e = 0; e < 4; ++e)
      if (d->t_kind[e] != LKS_T_FIXED && d->t_kind[e] != LKS_T_FLUX) return bad("bad thermal edge kind");
  }
  if (d->checkpoint_every < 0) return bad("checkpoint_every must be >= 0");
  if (d->snapshot_type < LKS_SNAP_F32 || d->snapshot_type > LKS_SNAP_F16) return bad("bad snapshot_type");
  if (d->exec_path < LKS_PATH_AUTO || d->exec_path > LKS_PATH_COLUMN) return bad("bad exec_path");
  if (d->res_steps < 0 || d->res_steps > 3) return bad("res_steps must lie in 0..3");
  if (!std::isfinite(d->kappa_p)) return bad("kappa_p must be finite");
  if (d->kappa_p != 0.0 && !d->steady) return bad("D2Q9: kappa_p != 0 needs a steady problem");
  if (!std::isfinite(d->kappa_E)) return bad("kappa_E must be finite");
  if (d->kappa_E != 0.0 && (d->exec_path == LKS_PATH_RESIDENT || d->exec_path == LKS_PATH_COLUMN))
    return bad("the energy loss runs on the per-step kernels (exec_path AUTO or STEP)");
  if (d->kappa_E != 0.0 && !(d->rho_out > 0.0)) return bad("kappa_E != 0 needs rho_out > 0");
  if (!(d->tol >= 0.0) || !std::isfinite(d->tol)) return bad("tol must be >= 0");
  if (d->tol > 0.0) {
    if (!d->steady) return bad("tol > 0: steady problems only");
    if (d->max_steps < d->n_steps || d->max_steps < d->n_adj) return bad("tol > 0: max_steps >= n_steps, n_adj");
  }
  if (has_sources(*d)) {
    if (!d->thermal) return bad("heat source, heat-exchange objective and Boussinesq force need thermal = 1");
    if (d->exec_path == LKS_PATH_RESIDENT || d->exec_path == LKS_PATH_COLUMN)
      return bad("thermal source terms run on the per-step kernels (exec_path AUTO or STEP)");
    if (d->beta_bar != 0.0 && !(d->q_beta > 0.0)) return bad("q_beta must be > 0");
    if (!std::isfinite(d->beta_bar) || !std::isfinite(d->kappa_Q) || !std::isfinite(d->gb[0]) ||
        !std::isfinite(d->gb[1]) || !std::isfinite(d->T_ref) || d->beta_bar < 0.0)
      return bad("thermal source parameters must be finite, beta_bar >= 0");
  }
  if (d->warm_start != 0 && d->warm_start != 1) return bad("warm_start must be 0 or 1");
  if (d->warm_start && !d->steady) return bad("warm_start: steady problems only");
  if (d->segment_type < LKS_SNAP_F32 || d->segment_type > LKS_SNAP_F16) return bad("bad segment_type");
  if (d->segment_type != LKS_SNAP_F32 && (d->steady || d->real_type != LKS_REAL_F32))
    return bad("segment_type BF16 / F16: unsteady FP32 problems only");
  for (int q = 0; q < 4; ++q)
    if (d->reserved[q] != 0) return bad("reserved fields must be zero");
  return LKS_OK;
}

// ------------------------------------------------------------------------------------
// Generalized-inverse edge maps (Sec. 2.5; App. A)
// ------------------------------------------------------------------------------------
// Solves min ||Acols x + b||_2 for several right-hand sides by the normal equations.
// A: 9 x nc (row major); zero columns are dropped (their unknowns set to zero).
inline void lsq_solve(const double* A, int nc, const double* rhs /* 9 */, double* x) {
  int live[16], nl = 0;
  for (int cidx = 0; cidx < nc; ++cidx) {
    double s = 0;
    for (int r = 0; r < 9; ++r) s += std::fabs(A[r * nc + cidx]);
    x[cidx] = 0.0;
    if (s > 0) live[nl++] = cidx;
  }
  double G[16][17];
  for (int a = 0; a < nl; ++a) {
    for (int b = 0; b < nl; ++b) {
      double s = 0;
      for (int r = 0; r < 9; ++r) s += A[r * nc + live[a]] * A[r * nc + live[b]];
      G[a][b] = s;
    }
    double s = 0;
    for (int r = 0; r < 9; ++r) s += A[r * nc + live[a]] * rhs[r];
    G[a][nl] = s;
  }
  for (int col = 0; col < nl; ++col) {
    int p = col;
    for (int r = col + 1; r < nl; ++r)
      if (std::fabs(G[r][col]) > std::fabs(G[p][col])) p = r;
    for (int q = 0; q <= nl; ++q) std::swap(G[col][q], G[p][q]);
    for (int r = 0; r < nl; ++r) {
      if (r == col) continue;
      const double f = G[r][col] / G[col][col];
      for (int q = col; q <= nl; ++q) G[r][q] -= f * G[col][q];
    }
  }
  for (int a = 0; a < nl; ++a) x[live[a]] = G[a][nl] / G[a][a];
}

inline void class_geometry(int cls, int* nx, int* ny, int* pressure) {
  static const int tab[9][3] = {{-1, 0, 0}, {1, 0, 1}, {1, 0, 0}, {0, -1, 0}, {0, 1, 0},
                                {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0}, {1, 1, 0}};
  *nx = tab[cls][0];
  *ny = tab[cls][1];
  *pressure = tab[cls][2];
}

// Flow: 6 x 10 moment map for edge class cls at parameter A: columns 0..8 map the
// nine gathered f~ (unknown entries ignored); column 9 is the response of the
// moments to the heat-flux coupling term kappa~ T (c.n) of Eqs. afboundaryuq /
// afboundarypq, which enters the residual as -kappa~ T (c_i.n).  jb_out (optional,
// 6 values): the response to a boundary objective term added to every residual row
// (dJ_dO/df_i of Eqs. afboundaryu / afboundaryp; +kappa_p on inlet nodes and
// -kappa_p on outlet nodes for the static pressure drop).
inline void flow_moment_map(double A, int cls, double* out, double* jb_out = nullptr) {
  int n_x, n_y, pres;
  class_geometry(cls, &n_x, &n_y, &pres);
  bool unk[9];
  int U[9], nu = 0;
  for (int k = 0; k < 9; ++k) {
    unk[k] = (CXh[k] * n_x > 0) || (CYh[k] * n_y > 0);
    if (unk[k]) U[nu++] = k;
  }
  double M[9][9];
  for (int r = 0; r < 9; ++r)
    for (int c = 0; c < 9; ++c) {
      const int cnc = CXh[c] * n_x + CYh[c] * n_y;
      const double cc = CXh[c] * CXh[r] + CYh[c] * CYh[r];
      M[r][c] = (r == c ? (double)(CXh[r] * n_x + CYh[r] * n_y) : 0.0) - 2.0 * A * Wh[c] * cnc * cc;
    }
  const int nc = nu + 2;
  std::vector<double> Am(9 * nc);
  for (int r = 0; r < 9; ++r) {
    for (int q = 0; q < nu; ++q) Am[r * nc + q] = M[r][U[q]];
    if (pres) {
      Am[r * nc + nu] = 1.0;
      Am[r * nc + nu + 1] = (double)(CXh[r] * (-n_y) + CYh[r] * n_x);
    } else {
      Am[r * nc + nu] = CXh[r];
      Am[r * nc + nu + 1] = CYh[r];
    }
  }
  double X[9][11] = {};  // X[u][k]: unknown u from known k; 9: from kappa~ T; 10: from a unit row term
  for (int k = 0; k < 11; ++k) {
    if (k < 9 && unk[k]) continue;
    double rhs[9], x[16];
    for (int r = 0; r < 9; ++r) rhs[r] = k < 9 ? -M[r][k] : (k == 9 ? (double)(CXh[r] * n_x + CYh[r] * n_y) : -1.0);
    lsq_solve(Am.data(), nc, rhs, x);
    for (int q = 0; q < nu; ++q) X[U[q]][k] = x[q];
  }
  for (int r = 0; r < 6; ++r)
    for (int k = 0; k < 10; ++k) {
      auto mom = [&](int kk) {
        const double cx = CXh[kk], cy = CYh[kk];
        const double f[6] = {1, cx, cy, cx * cx, cx * cy, cy * cy};
        return Wh[kk] * f[r];
      };
      double s = 0.0;
      if (k == 9 || !unk[k]) {
        s = k < 9 ? mom(k) : 0.0;
        for (int q = 0; q < nu; ++q) s += mom(U[q]) * X[U[q]][k];
      }
      out[r * 10 + k] = s;
    }
  if (jb_out)
    for (int r = 0; r < 6; ++r) {
      double s = 0.0;
      for (int q = 0; q < nu; ++q) {
        const double cx = CXh[U[q]], cy = CYh[U[q]];
        const double f[6] = {1, cx, cy, cx * cx, cx * cy, cy * cy};
        s += Wh[U[q]] * f[r] * X[U[q]][10];
      }
      jb_out[r] = s;
    }
}

template <typename R>
inline Coef<R> make_coef(const lks_problem_desc& d) {
  Coef<R> c;
  c.A = (R)((1.0 / 6.0 - d.nu) * 4.5);
  c.nu = (R)d.nu;
  c.alpha_bar = (R)d.alpha_bar;
  c.q_alpha = (R)d.q_alpha;
  c.drho_out = (R)(d.rho_out - 1.0);
  c.K_f = (R)d.K_f;
  c.K_s = (R)d.K_s;
  c.q_K = (R)d.q_K;
  c.kappa_T = (R)d.kappa_T;
  c.kappa_p = (R)d.kappa_p;
  c.beta_bar = (R)d.beta_bar;
  c.q_beta = (R)d.q_beta;
  c.kappa_Q = (R)d.kappa_Q;
  c.gb_x = (R)d.gb[0];
  c.gb_y = (R)d.gb[1];
  c.T_ref = (R)d.T_ref;
  c.heat_q = (R)d.heat_q;
  c.kappa_E = (R)d.kappa_E;
  for (int e = 0; e < 4; ++e) c.t_val[e] = (R)d.t_val[e];
  return c;
}

inline Geom make_geom(const lks_problem_desc& d) {
  Geom g;
  g.nx = d.nx;
  g.ny = d.ny;
  g.in_y0 = d.in_y0;
  g.in_y1 = d.in_y1;
  g.out_y0 = d.out_y0;
  g.out_y1 = d.out_y1;
  for (int e = 0; e < 4; ++e) g.t_kind[e] = d.thermal ? d.t_kind[e] : 0;
  g.hx0 = d.heat_x0;
  g.hx1 = d.heat_x1;
  return g;
}

inline double inlet_amp(const lks_problem_desc& d, int t) {
  double a = d.pulse_mean;
  if (d.pulse_period > 0.0) a += d.pulse_amp * std::sin(2.0 * M_PI * (double)t / d.pulse_period);
  return d.u_max * a;
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

inline EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = []() -> EncodeTiledFn {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return nullptr;
    return reinterpret_cast<EncodeTiledFn>(p);
  }();
  return fn;
}


}  // namespace lks_host
