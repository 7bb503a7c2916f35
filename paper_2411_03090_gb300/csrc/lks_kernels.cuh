// lks_kernels.cuh -- sm_103a kernels of the LKS forward march, the ALKS adjoint
// march, the objective and the design sensitivity (arXiv 2411.03090, Secs. 2.4-2.5,
// App. A).  Templated on the arithmetic type R (float for production, double for
// the tight parity instance) and on the thermal lattice.
//
// Data layout: structure of arrays in HBM, one array of nx*ny values per field,
// node (i, j) at j*nx + i.  The density is stored as the deviation drho = rho - 1
// so that FP32 keeps its digits for the O(1e-3) pressure variations.
//
// Each CTA owns a TX x TY tile of output nodes.  It stages the fields it reads in
// shared memory with a halo of two nodes (the velocity gradient of a neighbour
// needs the neighbour's neighbours), evaluates the per-node equilibrium
// coefficients once on the tile plus a one-node ring, and then gathers the nine
// streamed populations of every output node from shared memory.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace lks {

constexpr int TX = 32;            // tile width (outputs)
constexpr int TY = 16;            // tile height (outputs)
constexpr int NTHREADS = 256;     // 32 x 8 threads, two output rows per thread
constexpr int H2X = TX + 4, H2Y = TY + 4;  // halo-2 staging region
constexpr int H1X = TX + 2, H1Y = TY + 2;  // halo-1 coefficient region

// D2Q9 velocities (Eq. D2Q9w numbering, opposite pairs 1-3, 2-4, 5-7, 6-8).
__device__ __forceinline__ int cxk(int k) {
  constexpr int c[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
  return c[k];
}
__device__ __forceinline__ int cyk(int k) {
  constexpr int c[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
  return c[k];
}
template <typename R>
__device__ __forceinline__ R wk(int k) {
  return k == 0 ? R(4) / R(9) : (k < 5 ? R(1) / R(9) : R(1) / R(36));
}

// Node classes; edge normal (nx, ny) outward, summed at corners.
enum NodeClass { C_INTERIOR = 0, C_VELOCITY = 1, C_PRESSURE = 2, C_CORNER = 3 };

struct Geom {
  int nx, ny;
  int in_y0, in_y1, out_y0, out_y1;
  int t_kind[4];  // left, right, bottom, top
  int hx0, hx1;   // heated segment of a heat-flux bottom edge (none when hx1 < hx0)
};

// Parabolic inlet profile 4 y (H - y) / H^2 at row j (y = j - in_y0, H = in_y1 -
// in_y0), in the arithmetic of the instance: FP64 for double, explicitly rounded
// FP32 for float (the same value in every FP32 kernel).
template <typename R>
__device__ __forceinline__ R inlet_profile(const Geom& g, int j) {
  if constexpr (sizeof(R) == 8) {
    const double H = (double)(g.in_y1 - g.in_y0), y = (double)(j - g.in_y0);
    return 4.0 * y * (H - y) / (H * H);
  } else {
    const float H = (float)(g.in_y1 - g.in_y0), y = (float)(j - g.in_y0);
    return __fdiv_rn(__fmul_rn(__fmul_rn(4.f, y), __fsub_rn(H, y)), __fmul_rn(H, H));
  }
}

template <typename R>
struct Coef {
  R A;          // Eq. (A): nu = 1/6 - 2A/9
  R nu;
  R alpha_bar, q_alpha;
  R drho_out;   // rho_out - 1
  R K_f, K_s, q_K;
  R kappa_T;
  R t_val[4];
  R kappa_p;    // weight of the static pressure drop J_p in J (steady problems)
  R beta_bar, q_beta;  // heat source Q = beta_gamma (1 - T) (Eqs. heatsource, betagamma); 0: none
  R kappa_Q;           // weight of the heat-exchange objective -sum beta_gamma (1 - T)
  R gb_x, gb_y, T_ref; // Boussinesq force G = g beta (T - T_ref) (Eq. boussinesqforce)
  R heat_q;            // heat flux q_w of the heated bottom segment
  R kappa_E;           // weight of the energy loss J_E (Eq. objective_doublepipe); 0: none
};

// Edge maps of one lattice: 9 classes x 6 moments x 10 columns (lks_edge_moment_map),
// then 9 classes x 6 responses to a unit boundary objective term.
constexpr int kEdgeMapLen = 9 * 60 + 9 * 6;

// Boundary objective term of the static pressure drop at an edge node of class ec
// (dJ_dO/df_i of Eqs. afboundaryu / afboundaryp, every residual row): +kappa_p on the
// inlet nodes (left face inside the inlet span), -kappa_p on the outlet nodes
// (pressure class), 0 elsewhere.
template <typename R>
__device__ __forceinline__ R edge_objective_term(const Geom& g, const Coef<R>& c, int ec, int j) {
  if (ec == 1) return -c.kappa_p;
  if (ec == 0 && j >= g.in_y0 && j <= g.in_y1) return c.kappa_p;
  return R(0);
}

// Energy loss of one node (Eq. objective_doublepipe), kappa_E (-n.u) (p + |u|^2 / 2)
// with p = (rho - rho_out) / 3 = (drho - drho_out) / 3 and dGamma = 1, on the inlet
// nodes (left edge inside the inlet span, n = (-1, 0)) and the outlet nodes (right
// edge inside the outlet span, n = (1, 0)), corners excluded; zero elsewhere.  FP64.
template <typename R>
__device__ __forceinline__ double energy_loss_node(const Geom& g, const Coef<R>& c, int i, int j, R drho, R u, R v) {
  if (j < 1 || j > g.ny - 2) return 0.0;
  double un;  // -n.u
  if (i == 0 && j >= g.in_y0 && j <= g.in_y1) un = (double)u;
  else if (i == g.nx - 1 && j >= g.out_y0 && j <= g.out_y1) un = -(double)u;
  else return 0.0;
  const double p = ((double)drho - (double)c.drho_out) / 3.0;
  return (double)c.kappa_E * un * (p + 0.5 * ((double)u * (double)u + (double)v * (double)v));
}

// Edge-class index of the moment maps (see lks_edge_moment_map in lks.h).
__device__ __forceinline__ int edge_class(const Geom& g, int i, int j) {
  const bool L = i == 0, Rr = i == g.nx - 1, B = j == 0, T = j == g.ny - 1;
  if (B && L) return 5;
  if (B && Rr) return 6;
  if (T && L) return 7;
  if (T && Rr) return 8;
  if (L) return 0;
  if (B) return 3;
  if (T) return 4;
  return (j >= g.out_y0 && j <= g.out_y1) ? 1 : 2;
}

__device__ __forceinline__ int node_class(const Geom& g, int i, int j, int& nxo, int& nyo) {
  const bool L = i == 0, Rr = i == g.nx - 1, B = j == 0, T = j == g.ny - 1;
  nxo = (Rr ? 1 : 0) - (L ? 1 : 0);
  nyo = (T ? 1 : 0) - (B ? 1 : 0);
  if ((L || Rr) && (B || T)) return C_CORNER;
  if (L || B || T) return C_VELOCITY;
  if (Rr) return (j >= g.out_y0 && j <= g.out_y1) ? C_PRESSURE : C_VELOCITY;
  return C_INTERIOR;
}

// Thermal edge id of an edge or corner node (corners follow the horizontal edge).
__device__ __forceinline__ int thermal_edge(const Geom& g, int i, int j) {
  if (j == 0) return 2;
  if (j == g.ny - 1) return 3;
  return i == 0 ? 0 : 1;
}

// Prescribed heat flux -q.n of a heat-flux edge node: the edge's value, or heat_q on
// the heated segment [hx0, hx1] of the bottom edge.
template <typename R>
__device__ __forceinline__ R flux_value(const Geom& g, const Coef<R>& c, int e, int i) {
  return (e == 2 && i >= g.hx0 && i <= g.hx1) ? c.heat_q : c.t_val[e];
}

// Brinkman interpolation, Eq. (brinkman), and its derivative.
template <typename R>
__device__ __forceinline__ R alpha_of(const Coef<R>& c, R gm) {
  return c.alpha_bar * c.q_alpha * (R(1) - gm) / (c.q_alpha + gm);
}
template <typename R>
__device__ __forceinline__ R dalpha_of(const Coef<R>& c, R gm) {
  const R d = c.q_alpha + gm;
  return -c.alpha_bar * c.q_alpha * (R(1) + c.q_alpha) / (d * d);
}
// Conductivity interpolation, Eq. (conductivity), mapped to B by Eq. (B).
// Eq. (betagamma) and its derivative.
template <typename R>
__device__ __forceinline__ R beta_of(const Coef<R>& c, R gm) {
  return c.beta_bar * c.q_beta * (R(1) - gm) / (c.q_beta + gm);
}
template <typename R>
__device__ __forceinline__ R dbeta_of(const Coef<R>& c, R gm) {
  const R d = c.q_beta + gm;
  return -c.beta_bar * c.q_beta * (R(1) + c.q_beta) / (d * d);
}

// Heat source and Boussinesq force at an interior node of the forward step: the new
// T* becomes (T* + beta_gamma) / (1 + beta_gamma) (Q = beta_gamma (1 - T) at t + dt,
// taken implicitly), and u = u* inv gains inv g beta (T - T_ref) with that new T
// (Eq. lbef_ex with Eq. boussinesqforce; inv = 1 / (1 + alpha_gamma)).
template <typename R>
__device__ __forceinline__ void thermal_sources(const Coef<R>& c, R gm, R inv, R& T, R& u, R& v) {
  if (c.beta_bar != R(0)) {
    const R b = beta_of(c, gm);
    T = (T + b) / (R(1) + b);
  }
  if (c.gb_x != R(0) || c.gb_y != R(0)) {
    const R dT = T - c.T_ref;
    u += inv * (c.gb_x * dT);
    v += inv * (c.gb_y * dT);
  }
}
__device__ __forceinline__ bool has_thermal_sources(const Coef<float>& c) {
  return c.beta_bar != 0.f || c.gb_x != 0.f || c.gb_y != 0.f || c.kappa_Q != 0.f;
}
template <typename R>
__device__ __forceinline__ bool has_thermal_sources(const Coef<R>& c) {
  return c.beta_bar != R(0) || c.gb_x != R(0) || c.gb_y != R(0) || c.kappa_Q != R(0);
}

// T~ of an interior node (Eq. albeg_ex) with the heat source and the Boussinesq
// coupling: (T~* + 3 g beta . u~ - dJ_O/dT) / (1 + beta_gamma) with
// dJ_O/dT = kappa_T + kappa_Q beta_gamma; u~ is the node's adjoint velocity of the
// same level, after its Brinkman division.
template <typename R>
__device__ __forceinline__ R adj_thermal_T(const Coef<R>& c, R gm, R Tstar, R ux, R uy) {
  const R b = c.beta_bar != R(0) ? beta_of(c, gm) : R(0);
  return (Tstar + R(3) * (c.gb_x * ux + c.gb_y * uy) - (c.kappa_T + c.kappa_Q * b)) / (R(1) + b);
}

// Heat-exchange objective at an interior node, -kappa_Q beta_gamma (1 - T)
// (Eq. objective_heatexchanger), and its sensitivity terms with the heat source:
// -beta' (1 - T) (T~ + kappa_Q).
template <typename R>
__device__ __forceinline__ R heat_objective(const Coef<R>& c, R gm, R T) {
  return c.kappa_Q != R(0) ? -c.kappa_Q * beta_of(c, gm) * (R(1) - T) : R(0);
}
template <typename R>
__device__ __forceinline__ R heat_sensitivity(const Coef<R>& c, R gm, R T, R Tt) {
  return c.beta_bar != R(0) ? -dbeta_of(c, gm) * (R(1) - T) * (Tt + c.kappa_Q) : R(0);
}

template <typename R>
__device__ __forceinline__ R B_of(const Coef<R>& c, R gm) {
  const R K = c.K_f + (c.K_s - c.K_f) * c.q_K * (R(1) - gm) / (c.q_K + gm);
  return R(3) * (R(1) / R(6) - K);
}
template <typename R>
__device__ __forceinline__ R dB_of(const Coef<R>& c, R gm) {
  const R d = c.q_K + gm;
  return R(3) * (c.K_s - c.K_f) * c.q_K * (R(1) + c.q_K) / (d * d);
}

// Derivative along x of a field staged in shared memory with row length LX; (lx,
// ly) is the staged position of global node (i, j).  Central inside, second-order
// one-sided on the domain edge.
template <typename R, int LX>
__device__ __forceinline__ R dfdx(const R* s, int lx, int ly, int i, int nx) {
  const R* r = s + ly * LX + lx;
  if (i == 0) return (R(-3) * r[0] + R(4) * r[1] - r[2]) * R(0.5);
  if (i == nx - 1) return (R(3) * r[0] - R(4) * r[-1] + r[-2]) * R(0.5);
  return (r[1] - r[-1]) * R(0.5);
}
template <typename R, int LX>
__device__ __forceinline__ R dfdy(const R* s, int lx, int ly, int j, int ny) {
  const R* r = s + ly * LX + lx;
  if (j == 0) return (R(-3) * r[0] + R(4) * r[LX] - r[2 * LX]) * R(0.5);
  if (j == ny - 1) return (R(3) * r[0] - R(4) * r[-LX] + r[-2 * LX]) * R(0.5);
  return (r[LX] - r[-LX]) * R(0.5);
}

// Stage a field with halo h into shared memory (row length LX = TX + 2h); values
// outside the lattice are zero.
template <typename R, int LX, int LY>
__device__ __forceinline__ void stage(R* s, const R* __restrict__ g, int x0, int y0, int h,
                                      int nx, int ny) {
  for (int q = threadIdx.x; q < LX * LY; q += NTHREADS) {
    const int ly = q / LX, lx = q - ly * LX;
    const int i = x0 - h + lx, j = y0 - h + ly;
    R v = R(0);
    if (i >= 0 && i < nx && j >= 0 && j < ny) v = __ldg(g + (size_t)j * nx + i);
    s[q] = v;
  }
}

template <typename R>
__device__ __forceinline__ bool bad_velocity(R u, R v) {
  const R m = u * u + v * v;
  return !(m <= R(0.25));  // also catches NaN
}

__device__ __forceinline__ void raise_status(int* status, int code) {
  if (status) atomicCAS(status, 0, code);
}

// FP64 block reduction of one value per thread (NT threads); thread 0 receives the
// sum, in a fixed order.
template <int NT = NTHREADS>
__device__ __forceinline__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int q = 0; q < NT / 32; ++q) s += red[q];
  __syncthreads();
  return s;
}

// =====================================================================================
// Forward LKS step
// =====================================================================================
template <typename R>
struct FwdArgs {
  const R* drho;
  const R* u;
  const R* v;
  const R* T;
  R* drho_n;
  R* u_n;
  R* v_n;
  R* T_n;
  const R* gamma;
  R u_in;             // inlet peak velocity at the new time level
  double* J_partial;  // per-block accumulator of J_O(old state), or null
  int* status;
  R* traj_u;          // optional store of the new level (u, v, T) for the adjoint
  R* traj_v;
  R* traj_T;
};

// Shared memory of the forward kernel (elements of R).
template <bool TH>
constexpr int fwd_smem_elems() {
  return 2 * H2X * H2Y + H1X * H1Y * 7 + (TH ? (H2X * H2Y + H1X * H1Y * 4) : 0);
}

// One LKS step (Eqs. rho, u, T; f^eq Eq. feq2, g^eq Eq. geq2; implicit Brinkman of
// Eq. lbef_ex; edge rules of Sec. 2.4).  Each node's f_k^eq is written as
//   f_k^eq = w_k (drho + e0 + c_x bx + c_y by + c_x^2 qxx + c_y^2 qyy + c_x c_y qxy)
// with e0 = -3/2 |u|^2, bx = 3u, by = 3v, qxx = 9/2 u^2 + A S_xx,
// qyy = 9/2 v^2 + A S_yy, qxy = 9 u v + 2 A S_xy; g_k^eq = w_k (T + c.tq) with
// tq = 3 T u + B grad T.  The new density is accumulated as an increment on the
// node's own value, drho(x) + sum_k w_k [(drho(x - c_k) - drho(x)) + ...] (the
// weights of the sum add to one, also in the edge rule), which keeps FP32 rounding
// of a large pressure level out of the O(u) terms; T likewise.
template <typename R, bool TH>
__global__ void __launch_bounds__(NTHREADS) fwd_step_kernel(FwdArgs<R> a, Geom g, Coef<R> c) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R* sm = reinterpret_cast<R*>(smem_raw);
  R* su = sm;
  R* sv = su + H2X * H2Y;
  R* sr = sv + H2X * H2Y;            // drho, halo 1
  R* ca0 = sr + H1X * H1Y;
  R* cbx = ca0 + H1X * H1Y;
  R* cby = cbx + H1X * H1Y;
  R* cqx = cby + H1X * H1Y;
  R* cqy = cqx + H1X * H1Y;
  R* cqxy = cqy + H1X * H1Y;
  R* sT = cqxy + H1X * H1Y;          // thermal: T halo 2, then t0, tqx, tqy, gamma(h1)
  R* ct0 = sT + (TH ? H2X * H2Y : 0);
  R* ctx = ct0 + H1X * H1Y;
  R* cty = ctx + H1X * H1Y;
  R* sgB = cty + H1X * H1Y;          // B_gamma on the halo-1 region
  __shared__ double red[NTHREADS / 32];

  const int nx = g.nx, ny = g.ny;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  stage<R, H2X, H2Y>(su, a.u, x0, y0, 2, nx, ny);
  stage<R, H2X, H2Y>(sv, a.v, x0, y0, 2, nx, ny);
  stage<R, H1X, H1Y>(sr, a.drho, x0, y0, 1, nx, ny);
  if (TH) {
    stage<R, H2X, H2Y>(sT, a.T, x0, y0, 2, nx, ny);
    for (int q = threadIdx.x; q < H1X * H1Y; q += NTHREADS) {
      const int ly = q / H1X, lx = q - ly * H1X;
      const int i = x0 - 1 + lx, j = y0 - 1 + ly;
      R b = R(0);
      if (i >= 0 && i < nx && j >= 0 && j < ny) b = B_of(c, __ldg(a.gamma + (size_t)j * nx + i));
      sgB[q] = b;
    }
  }
  __syncthreads();

  // Equilibrium coefficients on the halo-1 region; also the objective of the old
  // state at interior output nodes (unsteady accumulation).
  double jloc = 0.0;
  for (int q = threadIdx.x; q < H1X * H1Y; q += NTHREADS) {
    const int ly = q / H1X, lx = q - ly * H1X;
    const int i = x0 - 1 + lx, j = y0 - 1 + ly;
    if (i < 0 || i >= nx || j < 0 || j >= ny) {
      ca0[q] = cbx[q] = cby[q] = cqx[q] = cqy[q] = cqxy[q] = R(0);
      if (TH) ct0[q] = ctx[q] = cty[q] = R(0);
      continue;
    }
    const int sx = lx + 1, sy = ly + 1;  // position in the halo-2 arrays
    const R uu = su[sy * H2X + sx], vv = sv[sy * H2X + sx];
    R dudx = dfdx<R, H2X>(su, sx, sy, i, nx);
    const R dudy = dfdy<R, H2X>(su, sx, sy, j, ny);
    const R dvdx = dfdx<R, H2X>(sv, sx, sy, i, nx);
    R dvdy = dfdy<R, H2X>(sv, sx, sy, j, ny);
    // Edge nodes: normal derivative of the normal velocity from continuity (Eq. cont).
    const bool xe = (i == 0 || i == nx - 1), ye = (j == 0 || j == ny - 1);
    if (xe && ye) {
      dudx = R(0);
      dvdy = R(0);
    } else if (xe) {
      dudx = -dvdy;
    } else if (ye) {
      dvdy = -dudx;
    }
    const R Sxx = R(2) * dudx, Syy = R(2) * dvdy, Sxy = dudy + dvdx;
    ca0[q] = -R(1.5) * (uu * uu + vv * vv);
    cbx[q] = R(3) * uu;
    cby[q] = R(3) * vv;
    cqx[q] = R(4.5) * uu * uu + c.A * Sxx;
    cqy[q] = R(4.5) * vv * vv + c.A * Syy;
    cqxy[q] = R(9) * uu * vv + R(2) * c.A * Sxy;
    if (TH) {
      const R TT = sT[sy * H2X + sx];
      const R dTdx = dfdx<R, H2X>(sT, sx, sy, i, nx), dTdy = dfdy<R, H2X>(sT, sx, sy, j, ny);
      const R Bn = sgB[q];
      ct0[q] = TT;
      ctx[q] = R(3) * TT * uu + Bn * dTdx;
      cty[q] = R(3) * TT * vv + Bn * dTdy;
    }
    if (a.J_partial && lx >= 1 && lx <= TX && ly >= 1 && ly <= TY && i > 0 && j > 0 &&
        i < nx - 1 && j < ny - 1) {
      // central differences at interior nodes (objective J_O)
      const R cSxx = R(2) * dudx, cSyy = R(2) * dvdy, cSxy = dudy + dvdx;
      const R gmo = __ldg(a.gamma + (size_t)j * nx + i);
      const R al = alpha_of(c, gmo);
      jloc += (double)(R(0.5) * c.nu * (cSxx * cSxx + R(2) * cSxy * cSxy + cSyy * cSyy) +
                       al * (uu * uu + vv * vv));
      if (TH) jloc += (double)(c.kappa_T * sT[sy * H2X + sx] + heat_objective(c, gmo, sT[sy * H2X + sx]));
    }
    // energy loss of the old state on the inlet and outlet nodes of the tile
    if (a.J_partial && c.kappa_E != R(0) && lx >= 1 && lx <= TX && ly >= 1 && ly <= TY && (i == 0 || i == nx - 1))
      jloc += energy_loss_node(g, c, i, j, sr[q], uu, vv);
  }
  __syncthreads();
  if (a.J_partial) {
    const double s = block_sum(jloc, red);
    if (threadIdx.x == 0) a.J_partial[blockIdx.y * gridDim.x + blockIdx.x] += s;
  }

  // Gather and update, two output rows per thread.
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
#pragma unroll
  for (int rr = 0; rr < TY / 8; ++rr) {
    const int oy = ty + 8 * rr;
    const int i = x0 + tx, j = y0 + oy;
    if (i >= nx || j >= ny) continue;
    const int q = (oy + 1) * H1X + (tx + 1);  // position in the halo-1 arrays
    int nxo, nyo;
    const int cls = node_class(g, i, j, nxo, nyo);
    R drn, un, vn, Tn = R(0);
    const R drx = sr[q];
    if (cls == C_INTERIOR) {
      const int W = q - 1, E = q + 1, S = q - H1X, N = q + H1X;
      const int SW = S - 1, SE = S + 1, NE = N + 1, NW = N - 1;
      // populations without the node's own density (increment form)
      const R f0 = ca0[q] * (R(4) / R(9));
      const R f1 = ((sr[W] - drx) + ca0[W] + cbx[W] + cqx[W]) * (R(1) / R(9));
      const R f3 = ((sr[E] - drx) + ca0[E] - cbx[E] + cqx[E]) * (R(1) / R(9));
      const R f2 = ((sr[S] - drx) + ca0[S] + cby[S] + cqy[S]) * (R(1) / R(9));
      const R f4 = ((sr[N] - drx) + ca0[N] - cby[N] + cqy[N]) * (R(1) / R(9));
      const R d5 = (sr[SW] - drx) + ca0[SW] + cqx[SW] + cqy[SW];
      const R d6 = (sr[SE] - drx) + ca0[SE] + cqx[SE] + cqy[SE];
      const R d7 = (sr[NE] - drx) + ca0[NE] + cqx[NE] + cqy[NE];
      const R d8 = (sr[NW] - drx) + ca0[NW] + cqx[NW] + cqy[NW];
      const R f5 = (d5 + cbx[SW] + cby[SW] + cqxy[SW]) * (R(1) / R(36));
      const R f6 = (d6 - cbx[SE] + cby[SE] - cqxy[SE]) * (R(1) / R(36));
      const R f7 = (d7 - cbx[NE] - cby[NE] + cqxy[NE]) * (R(1) / R(36));
      const R f8 = (d8 + cbx[NW] - cby[NW] - cqxy[NW]) * (R(1) / R(36));
      drn = drx + (f0 + f1 + f2 + f3 + f4 + f5 + f6 + f7 + f8);
      const R us = f1 - f3 + f5 - f6 - f7 + f8;
      const R vs = f2 - f4 + f5 + f6 - f7 - f8;
      const R inv = R(1) / (R(1) + alpha_of(c, __ldg(a.gamma + (size_t)j * nx + i)));
      un = us * inv;
      vn = vs * inv;
      if (TH) {
        const R Tx = ct0[q];
        R Ts = ((ct0[W] - Tx) + ctx[W] + (ct0[E] - Tx) - ctx[E] + (ct0[S] - Tx) + cty[S] +
                (ct0[N] - Tx) - cty[N]) * (R(1) / R(9));
        Ts += ((ct0[SW] - Tx) + ctx[SW] + cty[SW] + (ct0[SE] - Tx) - ctx[SE] + cty[SE] +
               (ct0[NE] - Tx) - ctx[NE] - cty[NE] + (ct0[NW] - Tx) + ctx[NW] - cty[NW]) * (R(1) / R(36));
        Tn = Tx + Ts;
        if (has_thermal_sources(c)) thermal_sources(c, __ldg(a.gamma + (size_t)j * nx + i), inv, Tn, un, vn);
      }
    } else {
      // Edge node: the nine streamed populations, split by c.n.
      R s0 = R(0), sp = R(0), g0 = R(0), gp = R(0);
#pragma unroll
      for (int k = 0; k < 9; ++k) {
        const int cx = cxk(k), cy = cyk(k);
        const int si = i - cx, sj = j - cy;
        if (si < 0 || si >= nx || sj < 0 || sj >= ny) continue;
        const int qs = q - cx - cy * H1X;
        // increments on the node's own drho and T (the edge weights add to one)
        const R fk = wk<R>(k) * ((sr[qs] - drx) + ca0[qs] + R(cx) * cbx[qs] + R(cy) * cby[qs] +
                                 R(cx * cx) * cqx[qs] + R(cy * cy) * cqy[qs] + R(cx * cy) * cqxy[qs]);
        const int cn = cx * nxo + cy * nyo;
        if (cn == 0) s0 += fk;
        else if (cn > 0) sp += fk;
        if (TH) {
          const R gk = wk<R>(k) * ((ct0[qs] - ct0[q]) + R(cx) * ctx[qs] + R(cy) * cty[qs]);
          if (cn == 0) g0 += gk;
          else if (cn > 0) gp += gk;
        }
      }
      if (cls == C_CORNER) {
        const int jn = (j == 0) ? 1 : ny - 2;
        drn = sr[(jn - y0 + 1) * H1X + (tx + 1)];
        un = vn = R(0);
      } else if (cls == C_VELOCITY) {
        un = R(0);
        if (i == 0 && j >= g.in_y0 && j <= g.in_y1) {
          un = a.u_in * inlet_profile<R>(g, j);
        }
        vn = R(0);
        drn = drx + (s0 + R(2) * sp - (un * R(nxo) + vn * R(nyo)));
      } else {
        drn = c.drho_out;
        const R unorm = (s0 + R(2) * sp) + (drx - c.drho_out);
        un = unorm * R(nxo);
        vn = unorm * R(nyo);
      }
      if (TH) {
        const int e = thermal_edge(g, i, j);
        if (g.t_kind[e] == 0) {
          Tn = c.t_val[e];
        } else if (cls == C_CORNER) {
          const int jn = (j == 0) ? 1 : ny - 2;
          Tn = sT[(jn - y0 + 2) * H2X + (tx + 2)];
        } else {
          Tn = (ct0[q] + g0 + R(2) * gp + flux_value(g, c, e, i)) / (R(1) + un * R(nxo) + vn * R(nyo));
        }
      }
    }
    const size_t o = (size_t)j * nx + i;
    a.drho_n[o] = drn;
    a.u_n[o] = un;
    a.v_n[o] = vn;
    if (TH) a.T_n[o] = Tn;
    if (a.traj_u) {
      a.traj_u[o] = un;
      a.traj_v[o] = vn;
      if (TH) a.traj_T[o] = Tn;
    }
    if (bad_velocity(un, vn)) raise_status(a.status, 4);
  }
}

// Thermal adjoint edge rule at one node (App. A, Eqs. agboundaryT / agboundaryq):
// residual r_i = (n.c_i) g~_i - B sum_j w_j (n.c_j) g~_j + m_i with the multiplier
// column m = 1 (prescribed T) or m = c.n - u.n (prescribed flux); the g~_i whose
// gather point is off the lattice and the multiplier minimise ||r||_2 over the nine
// rows (unknown links with c.n = 0 do not enter the residual and are set to zero).
// For every edge or corner normal exactly three unknown links have c.n != 0, so the
// normal equations are a 4x4 Gram system, symmetric positive definite: Gauss-Jordan
// elimination without pivoting is stable on it.  The normal is a template parameter so
// that the link sets are compile-time constants and the whole solve stays in registers
// (the double-precision pipe of this part is a small fraction of the FP32 one, so the
// solve runs in the kernel's own precision).  g[] holds the known values (zeros
// elsewhere) on entry and all nine on exit; returns the multiplier.
template <int NX, int NY>
struct EdgeLinks {
  __host__ __device__ static constexpr int cx(int k) { return k == 1 || k == 5 || k == 8 ? 1 : (k == 3 || k == 6 || k == 7 ? -1 : 0); }
  __host__ __device__ static constexpr int cy(int k) { return k == 2 || k == 5 || k == 6 ? 1 : (k == 4 || k == 7 || k == 8 ? -1 : 0); }
  __host__ __device__ static constexpr int cn(int k) { return cx(k) * NX + cy(k) * NY; }
  __host__ __device__ static constexpr bool unknown(int k) { return cx(k) * NX > 0 || cy(k) * NY > 0; }
  __host__ __device__ static constexpr int live(int a) {
    int n = 0;
    for (int k = 0; k < 9; ++k)
      if (unknown(k) && cn(k) != 0) {
        if (n == a) return k;
        ++n;
      }
    return -1;
  }
  __host__ __device__ static constexpr int nlive() {
    int n = 0;
    for (int k = 0; k < 9; ++k)
      if (unknown(k) && cn(k) != 0) ++n;
    return n;
  }
};

template <typename T, int NX, int NY>
__device__ __forceinline__ T thermal_edge_solve_n(T B, bool flux, T un, T* g) {
  using L = EdgeLinks<NX, NY>;
  constexpr int NL = 3, NC = 4;
  static_assert(L::nlive() == NL, "three unknown links with c.n != 0 on every edge normal");
  T sknown = T(0);  // sum_j w_j (n.c_j) g_j over known j
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    if (L::unknown(k))
      g[k] = T(0);
    else if (L::cn(k) != 0)
      sknown += wk<T>(k) * T(L::cn(k)) * g[k];
  }
  T G[NC][NC + 1];
#pragma unroll
  for (int a = 0; a < NC; ++a)
#pragma unroll
    for (int b = 0; b <= NC; ++b) G[a][b] = T(0);
#pragma unroll
  for (int r = 0; r < 9; ++r) {
    T col[NC];
#pragma unroll
    for (int a = 0; a < NL; ++a) {
      const int u = L::live(a);
      col[a] = (r == u ? T(L::cn(u)) : T(0)) - B * wk<T>(u) * T(L::cn(u));
    }
    col[NL] = flux ? (T(L::cn(r)) - un) : T(1);
    const T rhs = B * sknown - (L::unknown(r) ? T(0) : T(L::cn(r)) * g[r]);
#pragma unroll
    for (int a = 0; a < NC; ++a) {
#pragma unroll
      for (int b = a; b < NC; ++b) G[a][b] += col[a] * col[b];
      G[a][NC] += col[a] * rhs;
    }
  }
#pragma unroll
  for (int a = 1; a < NC; ++a)
#pragma unroll
    for (int b = 0; b < a; ++b) G[a][b] = G[b][a];
  T inv[NC];
#pragma unroll
  for (int cc = 0; cc < NC; ++cc) {
    inv[cc] = T(1) / G[cc][cc];
#pragma unroll
    for (int r = 0; r < NC; ++r) {
      if (r == cc) continue;
      const T f = G[r][cc] * inv[cc];
#pragma unroll
      for (int q = cc; q <= NC; ++q) G[r][q] -= f * G[cc][q];
    }
  }
#pragma unroll
  for (int a = 0; a < NL; ++a) g[L::live(a)] = G[a][NC] * inv[a];
  return G[NL][NC] * inv[NL];
}

template <typename T>
__device__ __forceinline__ T thermal_edge_solve(int n_x, int n_y, T B, bool flux, T un, T* g) {
  switch ((n_x + 1) * 3 + (n_y + 1)) {
    case 0: return thermal_edge_solve_n<T, -1, -1>(B, flux, un, g);
    case 1: return thermal_edge_solve_n<T, -1, 0>(B, flux, un, g);
    case 2: return thermal_edge_solve_n<T, -1, 1>(B, flux, un, g);
    case 3: return thermal_edge_solve_n<T, 0, -1>(B, flux, un, g);
    case 5: return thermal_edge_solve_n<T, 0, 1>(B, flux, un, g);
    case 6: return thermal_edge_solve_n<T, 1, -1>(B, flux, un, g);
    case 7: return thermal_edge_solve_n<T, 1, 0>(B, flux, un, g);
    case 8: return thermal_edge_solve_n<T, 1, 1>(B, flux, un, g);
    default: return T(0);  // interior nodes have no edge rule
  }
}

// =====================================================================================
// ALKS step
// =====================================================================================
template <typename R>
struct AdjArgs {
  const R* m1[9];   // adjoint moments at level t+1: rho~, u~x, u~y, s~xx, s~xy, s~yy, T~, q~x, q~y
  R* m0[9];         // adjoint moments at level t
  const R* u1;      // state at t+1 (enters f~^eq)
  const R* v1;
  const R* u0;      // state at t (objective source, sensitivity, coupling)
  const R* v0;
  const R* T0;
  const R* gamma;
  const R* emap;    // 9 classes x 6 x 10 edge moment maps (flow); column 9 is the
                    // moments' response to the heat-flux coupling kappa~ T
  R* sens;          // optional: sensitivity accumulator (interior nodes)
  int sens_flow;    // add the flow and objective terms of level t
  int sens_thermal; // add the thermal term of level t
  int* status;
};

template <bool TH>
constexpr int adj_smem_elems() {
  // 6 adjoint fields + u1, v1, u0, v0 (halo 2); P, Vx, Vy, Sxx, Sxy, Syy (halo 1)
  return 10 * H2X * H2Y + 6 * H1X * H1Y + (TH ? (3 * H2X * H2Y + 2 * H2X * H2Y + H1X * H1Y) : 0);
}

// One ALKS step (Eqs. afeq, ageq, albef, albef_ex, albeg, albeg_ex and the moments
// ap-aq).  Per node y at level t+1: P = rho~, V = 3 (u~ + 3 s~ u - rho~ u) - A D,
// D_a = 2 d_b s~_ab; f~_k(x) = P(x + c_k) + c_k . V(x + c_k).  Thermal:
// G~ = T~ + 3 q~.u - B div q~ - grad B . q~, g~_k(x) = G~(x + c_k).
template <typename R, bool TH>
__global__ void __launch_bounds__(NTHREADS) adj_step_kernel(AdjArgs<R> a, Geom g, Coef<R> c) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R* sm = reinterpret_cast<R*>(smem_raw);
  R* sa[6];
  for (int f = 0; f < 6; ++f) sa[f] = sm + f * H2X * H2Y;
  R* su1 = sm + 6 * H2X * H2Y;
  R* sv1 = su1 + H2X * H2Y;
  R* su0 = sv1 + H2X * H2Y;
  R* sv0 = su0 + H2X * H2Y;
  R* cP = sv0 + H2X * H2Y;
  R* cVx = cP + H1X * H1Y;
  R* cVy = cVx + H1X * H1Y;
  R* cSxx = cVy + H1X * H1Y;
  R* cSxy = cSxx + H1X * H1Y;
  R* cSyy = cSxy + H1X * H1Y;
  R* sTt = cSyy + H1X * H1Y;        // thermal: T~, q~x, q~y (halo 2), B, T0 (halo 2), G (halo 1)
  R* sqx = sTt + (TH ? H2X * H2Y : 0);
  R* sqy = sqx + (TH ? H2X * H2Y : 0);
  R* sB = sqy + (TH ? H2X * H2Y : 0);
  R* sT0 = sB + (TH ? H2X * H2Y : 0);
  R* cG = sT0 + (TH ? H2X * H2Y : 0);

  const int nx = g.nx, ny = g.ny;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  for (int f = 0; f < 6; ++f) stage<R, H2X, H2Y>(sa[f], a.m1[f], x0, y0, 2, nx, ny);
  stage<R, H2X, H2Y>(su1, a.u1, x0, y0, 2, nx, ny);
  stage<R, H2X, H2Y>(sv1, a.v1, x0, y0, 2, nx, ny);
  stage<R, H2X, H2Y>(su0, a.u0, x0, y0, 2, nx, ny);
  stage<R, H2X, H2Y>(sv0, a.v0, x0, y0, 2, nx, ny);
  if (TH) {
    stage<R, H2X, H2Y>(sTt, a.m1[6], x0, y0, 2, nx, ny);
    stage<R, H2X, H2Y>(sqx, a.m1[7], x0, y0, 2, nx, ny);
    stage<R, H2X, H2Y>(sqy, a.m1[8], x0, y0, 2, nx, ny);
    stage<R, H2X, H2Y>(sT0, a.T0, x0, y0, 2, nx, ny);
    for (int q = threadIdx.x; q < H2X * H2Y; q += NTHREADS) {
      const int ly = q / H2X, lx = q - ly * H2X;
      const int i = x0 - 2 + lx, j = y0 - 2 + ly;
      R b = R(0);
      if (i >= 0 && i < nx && j >= 0 && j < ny) b = B_of(c, __ldg(a.gamma + (size_t)j * nx + i));
      sB[q] = b;
    }
  }
  __syncthreads();

  for (int q = threadIdx.x; q < H1X * H1Y; q += NTHREADS) {
    const int ly = q / H1X, lx = q - ly * H1X;
    const int i = x0 - 1 + lx, j = y0 - 1 + ly;
    if (i < 0 || i >= nx || j < 0 || j >= ny) {
      cP[q] = cVx[q] = cVy[q] = cSxx[q] = cSxy[q] = cSyy[q] = R(0);
      if (TH) cG[q] = R(0);
      continue;
    }
    const int sx = lx + 1, sy = ly + 1, s2 = sy * H2X + sx;
    const R rt = sa[0][s2], ux = sa[1][s2], uy = sa[2][s2];
    const R sxx = sa[3][s2], sxy = sa[4][s2], syy = sa[5][s2];
    const R uu = su1[s2], vv = sv1[s2];
    const R Dx = R(2) * (dfdx<R, H2X>(sa[3], sx, sy, i, nx) + dfdy<R, H2X>(sa[4], sx, sy, j, ny));
    const R Dy = R(2) * (dfdx<R, H2X>(sa[4], sx, sy, i, nx) + dfdy<R, H2X>(sa[5], sx, sy, j, ny));
    cP[q] = rt;
    cVx[q] = R(3) * (ux + R(3) * (sxx * uu + sxy * vv) - rt * uu) - c.A * Dx;
    cVy[q] = R(3) * (uy + R(3) * (sxy * uu + syy * vv) - rt * vv) - c.A * Dy;
    // Strain of the level-t state, kept only on interior nodes (the objective's sum).
    if (i > 0 && j > 0 && i < nx - 1 && j < ny - 1) {
      const R dudx = (su0[s2 + 1] - su0[s2 - 1]) * R(0.5);
      const R dudy = (su0[s2 + H2X] - su0[s2 - H2X]) * R(0.5);
      const R dvdx = (sv0[s2 + 1] - sv0[s2 - 1]) * R(0.5);
      const R dvdy = (sv0[s2 + H2X] - sv0[s2 - H2X]) * R(0.5);
      cSxx[q] = R(2) * dudx;
      cSyy[q] = R(2) * dvdy;
      cSxy[q] = dudy + dvdx;
    } else {
      cSxx[q] = cSxy[q] = cSyy[q] = R(0);
    }
    if (TH) {
      const R qx = sqx[s2], qy = sqy[s2];
      const R divq = dfdx<R, H2X>(sqx, sx, sy, i, nx) + dfdy<R, H2X>(sqy, sx, sy, j, ny);
      const R dBx = dfdx<R, H2X>(sB, sx, sy, i, nx), dBy = dfdy<R, H2X>(sB, sx, sy, j, ny);
      cG[q] = sTt[s2] + R(3) * (qx * uu + qy * vv) - sB[s2] * divq - (dBx * qx + dBy * qy);
    }
  }
  __syncthreads();

  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
#pragma unroll
  for (int rr = 0; rr < TY / 8; ++rr) {
    const int oy = ty + 8 * rr;
    const int i = x0 + tx, j = y0 + oy;
    if (i >= nx || j >= ny) continue;
    const int q = (oy + 1) * H1X + (tx + 1);
    const int s2 = (oy + 2) * H2X + (tx + 2);
    const bool interior = i > 0 && j > 0 && i < nx - 1 && j < ny - 1;
    R m[9];
    if (interior) {
      R ft[9], gt[9];
#pragma unroll
      for (int k = 0; k < 9; ++k) {
        const int cx = cxk(k), cy = cyk(k);
        const int qg = q + cx + cy * H1X;
        ft[k] = cP[qg] + R(cx) * cVx[qg] + R(cy) * cVy[qg];
        if (TH) gt[k] = cG[qg];
      }
      const R w0 = R(4) / R(9), w1 = R(1) / R(9), w5 = R(1) / R(36);
      const R ax = ft[1] + ft[3], ay = ft[2] + ft[4], dg = ft[5] + ft[6] + ft[7] + ft[8];
      m[0] = w0 * ft[0] + w1 * (ax + ay) + w5 * dg;
      m[1] = w1 * (ft[1] - ft[3]) + w5 * (ft[5] - ft[6] - ft[7] + ft[8]);
      m[2] = w1 * (ft[2] - ft[4]) + w5 * (ft[5] + ft[6] - ft[7] - ft[8]);
      m[3] = w1 * ax + w5 * dg;
      m[4] = w5 * (ft[5] - ft[6] + ft[7] - ft[8]);
      m[5] = w1 * ay + w5 * dg;
      // objective source dJ_O/du (transposed strain stencil + 2 alpha u)
      const R gm = __ldg(a.gamma + (size_t)j * nx + i);
      const R al = alpha_of(c, gm);
      const R uu0 = su0[s2], vv0 = sv0[s2];
      const R ju = c.nu * (cSxx[q - 1] - cSxx[q + 1] + cSxy[q - H1X] - cSxy[q + H1X]) + R(2) * al * uu0;
      const R jv = c.nu * (cSyy[q - H1X] - cSyy[q + H1X] + cSxy[q - 1] - cSxy[q + 1]) + R(2) * al * vv0;
      R cpx = R(0), cpy = R(0);
      if (TH) {
        const R gx = gt[1] + gt[3], gy = gt[2] + gt[4], gd = gt[5] + gt[6] + gt[7] + gt[8];
        m[6] = w0 * gt[0] + w1 * (gx + gy) + w5 * gd - c.kappa_T;
        m[7] = w1 * (gt[1] - gt[3]) + w5 * (gt[5] - gt[6] - gt[7] + gt[8]);
        m[8] = w1 * (gt[2] - gt[4]) + w5 * (gt[5] + gt[6] - gt[7] - gt[8]);
        const R T0 = sT0[s2];
        cpx = T0 * m[7];
        cpy = T0 * m[8];
      }
      const R inv = R(1) / (R(1) + al);
      m[1] = (m[1] - ju * (R(1) / R(3)) + cpx) * inv;
      m[2] = (m[2] - jv * (R(1) / R(3)) + cpy) * inv;
      if (TH && has_thermal_sources(c)) m[6] = adj_thermal_T(c, gm, m[6] + c.kappa_T, m[1], m[2]);
      if (a.sens) {
        R s = R(0);
        if (a.sens_flow) {
          const R da = dalpha_of(c, gm);
          s += da * (uu0 * uu0 + vv0 * vv0) + R(3) * da * (uu0 * m[1] + vv0 * m[2]);
          if (TH) s += heat_sensitivity(c, gm, sT0[s2], m[6]);
        }
        if (TH && a.sens_thermal) {
          const R dTx = (sT0[s2 + 1] - sT0[s2 - 1]) * R(0.5);
          const R dTy = (sT0[s2 + H2X] - sT0[s2 - H2X]) * R(0.5);
          s -= dB_of(c, gm) * (dTx * m[7] + dTy * m[8]);
        }
        a.sens[(size_t)j * nx + i] += s;
      }
    } else {
      // Edge node: gathered f~ (zero where x + c_k is off the lattice) mapped to the
      // moments by the least-squares rule of the node's class.
      const int ec = edge_class(g, i, j);
      R ft[9], gt[9];
#pragma unroll
      for (int k = 0; k < 9; ++k) {
        const int cx = cxk(k), cy = cyk(k);
        const int gi = i + cx, gj = j + cy;
        const bool in = gi >= 0 && gi < nx && gj >= 0 && gj < ny;
        const int qg = q + cx + cy * H1X;
        ft[k] = in ? cP[qg] + R(cx) * cVx[qg] + R(cy) * cVy[qg] : R(0);
        if (TH) gt[k] = in ? cG[qg] : R(0);
      }
      R kT = R(0);
      if (TH) {
        // Thermal edge rule solved per node (its multiplier column depends on u.n).
        int nxo, nyo;
        node_class(g, i, j, nxo, nyo);
        const int e = thermal_edge(g, i, j);
        const bool flux = g.t_kind[e] != 0;
        const R un = su0[s2] * R(nxo) + sv0[s2] * R(nyo);
        const R kap = thermal_edge_solve<R>(nxo, nyo, B_of(c, __ldg(a.gamma + (size_t)j * nx + i)), flux, un, gt);
        R T_, qx_, qy_;
        T_ = qx_ = qy_ = R(0);
#pragma unroll
        for (int k = 0; k < 9; ++k) {
          const R gk = gt[k] * wk<R>(k);
          T_ += gk;
          qx_ += R(cxk(k)) * gk;
          qy_ += R(cyk(k)) * gk;
        }
        m[6] = T_;
        m[7] = qx_;
        m[8] = qy_;
        if (flux) kT = kap * sT0[s2];
      }
      const R* M = a.emap + ec * 60;
      R jb = edge_objective_term(g, c, ec, j);
      if (c.kappa_E != R(0)) {
        // energy loss: kappa_E u in every row of an inlet node (d/dp of its
        // integrand); on an outlet node 3 kappa_E (-3/2 u_n^2) (c_i.n) / rho_out, a
        // row term along c.n like the heat-flux coupling -kappa~ T (c_i.n), whose
        // response is column 9 of the map
        if (ec == 0 && j >= g.in_y0 && j <= g.in_y1) jb += c.kappa_E * su0[s2];
        if (ec == 1) {
          const R un = su0[s2];
          kT += R(3) * c.kappa_E * (R(1.5) * un * un) / (R(1) + c.drho_out);
        }
      }
#pragma unroll
      for (int r = 0; r < 6; ++r) {
        R s = R(0);
#pragma unroll
        for (int k = 0; k < 9; ++k) s += M[r * 10 + k] * ft[k];
        m[r] = s + M[r * 10 + 9] * kT;
        if (jb != R(0)) m[r] += jb * a.emap[540 + ec * 6 + r];
      }
    }
    const size_t o = (size_t)j * nx + i;
#pragma unroll
    for (int f = 0; f < 6; ++f) a.m0[f][o] = m[f];
    if (TH) {
      a.m0[6][o] = m[6];
      a.m0[7][o] = m[7];
      a.m0[8][o] = m[8];
    }
    if (!(m[1] * m[1] + m[2] * m[2] < R(1e30))) raise_status(a.status, 4);
  }
}

// =====================================================================================
// Objective, sensitivity, utilities
// =====================================================================================

// J_O of one state, per block into partial[block] (+= when accumulate).
template <typename R, bool TH>
__global__ void __launch_bounds__(NTHREADS) objective_kernel(const R* __restrict__ u,
                                                             const R* __restrict__ v,
                                                             const R* __restrict__ T,
                                                             const R* __restrict__ gamma, Geom g,
                                                             Coef<R> c, double* partial) {
  __shared__ double red[NTHREADS / 32];
  const int nx = g.nx, ny = g.ny;
  double acc = 0.0;
  const size_t N = (size_t)nx * ny;
  for (size_t o = (size_t)blockIdx.x * NTHREADS + threadIdx.x; o < N; o += (size_t)gridDim.x * NTHREADS) {
    const int j = (int)(o / nx), i = (int)(o - (size_t)j * nx);
    if (i == 0 || j == 0 || i == nx - 1 || j == ny - 1) continue;
    const R dudx = (u[o + 1] - u[o - 1]) * R(0.5), dudy = (u[o + nx] - u[o - nx]) * R(0.5);
    const R dvdx = (v[o + 1] - v[o - 1]) * R(0.5), dvdy = (v[o + nx] - v[o - nx]) * R(0.5);
    const R Sxx = R(2) * dudx, Syy = R(2) * dvdy, Sxy = dudy + dvdx;
    const R al = alpha_of(c, gamma[o]);
    acc += (double)(R(0.5) * c.nu * (Sxx * Sxx + R(2) * Sxy * Sxy + Syy * Syy) +
                    al * (u[o] * u[o] + v[o] * v[o]));
    if (TH) acc += (double)(c.kappa_T * T[o] + heat_objective(c, gamma[o], T[o]));
  }
  const double s = block_sum(acc, red);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

// Boundary objectives of one state: the static pressure drop of Eq.
// objective_pipebend, kappa_p J_p with J_p = 1/3 (sum of rho over the inlet nodes -
// over the outlet nodes) (p = rho / 3, dGamma = 1; inlet: left face inside the inlet
// span, corners excluded; outlet: the pressure nodes), plus the energy loss
// kappa_E J_E on the same nodes (energy_loss_node).  One block; drho = rho - 1 is the
// stored density.
template <typename R>
__global__ void __launch_bounds__(NTHREADS) boundary_objective_kernel(const R* __restrict__ drho,
                                                                      const R* __restrict__ u,
                                                                      const R* __restrict__ v, Geom g, Coef<R> c,
                                                                      double* out) {
  __shared__ double red[NTHREADS / 32];
  double acc = 0.0, accE = 0.0;
  for (int j = 1 + threadIdx.x; j < g.ny - 1; j += NTHREADS) {
    const size_t l = (size_t)j * g.nx, r = l + g.nx - 1;
    if (j >= g.in_y0 && j <= g.in_y1) acc += 1.0 + (double)drho[l];
    if (j >= g.out_y0 && j <= g.out_y1) acc -= 1.0 + (double)drho[r];
    if (c.kappa_E != R(0))
      accE += energy_loss_node(g, c, 0, j, drho[l], u[l], v[l]) + energy_loss_node(g, c, g.nx - 1, j, drho[r], u[r], v[r]);
  }
  const double s = block_sum((double)c.kappa_p * acc / 3.0 + accE, red);
  if (threadIdx.x == 0) *out = s;
}

// Deterministic sum of n partials (one block) plus an optional second array.
static __global__ void reduce_partials_kernel(const double* __restrict__ p, int n, const double* __restrict__ p2,
                                       int n2, double* out) {
  __shared__ double red[NTHREADS / 32];
  double acc = 0.0;
  for (int q = threadIdx.x; q < n; q += NTHREADS) acc += p[q];
  for (int q = threadIdx.x; q < n2; q += NTHREADS) acc += p2[q];
  const double s = block_sum(acc, red);
  if (threadIdx.x == 0) *out = s;
}

// Steady sensitivity of the final state (Sec. 2.5): interior nodes, zero on edges.
template <typename R, bool TH>
__global__ void __launch_bounds__(NTHREADS) sensitivity_kernel(const R* __restrict__ u,
                                                               const R* __restrict__ v,
                                                               const R* __restrict__ T,
                                                               const R* __restrict__ ux_t,
                                                               const R* __restrict__ uy_t,
                                                               const R* __restrict__ T_t,
                                                               const R* __restrict__ qx_t,
                                                               const R* __restrict__ qy_t,
                                                               const R* __restrict__ gamma, Geom g,
                                                               Coef<R> c, R* __restrict__ out) {
  const int nx = g.nx, ny = g.ny;
  const size_t N = (size_t)nx * ny;
  for (size_t o = (size_t)blockIdx.x * NTHREADS + threadIdx.x; o < N; o += (size_t)gridDim.x * NTHREADS) {
    const int j = (int)(o / nx), i = (int)(o - (size_t)j * nx);
    R s = R(0);
    if (!(i == 0 || j == 0 || i == nx - 1 || j == ny - 1)) {
      const R gm = gamma[o];
      const R da = dalpha_of(c, gm);
      const R uu = u[o], vv = v[o];
      s = da * (uu * uu + vv * vv) + R(3) * da * (uu * ux_t[o] + vv * uy_t[o]);
      if (TH) {
        const R dTx = (T[o + 1] - T[o - 1]) * R(0.5), dTy = (T[o + nx] - T[o - nx]) * R(0.5);
        s -= dB_of(c, gm) * (dTx * qx_t[o] + dTy * qy_t[o]);
        s += heat_sensitivity(c, gm, T[o], T_t[o]);
      }
    }
    out[o] = s;
  }
}

// y = x (+ shift), element type R -> S.
template <typename R, typename S>
__global__ void copy_shift_kernel(const R* __restrict__ x, S* __restrict__ y, size_t n, R shift) {
  for (size_t o = (size_t)blockIdx.x * blockDim.x + threadIdx.x; o < n; o += (size_t)gridDim.x * blockDim.x)
    y[o] = (S)(x[o] + shift);
}

// Change of one step of two fields: out[0] = max over nodes of |a1 - a0| + |b1 - b0|,
// out[1] = max of |a1| + |b1|, both as the bits of non-negative floats (which order
// like the values, so an integer maximum finds them).  out is zeroed by the caller.
template <typename R>
__global__ void change_kernel(const R* __restrict__ a0, const R* __restrict__ a1, const R* __restrict__ b0,
                              const R* __restrict__ b1, size_t n, unsigned* __restrict__ out) {
  float dm = 0.f, mm = 0.f;
  for (size_t o = (size_t)blockIdx.x * blockDim.x + threadIdx.x; o < n; o += (size_t)gridDim.x * blockDim.x) {
    dm = fmaxf(dm, (float)(fabs(a1[o] - a0[o]) + fabs(b1[o] - b0[o])));
    mm = fmaxf(mm, (float)(fabs(a1[o]) + fabs(b1[o])));
  }
  for (int off = 16; off > 0; off >>= 1) {
    dm = fmaxf(dm, __shfl_xor_sync(0xffffffffu, dm, off));
    mm = fmaxf(mm, __shfl_xor_sync(0xffffffffu, mm, off));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(out, __float_as_uint(dm));
    atomicMax(out + 1, __float_as_uint(mm));
  }
}

// Accumulate a in FP64: acc += a; then a = 0.
template <typename R>
__global__ void flush_accum_kernel(R* __restrict__ a, double* __restrict__ acc, size_t n) {
  for (size_t o = (size_t)blockIdx.x * blockDim.x + threadIdx.x; o < n; o += (size_t)gridDim.x * blockDim.x) {
    acc[o] += (double)a[o];
    a[o] = R(0);
  }
}

}  // namespace lks
