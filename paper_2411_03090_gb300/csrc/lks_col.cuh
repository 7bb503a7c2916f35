// lks_col.cuh -- warp-column forms of the FP32 LKS and ALKS steps of one lattice
// (non-thermal).
//
// A warp owns adjacent lattice columns and marches down its rows with the values of
// three rows held in registers.  A lane computes the per-node coefficients of its
// column(s) (the arithmetic of the TMA-staged kernels, term for term), hands the
// values that cross a column to the neighbour lane by warp shuffle, and completes a
// row once the row below it has been processed.  Each tile is staged by one tensor
// copy per field (its halo included, x on a 16-byte boundary); there is no shared
// push array and no barrier inside a tile.  Tiles whose halo reaches the domain edge
// run the same march with the edge rules (one-sided derivatives, continuity, Zou-He
// edges, corners).
#pragma once
#include "lks_tma.cuh"

namespace lks {

constexpr int COL_W = 28;     // adjoint: output columns per warp (32 lanes, 2 halo lanes per side)
constexpr int COL_WARPS = 4;  // warps per CTA, stacked in y
constexpr int COL_BW = COL_W + 8;
constexpr int COL_NT = 32 * COL_WARPS;

// ---------------------------------------------------------------------------------
// Warp-column forward with two columns per lane
// ---------------------------------------------------------------------------------
// Lane l owns the columns x0 - 2 + 2l and x0 - 1 + 2l and marches down R rows with
// three rows of values in registers.  A row pushes the nine populations of both
// nodes and completes the row above it.  Neighbours inside the lane pair need no
// shuffle; a row costs two
// shuffles per field crossing the lane boundary and six for the populations moving
// to the neighbour lanes, and its loads and stores are 8-byte vectors.  Lanes 1..30
// write, so a tile is 60 columns wide; tiles start at x = 0 (the first box starts
// at x = -4 and reads zeros left of the lattice).  nx even keeps a lane's two
// columns both inside or both outside the lattice.  Tiles at least two nodes inside
// the lattice take the march without edge tests; the others recompute velocity
// gradients at edge nodes from the staged box (one-sided differences, continuity)
// and apply the edge rules of Sec. 2.4 at the output.  The per-node arithmetic is
// push9 / gather9, as in the other FP32 staged kernels.
constexpr int C2_W = 60;
constexpr int C2_BW = C2_W + 8;
template <int R>
struct Col2Geo {
  static constexpr int H = COL_WARPS * R;  // output rows per tile
  static constexpr int BH = H + 4, BOX = C2_BW * BH;
  static constexpr int FS = (BOX * 4 + 127) / 128 * 128 / 4;  // field stride: 128-byte aligned copies
  static constexpr size_t smem = (size_t)4 * FS * 4 + 128 + 8 + 8 * COL_WARPS;
  static_assert((R + 2) % 3 == 0, "the unrolled march covers R + 2 rows in threes");
};
constexpr int C2_R = 10;

struct Col2Args {
  float* out[3];      // drho, u, v of the new level
  float* traj_u;      // optional trajectory copies of u, v
  float* traj_v;
  double* J_partial;  // per-tile accumulator of J_O(old state), or null
  int* status;
  float u_in;         // inlet amplitude of the new level (single lattice)
  int ntx;            // tiles along x (single lattice)
  // batched form: one work-list entry per CTA, per-design tables, arena row pitch
  const BatchTile* work;
  const BatchDesign* designs;
  const float* u_in_d;  // inlet amplitude of the new level, per design
  int pitch;
};

// BATCH: the lattices of many designs packed in one arena (tile origins and the
// interior flag from the work list; geometry, coefficients and inlet amplitude from
// the design table; fields addressed with the arena pitch, nx may be odd).
template <int R, bool BATCH>
__global__ void __launch_bounds__(COL_NT) fwd_col2_kernel(const __grid_constant__ TmaMaps<4> maps,
                                                          const __grid_constant__ Col2Args a,
                                                          const __grid_constant__ Geom g0,
                                                          const __grid_constant__ Coef<float> c0) {
  using G2 = Col2Geo<R>;
  constexpr int BW = C2_BW, FS = G2::FS;
  extern __shared__ unsigned char smem_raw[];
  float* box = reinterpret_cast<float*>(smem_base128(smem_raw));  // [drho, u, v, 1/(1+alpha)][FS]
  uint64_t* bar = reinterpret_cast<uint64_t*>(box + 4 * FS);
  double* red = reinterpret_cast<double*>(bar + 1);
  if (timed_out_before(a.status)) return;
  if (!tma_layout_ok(box, bar, a.status)) return;
  int x0, y0, ax = 0, ay = 0;
  bool fast;
  const Geom* gp = &g0;
  const Coef<float>* cp = &c0;
  float u_in = a.u_in;
  size_t pitch;
  if constexpr (BATCH) {
    const BatchTile w = a.work[blockIdx.x];
    const BatchDesign& bd = a.designs[w.d];
    gp = &bd.g;
    cp = &bd.c;
    x0 = w.x0;
    y0 = w.y0;
    ax = bd.ax;
    ay = bd.ay;
    fast = w.interior != 0;
    u_in = a.u_in_d[w.d];
    pitch = (size_t)a.pitch;
  } else {
    x0 = (int)(blockIdx.x % a.ntx) * C2_W;
    y0 = (int)(blockIdx.x / a.ntx) * G2::H;
    fast = x0 >= 2 && x0 + C2_W + 2 <= g0.nx && y0 >= 2 && y0 + G2::H + 2 <= g0.ny;
    pitch = (size_t)g0.nx;
  }
  // copies held in registers: the kernel's global stores could alias the design
  // table, so references into it would be re-read inside the march
  const Geom g = *gp;
  const Coef<float> c = *cp;
  const int nx = g.nx, ny = g.ny;
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
    fence_proxy_async();
    mbar_expect_tx(bar, 4 * G2::BOX * 4);
    for (int f = 0; f < 4; ++f) tma_load_2d(box + f * FS, &maps.m[f], ax + x0 - TMA_BXPAD, ay + y0 - 2, bar);
  }
  __syncthreads();
  if (!mbar_wait(bar, 0)) {
    raise_status(a.status, 6);
    if (threadIdx.x == 0) mbar_wait(bar, 0);
    return;
  }
  const float* sdr = box;
  const float* su = box + FS;
  const float* sv = box + 2 * FS;
  const float* sbi = box + 3 * FS;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int i0 = x0 - 2 + 2 * lane;         // the lane's first lattice column
  const int bx = TMA_BXPAD - 2 + 2 * lane;  // its column in the box (even: 8-byte aligned)
  const int r0 = y0 + warp * R;
  const bool out_lane = lane >= 1 && lane <= 30 && i0 >= 0 && i0 < nx;
  const bool out1 = i0 + 1 < nx;  // second column inside too (always, for even nx)
  auto brow = [&](int y) { return (y - y0 + 2) * BW; };
  double jloc = 0.0;
  bool bad = false;

  struct Row {
    float2 d, u, v;  // drho, u, v of the lane's two columns
    float dl, dr;    // drho of the columns left and right of the pair
  };
  auto load_row = [&](Row& Q, int y) {
    const int o = brow(y) + bx;
    Q.d = *reinterpret_cast<const float2*>(sdr + o);
    Q.u = *reinterpret_cast<const float2*>(su + o);
    Q.v = *reinterpret_cast<const float2*>(sv + o);
    Q.dl = __shfl_up_sync(0xffffffffu, Q.d.y, 1);
    Q.dr = __shfl_down_sync(0xffffffffu, Q.d.x, 1);
  };
  // Velocity gradients of an edge-tile node at lattice (i, p), box column bc: the
  // one-sided differences and the continuity rule of the edge nodes.
  auto edge_grad = [&](int i, int p, int bc, float& dudx, float& dudy, float& dvdx, float& dvdy) {
    const int by = p - y0 + 2;
    dudx = dfdx<float, BW>(su, bc, by, i, nx);
    dudy = dfdy<float, BW>(su, bc, by, p, ny);
    dvdx = dfdx<float, BW>(sv, bc, by, i, nx);
    dvdy = dfdy<float, BW>(sv, bc, by, p, ny);
    const bool xe = (i == 0 || i == nx - 1), ye = (p == 0 || p == ny - 1);
    if (xe && ye) {
      dudx = 0.f;
      dvdy = 0.f;
    } else if (xe) {
      dudx = -dvdy;
    } else if (ye) {
      dvdy = -dudx;
    }
  };
  // New level of the lattice node (i, q), box column bc, from the populations fk
  // arriving there (fk[k] = F_k(x - c_k)): the interior gather, or the edge rule.
  auto out_node = [&](int i, int q, int bc, const float* fk, float drx, float inv, float& drn, float& un,
                      float& vn) {
    int nxo = 0, nyo = 0;
    const int cls = node_class(g, i, q, nxo, nyo);
    if (cls == C_INTERIOR) {
      gather9(fk, drx, inv, drn, un, vn);
      return;
    }
    float s0 = 0.f, sp = 0.f;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      const int cx = cxk(k), cy = cyk(k);
      const int si = i - cx, sj = q - cy;
      if (si < 0 || si >= nx || sj < 0 || sj >= ny) continue;
      const int cn = cx * nxo + cy * nyo;
      if (cn == 0) s0 += fk[k];
      else if (cn > 0) sp += fk[k];
    }
    if (cls == C_CORNER) {
      drn = sdr[brow(q == 0 ? 1 : ny - 2) + bc];
      un = vn = 0.f;
    } else if (cls == C_VELOCITY) {
      un = (i == 0 && q >= g.in_y0 && q <= g.in_y1) ? u_in * inlet_profile<float>(g, q) : 0.f;
      vn = 0.f;
      drn = __fadd_rn(drx, __fsub_rn(__fmaf_rn(2.f, sp, s0), __fmaf_rn(vn, (float)nyo, __fmul_rn(un, (float)nxo))));
    } else {
      drn = c.drho_out;
      const float unorm = __fadd_rn(__fmaf_rn(2.f, sp, s0), __fsub_rn(drx, c.drho_out));
      un = __fmul_rn(unorm, (float)nxo);
      vn = __fmul_rn(unorm, (float)nyo);
    }
  };
  // Destination row of the march: the nine populations arriving at each column.
  struct Dst {
    float a[9], b[9];
  };
  // Row p: A, B, C hold rows p-1, p, p+1; X, Y, Z collect destination rows p-1, p,
  // p+1.  Row p-1 is complete afterwards and is written; row p+2 is loaded into A.
  auto step = [&](auto edge_tag, int p, Row& A, Row& B, Row& C, Dst& X, Dst& Y, Dst& Z) {
    constexpr bool EDGE = decltype(edge_tag)::value;
    const float uL = __shfl_up_sync(0xffffffffu, B.u.y, 1), uR = __shfl_down_sync(0xffffffffu, B.u.x, 1);
    const float vL = __shfl_up_sync(0xffffffffu, B.v.y, 1), vR = __shfl_down_sync(0xffffffffu, B.v.x, 1);
    float gr0[4] = {cdiff(B.u.y, uL), cdiff(C.u.x, A.u.x), cdiff(B.v.y, vL), cdiff(C.v.x, A.v.x)};
    float gr1[4] = {cdiff(uR, B.u.x), cdiff(C.u.y, A.u.y), cdiff(vR, B.v.x), cdiff(C.v.y, A.v.y)};
    if (EDGE) {
      const bool ye = p == 0 || p == ny - 1;
      if (i0 == 0 || i0 == nx - 1 || ye) edge_grad(i0, p, bx, gr0[0], gr0[1], gr0[2], gr0[3]);
      if (i0 + 1 == nx - 1 || ye) edge_grad(i0 + 1, p, bx + 1, gr1[0], gr1[1], gr1[2], gr1[3]);
    }
    float F0[9], F1[9];
    {
      const float dn[9] = {0.f, B.d.y, C.d.x, B.dl, A.d.x, C.d.y, C.dl, A.dl, A.d.y};
      push9(B.d.x, dn, B.u.x, B.v.x, gr0[0], gr0[1], gr0[2], gr0[3], c.A, F0);
    }
    {
      const float dn[9] = {0.f, B.dr, C.d.y, B.d.x, A.d.y, C.dr, C.d.x, A.d.x, A.dr};
      push9(B.d.y, dn, B.u.y, B.v.y, gr1[0], gr1[1], gr1[2], gr1[3], c.A, F1);
    }
    // objective of the old state at the interior output nodes of row p
    if (a.J_partial && out_lane && p >= r0 && p < r0 + R && (!EDGE || (p > 0 && p < ny - 1))) {
      const int s2 = brow(p) + bx;
      const float2 inv = *reinterpret_cast<const float2*>(sbi + s2);
      if (!EDGE || i0 > 0) jloc += (double)jo_flow<BW>(su, sv, s2, c.nu, inv.x, B.u.x, B.v.x);
      if (!EDGE || i0 + 1 < nx - 1) jloc += (double)jo_flow<BW>(su, sv, s2 + 1, c.nu, inv.y, B.u.y, B.v.y);
    }
    // populations of the first column moving left go to the previous lane's second
    // column; those of the second column moving right to the next lane's first
    const float r7 = __shfl_down_sync(0xffffffffu, F0[7], 1), r3 = __shfl_down_sync(0xffffffffu, F0[3], 1);
    const float r6 = __shfl_down_sync(0xffffffffu, F0[6], 1);
    const float l8 = __shfl_up_sync(0xffffffffu, F1[8], 1), l1 = __shfl_up_sync(0xffffffffu, F1[1], 1);
    const float l5 = __shfl_up_sync(0xffffffffu, F1[5], 1);
    X.a[4] = F0[4], X.a[7] = F1[7], X.a[8] = l8;  // c_y = -1: destination row p - 1
    X.b[4] = F1[4], X.b[7] = r7, X.b[8] = F0[8];
    Y.a[0] = F0[0], Y.a[1] = l1, Y.a[3] = F1[3];  // c_y = 0: destination row p
    Y.b[0] = F1[0], Y.b[1] = F0[1], Y.b[3] = r3;
    Z.a[2] = F0[2], Z.a[5] = l5, Z.a[6] = F1[6];  // c_y = +1: destination row p + 1
    Z.b[2] = F1[2], Z.b[5] = F0[5], Z.b[6] = r6;
    const int q = p - 1;
    if (q >= r0 && out_lane && (!EDGE || q < ny)) {
      const float2 inv = *reinterpret_cast<const float2*>(sbi + brow(q) + bx);
      float2 dn, un, vn;
      const size_t o = (size_t)(ay + q) * pitch + (size_t)(ax + i0);
      if (EDGE) {
        out_node(i0, q, bx, X.a, A.d.x, inv.x, dn.x, un.x, vn.x);
        if (out1) {
          out_node(i0 + 1, q, bx + 1, X.b, A.d.y, inv.y, dn.y, un.y, vn.y);
        } else {  // odd nx (batched designs): the pair's second column lies outside
          a.out[0][o] = dn.x;
          a.out[1][o] = un.x;
          a.out[2][o] = vn.x;
          if (a.traj_u) {
            a.traj_u[o] = un.x;
            a.traj_v[o] = vn.x;
          }
          bad |= bad_velocity(un.x, vn.x);
        }
      } else {
        gather9(X.a, A.d.x, inv.x, dn.x, un.x, vn.x);
        gather9(X.b, A.d.y, inv.y, dn.y, un.y, vn.y);
      }
      if (!EDGE || out1) {
        *reinterpret_cast<float2*>(a.out[0] + o) = dn;
        *reinterpret_cast<float2*>(a.out[1] + o) = un;
        *reinterpret_cast<float2*>(a.out[2] + o) = vn;
        if (a.traj_u) {
          *reinterpret_cast<float2*>(a.traj_u + o) = un;
          *reinterpret_cast<float2*>(a.traj_v + o) = vn;
        }
        bad |= bad_velocity(un.x, vn.x) | bad_velocity(un.y, vn.y);
      }
    }
    if (p + 2 <= r0 + R + 1) load_row(A, p + 2);
  };
  Row R0, R1, R2;
  Dst X0, X1, X2;
  load_row(R0, r0 - 2);
  load_row(R1, r0 - 1);
  load_row(R2, r0);
  if (fast) {  // unrolled by three rows: the register rings rotate by renaming
#pragma unroll 1
    for (int p = r0 - 1; p <= r0 + R; p += 3) {
      step(std::false_type{}, p, R0, R1, R2, X0, X1, X2);
      step(std::false_type{}, p + 1, R1, R2, R0, X1, X2, X0);
      step(std::false_type{}, p + 2, R2, R0, R1, X2, X0, X1);
    }
  } else {  // edge tiles: one row per iteration and explicit rotation, a third of the
            // code (batched lattices run edge and interior tiles side by side)
#pragma unroll 1
    for (int p = r0 - 1; p <= r0 + R; ++p) {
      step(std::true_type{}, p, R0, R1, R2, X0, X1, X2);
      const Row t = R0;
      R0 = R1;
      R1 = R2;
      R2 = t;
      const Dst u = X0;
      X0 = X1;
      X1 = X2;
      X2 = u;
    }
  }
  if (bad) raise_status(a.status, 4);
  if (a.J_partial) {
    const double s = block_sum<COL_NT>(jloc, red);
    if (threadIdx.x == 0) a.J_partial[blockIdx.x] += s;
  }
}

// ---------------------------------------------------------------------------------
// Warp-column thermal forward (the temperature lattice; runs after fwd_col2_kernel)
// ---------------------------------------------------------------------------------
// T of the new level depends on T, u, v and B of the old level (Eq. geq2); only the
// heat-flux edge rule also takes the new normal velocity of its node, which the flow
// kernel of the same step has written.  Same tiles, lane pairs and march as
// fwd_col2_kernel; the per-node arithmetic is gpush9 / tgather8 / tflux_edge, as in
// fwd_tma_kernel<TH = true>.
struct ColTArgs {
  float* T_out;         // T of the new level
  float* traj_T;        // optional trajectory copy of T
  const float* u_new;   // new u, v written by the flow kernel (heat-flux edges)
  const float* v_new;
  double* J_partial;    // per-tile accumulator of kappa_T T (old level), or null
  int* status;
  int ntx;
};

// Staged fields: T, u, v (old level), B.
template <int R>
__global__ void __launch_bounds__(COL_NT) fwd_colT_kernel(const __grid_constant__ TmaMaps<4> maps,
                                                          const __grid_constant__ ColTArgs a,
                                                          const __grid_constant__ Geom g,
                                                          const __grid_constant__ Coef<float> c) {
  using G2 = Col2Geo<R>;
  constexpr int BW = C2_BW, FS = G2::FS;
  extern __shared__ unsigned char smem_raw[];
  float* box = reinterpret_cast<float*>(smem_base128(smem_raw));
  uint64_t* bar = reinterpret_cast<uint64_t*>(box + 4 * FS);
  double* red = reinterpret_cast<double*>(bar + 1);
  if (timed_out_before(a.status)) return;
  if (!tma_layout_ok(box, bar, a.status)) return;
  const int nx = g.nx, ny = g.ny;
  const int x0 = (int)(blockIdx.x % a.ntx) * C2_W, y0 = (int)(blockIdx.x / a.ntx) * G2::H;
  const bool fast = x0 >= 2 && x0 + C2_W + 2 <= nx && y0 >= 2 && y0 + G2::H + 2 <= ny;
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
    fence_proxy_async();
    mbar_expect_tx(bar, 4 * G2::BOX * 4);
    for (int f = 0; f < 4; ++f) tma_load_2d(box + f * FS, &maps.m[f], x0 - TMA_BXPAD, y0 - 2, bar);
  }
  __syncthreads();
  if (!mbar_wait(bar, 0)) {
    raise_status(a.status, 6);
    if (threadIdx.x == 0) mbar_wait(bar, 0);
    return;
  }
  const float* sT = box;
  const float* su = box + FS;
  const float* sv = box + 2 * FS;
  const float* sB = box + 3 * FS;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int i0 = x0 - 2 + 2 * lane;
  const int bx = TMA_BXPAD - 2 + 2 * lane;
  const int r0 = y0 + warp * R;
  const bool out_lane = lane >= 1 && lane <= 30 && i0 >= 0 && i0 < nx;
  auto brow = [&](int y) { return (y - y0 + 2) * BW; };
  double jloc = 0.0;

  struct Row {
    float2 T, u, v;  // T, u, v of the lane's two columns
    float Tl, Tr;    // T of the columns left and right of the pair
  };
  auto load_row = [&](Row& Q, int y) {
    const int o = brow(y) + bx;
    Q.T = *reinterpret_cast<const float2*>(sT + o);
    Q.u = *reinterpret_cast<const float2*>(su + o);
    Q.v = *reinterpret_cast<const float2*>(sv + o);
    Q.Tl = __shfl_up_sync(0xffffffffu, Q.T.y, 1);
    Q.Tr = __shfl_down_sync(0xffffffffu, Q.T.x, 1);
  };
  // New T of the lattice node (i, q), box column bc, from the populations gk arriving
  // there: the interior gather or the thermal edge rule.
  auto out_node = [&](int i, int q, int bc, const float* gk, float TT) {
    int nxo = 0, nyo = 0;
    const int cls = node_class(g, i, q, nxo, nyo);
    if (cls == C_INTERIOR) return tgather8(TT, gk);
    const int e = thermal_edge(g, i, q);
    if (g.t_kind[e] == 0) return c.t_val[e];
    if (cls == C_CORNER) return sT[brow(q == 0 ? 1 : ny - 2) + bc];
    float g0 = 0.f, gp = 0.f;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      const int cx = cxk(k), cy = cyk(k);
      const int si = i - cx, sj = q - cy;
      if (si < 0 || si >= nx || sj < 0 || sj >= ny) continue;
      const int cn = cx * nxo + cy * nyo;
      if (cn == 0) g0 += gk[k];
      else if (cn > 0) gp += gk[k];
    }
    const size_t o = (size_t)q * nx + i;
    return tflux_edge(TT, g0, gp, flux_value(g, c, e, i), a.u_new[o], a.v_new[o], nxo, nyo);
  };
  struct Dst {
    float a[9], b[9];
  };
  auto step = [&](auto edge_tag, int p, Row& A, Row& B, Row& C, Dst& X, Dst& Y, Dst& Z) {
    constexpr bool EDGE = decltype(edge_tag)::value;
    float dT0[2] = {cdiff(B.T.y, B.Tl), cdiff(C.T.x, A.T.x)};
    float dT1[2] = {cdiff(B.Tr, B.T.x), cdiff(C.T.y, A.T.y)};
    if (EDGE) {
      const int by = p - y0 + 2;
      const bool ye = p == 0 || p == ny - 1;
      if (i0 == 0 || i0 == nx - 1 || ye) {
        dT0[0] = dfdx<float, BW>(sT, bx, by, i0, nx);
        dT0[1] = dfdy<float, BW>(sT, bx, by, p, ny);
      }
      if (i0 + 1 == nx - 1 || ye) {
        dT1[0] = dfdx<float, BW>(sT, bx + 1, by, i0 + 1, nx);
        dT1[1] = dfdy<float, BW>(sT, bx + 1, by, p, ny);
      }
    }
    const float2 Bn = *reinterpret_cast<const float2*>(sB + brow(p) + bx);
    float G0[9], G1[9];
    {
      const float tn[9] = {0.f, B.T.y, C.T.x, B.Tl, A.T.x, C.T.y, C.Tl, A.Tl, A.T.y};
      gpush9(B.T.x, tn, B.u.x, B.v.x, dT0[0], dT0[1], Bn.x, G0);
    }
    {
      const float tn[9] = {0.f, B.Tr, C.T.y, B.T.x, A.T.y, C.Tr, C.T.x, A.T.x, A.Tr};
      gpush9(B.T.y, tn, B.u.y, B.v.y, dT1[0], dT1[1], Bn.y, G1);
    }
    // objective term kappa_T T of the old level at the interior output nodes of row p
    if (a.J_partial && out_lane && p >= r0 && p < r0 + R && (!EDGE || (p > 0 && p < ny - 1))) {
      if (!EDGE || i0 > 0) jloc += (double)__fmul_rn(c.kappa_T, B.T.x);
      if (!EDGE || i0 + 1 < nx - 1) jloc += (double)__fmul_rn(c.kappa_T, B.T.y);
    }
    const float r7 = __shfl_down_sync(0xffffffffu, G0[7], 1), r3 = __shfl_down_sync(0xffffffffu, G0[3], 1);
    const float r6 = __shfl_down_sync(0xffffffffu, G0[6], 1);
    const float l8 = __shfl_up_sync(0xffffffffu, G1[8], 1), l1 = __shfl_up_sync(0xffffffffu, G1[1], 1);
    const float l5 = __shfl_up_sync(0xffffffffu, G1[5], 1);
    X.a[4] = G0[4], X.a[7] = G1[7], X.a[8] = l8;
    X.b[4] = G1[4], X.b[7] = r7, X.b[8] = G0[8];
    Y.a[0] = G0[0], Y.a[1] = l1, Y.a[3] = G1[3];
    Y.b[0] = G1[0], Y.b[1] = G0[1], Y.b[3] = r3;
    Z.a[2] = G0[2], Z.a[5] = l5, Z.a[6] = G1[6];
    Z.b[2] = G1[2], Z.b[5] = G0[5], Z.b[6] = r6;
    const int q = p - 1;
    if (q >= r0 && out_lane && (!EDGE || q < ny)) {
      const size_t o = (size_t)q * nx + i0;
      float2 Tn;
      if (EDGE) {
        Tn.x = out_node(i0, q, bx, X.a, A.T.x);
        Tn.y = out_node(i0 + 1, q, bx + 1, X.b, A.T.y);
      } else {
        Tn.x = tgather8(A.T.x, X.a);
        Tn.y = tgather8(A.T.y, X.b);
      }
      *reinterpret_cast<float2*>(a.T_out + o) = Tn;
      if (a.traj_T) *reinterpret_cast<float2*>(a.traj_T + o) = Tn;
    }
    if (p + 2 <= r0 + R + 1) load_row(A, p + 2);
  };
  Row R0, R1, R2;
  Dst X0, X1, X2;
  load_row(R0, r0 - 2);
  load_row(R1, r0 - 1);
  load_row(R2, r0);
  if (fast) {
#pragma unroll 1
    for (int p = r0 - 1; p <= r0 + R; p += 3) {
      step(std::false_type{}, p, R0, R1, R2, X0, X1, X2);
      step(std::false_type{}, p + 1, R1, R2, R0, X1, X2, X0);
      step(std::false_type{}, p + 2, R2, R0, R1, X2, X0, X1);
    }
  } else {
#pragma unroll 1
    for (int p = r0 - 1; p <= r0 + R; ++p) {
      step(std::true_type{}, p, R0, R1, R2, X0, X1, X2);
      const Row t = R0;
      R0 = R1;
      R1 = R2;
      R2 = t;
      const Dst u = X0;
      X0 = X1;
      X1 = X2;
      X2 = u;
    }
  }
  if (a.J_partial) {
    const double sj = block_sum<COL_NT>(jloc, red);
    if (threadIdx.x == 0) a.J_partial[blockIdx.x] += sj;
  }
}

// ---------------------------------------------------------------------------------
// Warp-column ALKS step (FP32, non-thermal, one lattice)
// ---------------------------------------------------------------------------------
// The same march for the adjoint: a lane computes P + c_k . V (Eq. afeq) of its node
// for the nine links and the strain of the level-t state, hands the values a
// neighbouring column gathers to it by shuffle, and completes the moments of a row
// once the row below has been computed.  One column per lane (lanes 2..29 write),
// tiles of 28 x 32 outputs (four warps of eight rows); the per-node arithmetic is
// that of adj_tma_kernel, term for term.  The batched form runs the same kernel over
// a (design, tile) work list.
constexpr int ACOL_R = 8;
constexpr int ACOL_H = COL_WARPS * ACOL_R;
constexpr int ACOL_BH = ACOL_H + 4, ACOL_BOX = COL_BW * ACOL_BH;
constexpr int ACOL_FS = (ACOL_BOX * 4 + 127) / 128 * 128 / 4;

__host__ __device__ constexpr int acol_nf(bool same) { return same ? 10 : 12; }
// staged fields, alignment slack, the mbarrier, the edge maps (9 classes x 60)
__host__ __device__ constexpr size_t acol_smem_bytes(bool same) {
  return (size_t)acol_nf(same) * ACOL_FS * 4 + 128 + 8 + kEdgeMapLen * 4;
}

struct AdjColArgs {
  float* m0[6];       // adjoint moments at level t
  const float* gamma;
  const float* emap;  // kEdgeMapLen values (batched form: per design, the 540 maps only)
  float* sens;        // optional sensitivity accumulator
  int sens_flow;
  int* status;
  int ntx;            // tiles along x (single lattice)
  // batched form: one work-list entry per CTA, per-design tables, arena row pitch
  const BatchTile* work;
  const BatchDesign* designs;
  int pitch;
};

// Staged fields: rho~, u~x, u~y, s~xx, s~xy, s~yy, u1, v1, [u0, v0], alpha, 1/(1+alpha).
// BATCH: the designs of a batch packed in one arena, as for fwd_col2_kernel.
template <bool SAME, bool BATCH>
__global__ void __launch_bounds__(COL_NT) adj_col_kernel(const __grid_constant__ TmaMaps<acol_nf(SAME)> maps,
                                                         const __grid_constant__ AdjColArgs a,
                                                         const __grid_constant__ Geom g0,
                                                         const __grid_constant__ Coef<float> c0) {
  constexpr int NF = acol_nf(SAME);
  constexpr int FU0 = SAME ? 6 : 8, FAL = SAME ? 8 : 10, FBI = FAL + 1;
  constexpr int BW = COL_BW;
  extern __shared__ unsigned char smem_raw[];
  float* box = reinterpret_cast<float*>(smem_base128(smem_raw));
  uint64_t* bar = reinterpret_cast<uint64_t*>(box + NF * ACOL_FS);
  if (timed_out_before(a.status)) return;
  if (!tma_layout_ok(box, bar, a.status)) return;
  int x0, y0, ax = 0, ay = 0;
  bool fast;
  const Geom* gp = &g0;
  const Coef<float>* cp = &c0;
  const float* emap = a.emap;
  size_t pitch;
  if constexpr (BATCH) {
    const BatchTile w = a.work[blockIdx.x];
    const BatchDesign& bd = a.designs[w.d];
    gp = &bd.g;
    cp = &bd.c;
    x0 = w.x0;
    y0 = w.y0;
    ax = bd.ax;
    ay = bd.ay;
    fast = w.interior != 0;
    emap += (size_t)w.d * 540;
    pitch = (size_t)a.pitch;
  } else {
    x0 = (blockIdx.x % a.ntx) * COL_W;
    y0 = (blockIdx.x / a.ntx) * ACOL_H;
    fast = x0 >= 2 && x0 + COL_W + 2 <= g0.nx && y0 >= 2 && y0 + ACOL_H + 2 <= g0.ny;
    pitch = (size_t)g0.nx;
  }
  const Geom g = *gp;  // register copies (see fwd_col2_kernel)
  const Coef<float> c = *cp;
  const int nx = g.nx, ny = g.ny;
  float* sem = reinterpret_cast<float*>(bar + 1);  // edge maps of the tile's lattice (edge tiles)
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
    fence_proxy_async();
    mbar_expect_tx(bar, NF * ACOL_BOX * 4);
    for (int f = 0; f < NF; ++f)
      tma_load_2d(box + f * ACOL_FS, &maps.m[f], ax + x0 - TMA_BXPAD, ay + y0 - 2, bar);
  }
  if (!fast)  // the batched form's per-design maps have no boundary objective terms
    for (int t = threadIdx.x; t < (BATCH ? 540 : kEdgeMapLen); t += COL_NT) sem[t] = __ldg(emap + t);
  __syncthreads();
  if (!mbar_wait(bar, 0)) {
    raise_status(a.status, 6);
    if (threadIdx.x == 0) mbar_wait(bar, 0);
    return;
  }
  const float* sa0 = box;
  const float* sa1 = box + ACOL_FS;
  const float* sa2 = box + 2 * ACOL_FS;
  const float* sa3 = box + 3 * ACOL_FS;
  const float* sa4 = box + 4 * ACOL_FS;
  const float* sa5 = box + 5 * ACOL_FS;
  const float* su1 = box + 6 * ACOL_FS;
  const float* sv1 = box + 7 * ACOL_FS;
  const float* su0 = box + FU0 * ACOL_FS;
  const float* sv0 = box + (FU0 + 1) * ACOL_FS;
  const float* sal = box + FAL * ACOL_FS;
  const float* sbi = box + FBI * ACOL_FS;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int i = x0 - 2 + lane;
  const int bx = lane + 2;
  const int r0 = y0 + warp * ACOL_R;
  const bool out_lane = lane >= 2 && lane < 2 + COL_W && i < nx;
  auto brow = [&](int y) { return (y - y0 + 2) * BW; };

  auto march = [&](auto edge_tag) {
    constexpr bool EDGE = decltype(edge_tag)::value;
    float X[9], Y[9], Z[9];  // gathered P + c.V of output rows p-1, p, p+1
#pragma unroll
    for (int k = 0; k < 9; ++k) X[k] = Y[k] = Z[k] = 0.f;
    float S0m = 0.f, S1m = 0.f, S2m = 0.f;  // strain of the level-t state, rows p-2 (m), p-1 (c), p (p)
    float S0c = 0.f, S1c = 0.f, S2c = 0.f;
    float gm_c = 0.f, sold_c = 0.f;  // gamma and sensitivity of output row p - 1
    for (int p = r0 - 1; p <= r0 + ACOL_R; ++p) {
      // gamma and the old sensitivity of output row p, written in the next iteration:
      // loaded a row ahead so that their latency overlaps a whole row
      float gm_n = 0.f, sold_n = 0.f;
      if (a.sens && out_lane && p >= r0 && p < r0 + ACOL_R && p < ny &&
          (!EDGE || (i > 0 && p > 0 && i < nx - 1 && p < ny - 1))) {
        const size_t gn = (size_t)(ay + p) * pitch + (size_t)(ax + i);
        gm_n = __ldg(a.gamma + gn);
        sold_n = a.sens[gn];
      }
      const int s2 = brow(p) + bx;
      float Pq[9];
      float S0p = 0.f, S1p = 0.f, S2p = 0.f;
      const bool live = !EDGE || (i >= 0 && i < nx && p >= 0 && p < ny);
      if (!live) {
#pragma unroll
        for (int k = 0; k < 9; ++k) Pq[k] = 0.f;
      } else {
        const float rt = sa0[s2], ux = sa1[s2], uy = sa2[s2];
        const float sxx = sa3[s2], sxy = sa4[s2], syy = sa5[s2];
        const float uu = su1[s2], vv = sv1[s2];
        float Dx, Dy;
        if (EDGE) {
          const int by = p - y0 + 2;
          Dx = adj_div2(dfdx<float, BW>(sa3, bx, by, i, nx), dfdy<float, BW>(sa4, bx, by, p, ny));
          Dy = adj_div2(dfdx<float, BW>(sa4, bx, by, i, nx), dfdy<float, BW>(sa5, bx, by, p, ny));
        } else {
          Dx = adj_div2(cdiff(sa3[s2 + 1], sa3[s2 - 1]), cdiff(sa4[s2 + BW], sa4[s2 - BW]));
          Dy = adj_div2(cdiff(sa4[s2 + 1], sa4[s2 - 1]), cdiff(sa5[s2 + BW], sa5[s2 - BW]));
        }
        adj_pv9(rt, ux, uy, sxx, sxy, syy, uu, vv, Dx, Dy, c.A, Pq);
        if (!EDGE || (i > 0 && p > 0 && i < nx - 1 && p < ny - 1)) {
          S0p = __fmul_rn(2.f, cdiff(su0[s2 + 1], su0[s2 - 1]));
          S1p = __fadd_rn(cdiff(su0[s2 + BW], su0[s2 - BW]), cdiff(sv0[s2 + 1], sv0[s2 - 1]));
          S2p = __fmul_rn(2.f, cdiff(sv0[s2 + BW], sv0[s2 - BW]));
        }
      }
      // output x gathers P + c_k.V at x + c_k: row p - c_y, column from the lane c_x away
      X[2] = Pq[2];
      X[5] = __shfl_down_sync(0xffffffffu, Pq[5], 1);
      X[6] = __shfl_up_sync(0xffffffffu, Pq[6], 1);
      Y[0] = Pq[0];
      Y[1] = __shfl_down_sync(0xffffffffu, Pq[1], 1);
      Y[3] = __shfl_up_sync(0xffffffffu, Pq[3], 1);
      Z[4] = Pq[4];
      Z[7] = __shfl_up_sync(0xffffffffu, Pq[7], 1);
      Z[8] = __shfl_down_sync(0xffffffffu, Pq[8], 1);
      // strain of row p - 1 from the neighbour lanes (J source of output row p - 1)
      const float S0l = __shfl_up_sync(0xffffffffu, S0c, 1), S0r = __shfl_down_sync(0xffffffffu, S0c, 1);
      const float S1l = __shfl_up_sync(0xffffffffu, S1c, 1), S1r = __shfl_down_sync(0xffffffffu, S1c, 1);
      const int q = p - 1;
      if (q >= r0 && q < r0 + ACOL_R && q < ny && out_lane) {
        const int sq = brow(q) + bx;
        const bool interior = !EDGE || (i > 0 && q > 0 && i < nx - 1 && q < ny - 1);
        const size_t gi = (size_t)(ay + q) * pitch + (size_t)(ax + i);
        const float gm = gm_c, sold = sold_c;
        float ft[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) ft[k] = X[k];
        float m[6];
        if (interior) {
          adj_moments6(ft, m);
          const float al = sal[sq];
          const float uu0 = su0[sq], vv0 = sv0[sq];
          const float ju = adj_jsrc(c.nu, __fsub_rn(__fadd_rn(__fsub_rn(S0l, S0r), S1m), S1p), al, uu0);
          const float jv = adj_jsrc(c.nu, __fsub_rn(__fadd_rn(__fsub_rn(S2m, S2p), S1l), S1r), al, vv0);
          const float inv = sbi[sq];
          m[1] = adj_brinkman(m[1], ju, 0.f, inv);
          m[2] = adj_brinkman(m[2], jv, 0.f, inv);
          if (a.sens) {
            float sacc = 0.f;
            if (a.sens_flow) sacc = __fadd_rn(sacc, sens_flow_term(c, gm, uu0, vv0, m[1], m[2]));
            a.sens[gi] = sold + sacc;
          }
        } else {
#pragma unroll
          for (int k = 0; k < 9; ++k) {
            const int gi = i + cxk(k), gj = q + cyk(k);
            if (gi < 0 || gi >= nx || gj < 0 || gj >= ny) ft[k] = 0.f;
          }
          const int ec = edge_class(g, i, q);
          const float* M = sem + ec * 60;
#pragma unroll
          for (int r = 0; r < 6; ++r) m[r] = adj_edge_row(M + r * 10, ft, 0.f);
          if constexpr (!BATCH) {  // the static pressure drop (steady single lattices only)
            const float jb = edge_objective_term(g, c, ec, q);
            if (jb != 0.f)
#pragma unroll
              for (int r = 0; r < 6; ++r) m[r] = __fmaf_rn(jb, sem[540 + ec * 6 + r], m[r]);
          }
        }
        (void)sq;
#pragma unroll
        for (int f = 0; f < 6; ++f) a.m0[f][gi] = m[f];
        if (!(m[1] * m[1] + m[2] * m[2] < 1e30f)) raise_status(a.status, 4);
      }
#pragma unroll
      for (int k = 0; k < 9; ++k) {
        X[k] = Y[k];
        Y[k] = Z[k];
        Z[k] = 0.f;
      }
      S0m = S0c, S1m = S1c, S2m = S2c;
      S0c = S0p, S1c = S1p, S2c = S2p;
      gm_c = gm_n;
      sold_c = sold_n;
    }
  };
  if (fast) march(std::false_type{});
  else march(std::true_type{});
}

}  // namespace lks
