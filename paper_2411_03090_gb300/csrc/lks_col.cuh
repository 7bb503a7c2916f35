// lks_col.cuh -- warp-column form of the FP32 forward step of one lattice (non-thermal).
//
// Each warp owns 32 adjacent lattice columns and marches down 16 output rows with
// the state of three rows held in registers.  A lane computes the nine pushed
// populations of its node (the per-node arithmetic of fwd_tma_kernel, term for
// term), hands the ones that cross a column to its neighbour lane by warp shuffle,
// and accumulates what its column receives per destination row; a row is complete
// once the row below it has been pushed.  The two outer lanes on each side only
// feed their neighbours, so a warp writes 28 columns.  Four warps stacked in y make
// a 28 x 64 tile, staged by one tensor copy of each field (box 36 x 68 from
// (x0 - 4, y0 - 2): the halo, with x on a 16-byte boundary).  There is no shared
// push array and no barrier inside a tile.  Tiles whose halo reaches the domain
// edge run the same march with the edge rules (one-sided derivatives, continuity,
// Zou-He edges, corners), reading neighbours from the staged box.
#pragma once
#include "lks_tma.cuh"

namespace lks {

constexpr int COL_W = 28;                       // output columns per warp (32 lanes, 2 halo lanes per side)
constexpr int COL_WARPS = 4;                    // warps per CTA, stacked in y
constexpr int COL_R = 16;                       // output rows per warp
constexpr int COL_H = COL_WARPS * COL_R;        // output rows per tile
constexpr int COL_BW = COL_W + 8, COL_BH = COL_H + 4, COL_BOX = COL_BW * COL_BH;
constexpr int COL_NT = 32 * COL_WARPS;
constexpr int COL_FS = (COL_BOX * 4 + 127) / 128 * 128 / 4;  // field stride: copies land on 128-byte boundaries

__host__ __device__ constexpr size_t col_smem_bytes() { return (size_t)4 * COL_FS * 4 + 128 + 8 + 8 * COL_WARPS; }

struct ColArgs {
  float* out[3];      // drho, u, v of the new level
  float* traj_u;      // optional trajectory copies of u, v
  float* traj_v;
  double* J_partial;  // per-tile accumulator of J_O(old state), or null
  int* status;
  float u_in;         // inlet amplitude of the new level
  int ntx, nty;       // tiles along x and y
  // Frame mode (fr_txb > 0): the launch covers only the tiles outside an interior
  // block [bx0, bx1) x [by0, by1) that fwd_col2_kernel computes: tile rows 0 and
  // >= fr_tyb in full, columns 0 and >= fr_txb of the rows between; nodes inside the
  // block are neither written nor counted in J.
  int fr_txb, fr_tyb;
  int bx0, bx1, by0, by1;
};

// Tile (tx, ty) of block b of a forward column launch (see ColArgs).
__device__ __forceinline__ void col_tile(const ColArgs& a, int b, int& tx, int& ty) {
  if (a.fr_txb <= 0) {
    tx = b % a.ntx;
    ty = b / a.ntx;
    return;
  }
  const int nr = 1 + a.nty - a.fr_tyb;  // full rows
  if (b < nr * a.ntx) {
    const int r = b / a.ntx;
    tx = b - r * a.ntx;
    ty = r == 0 ? 0 : a.fr_tyb + r - 1;
  } else {
    const int nc = 1 + a.ntx - a.fr_txb, b2 = b - nr * a.ntx, r = b2 / nc, ci = b2 - r * nc;
    ty = 1 + r;
    tx = ci == 0 ? 0 : a.fr_txb + ci - 1;
  }
}

__global__ void __launch_bounds__(COL_NT) fwd_col_kernel(const __grid_constant__ TmaMaps<4> maps,
                                                         const __grid_constant__ ColArgs a,
                                                         const __grid_constant__ Geom g,
                                                         const __grid_constant__ Coef<float> c) {
  extern __shared__ unsigned char smem_raw[];
  float* box = reinterpret_cast<float*>(smem_base128(smem_raw));  // [drho, u, v, 1/(1+alpha)][COL_FS]
  uint64_t* bar = reinterpret_cast<uint64_t*>(box + 4 * COL_FS);
  double* red = reinterpret_cast<double*>(bar + 1);
  if (timed_out_before(a.status)) return;
  if (!tma_layout_ok(box, bar, a.status)) return;
  const int nx = g.nx, ny = g.ny;
  int tx, ty;
  col_tile(a, (int)blockIdx.x, tx, ty);
  const int x0 = tx * COL_W, y0 = ty * COL_H;
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
    fence_proxy_async();
    mbar_expect_tx(bar, 4 * COL_BOX * 4);
    for (int f = 0; f < 4; ++f) tma_load_2d(box + f * COL_FS, &maps.m[f], x0 - TMA_BXPAD, y0 - 2, bar);
  }
  __syncthreads();
  if (!mbar_wait(bar, 0)) {
    raise_status(a.status, 6);
    if (threadIdx.x == 0) mbar_wait(bar, 0);
    return;
  }
  const float* sdr = box;
  const float* su = box + COL_FS;
  const float* sv = box + 2 * COL_FS;
  const float* sbi = box + 3 * COL_FS;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int i = x0 - 2 + lane;  // this lane's lattice column
  const int bx = lane + 2;      // its column in the box
  const int r0 = y0 + warp * COL_R;
  const bool out_lane = lane >= 2 && lane < 2 + COL_W && i < nx;
  const bool fast = a.fr_txb <= 0 && x0 >= 2 && x0 + COL_W + 2 <= nx && y0 >= 2 && y0 + COL_H + 2 <= ny;
  constexpr int BW = COL_BW;
  double jloc = 0.0;
  auto in_block = [&](int y) { return i >= a.bx0 && i < a.bx1 && y >= a.by0 && y < a.by1; };
  auto brow = [&](int y) { return (y - y0 + 2) * BW; };  // box offset of row y

  auto march = [&](auto edge_tag) {
    constexpr bool EDGE = decltype(edge_tag)::value;
    float X[9], Y[9], Z[9];  // received populations of destination rows p-1, p, p+1
#pragma unroll
    for (int k = 0; k < 9; ++k) X[k] = Y[k] = Z[k] = 0.f;
    // register ring (fast path): drho, u, v of rows p-1 (A), p (B), p+1 (C)
    float dA = 0.f, uA = 0.f, vA = 0.f, dB = 0.f, uB = 0.f, vB = 0.f, dC = 0.f, uC = 0.f, vC = 0.f;
    if (!EDGE) {
      const int o = brow(r0 - 2) + bx;
      dA = sdr[o], uA = su[o], vA = sv[o];
      dB = sdr[o + BW], uB = su[o + BW], vB = sv[o + BW];
      dC = sdr[o + 2 * BW], uC = su[o + 2 * BW], vC = sv[o + 2 * BW];
    }
    for (int p = r0 - 1; p <= r0 + COL_R; ++p) {
      float F[9];
      const int s2 = brow(p) + bx;
      bool has_obj = false, live = true;
      float uu = 0.f, vv = 0.f, dudx = 0.f, dudy = 0.f, dvdx = 0.f, dvdy = 0.f, dr = 0.f;
      float d_e = 0.f, d_w = 0.f, d_n = 0.f, d_s = 0.f, d_ne = 0.f, d_nw = 0.f, d_sw = 0.f, d_se = 0.f;
      if (!EDGE) {
        const float uL = __shfl_up_sync(0xffffffffu, uB, 1), uR = __shfl_down_sync(0xffffffffu, uB, 1);
        const float vL = __shfl_up_sync(0xffffffffu, vB, 1), vR = __shfl_down_sync(0xffffffffu, vB, 1);
        const float aL = __shfl_up_sync(0xffffffffu, dA, 1), aR = __shfl_down_sync(0xffffffffu, dA, 1);
        const float bL = __shfl_up_sync(0xffffffffu, dB, 1), bR = __shfl_down_sync(0xffffffffu, dB, 1);
        const float cL = __shfl_up_sync(0xffffffffu, dC, 1), cR = __shfl_down_sync(0xffffffffu, dC, 1);
        uu = uB;
        vv = vB;
        dudx = cdiff(uR, uL);
        dudy = cdiff(uC, uA);
        dvdx = cdiff(vR, vL);
        dvdy = cdiff(vC, vA);
        dr = dB;
        d_e = bR, d_w = bL, d_n = dC, d_s = dA, d_ne = cR, d_nw = cL, d_sw = aL, d_se = aR;
        has_obj = true;
      } else {
        live = i >= 0 && i < nx && p >= 0 && p < ny;
        if (!live) {
#pragma unroll
          for (int k = 0; k < 9; ++k) F[k] = 0.f;
        } else {
          const int by = p - y0 + 2;
          uu = su[s2];
          vv = sv[s2];
          dudx = dfdx<float, BW>(su, bx, by, i, nx);
          dudy = dfdy<float, BW>(su, bx, by, p, ny);
          dvdx = dfdx<float, BW>(sv, bx, by, i, nx);
          dvdy = dfdy<float, BW>(sv, bx, by, p, ny);
          const bool xe = (i == 0 || i == nx - 1), ye = (p == 0 || p == ny - 1);
          if (xe && ye) {
            dudx = 0.f;
            dvdy = 0.f;
          } else if (xe) {
            dudx = -dvdy;
          } else if (ye) {
            dvdy = -dudx;
          }
          dr = sdr[s2];
          d_e = sdr[s2 + 1], d_w = sdr[s2 - 1], d_n = sdr[s2 + BW], d_s = sdr[s2 - BW];
          d_ne = sdr[s2 + BW + 1], d_nw = sdr[s2 + BW - 1], d_sw = sdr[s2 - BW - 1], d_se = sdr[s2 - BW + 1];
          has_obj = i > 0 && p > 0 && i < nx - 1 && p < ny - 1;
        }
      }
      if (live) {
        const float dn[9] = {0.f, d_e, d_n, d_w, d_s, d_ne, d_nw, d_sw, d_se};
        push9(dr, dn, uu, vv, dudx, dudy, dvdx, dvdy, c.A, F);
        // objective of the old state at this warp's output nodes (unsteady accumulation)
        if (a.J_partial && has_obj && out_lane && p >= r0 && p < r0 + COL_R && p < ny && !in_block(p)) {
          jloc += (double)jo_flow<BW>(su, sv, s2, c.nu, sbi[s2], uu, vv);
        }
      }
      // hand the populations that cross a column to the neighbour lane
      {
        const float g1 = __shfl_up_sync(0xffffffffu, F[1], 1);
        const float g5 = __shfl_up_sync(0xffffffffu, F[5], 1);
        const float g8 = __shfl_up_sync(0xffffffffu, F[8], 1);
        const float g3 = __shfl_down_sync(0xffffffffu, F[3], 1);
        const float g6 = __shfl_down_sync(0xffffffffu, F[6], 1);
        const float g7 = __shfl_down_sync(0xffffffffu, F[7], 1);
        X[4] = F[4];  // c = (0, -1): destination row p - 1
        X[7] = g7;
        X[8] = g8;
        Y[0] = F[0];  // c_y = 0: destination row p
        Y[1] = g1;
        Y[3] = g3;
        Z[2] = F[2];  // c_y = +1: destination row p + 1
        Z[5] = g5;
        Z[6] = g6;
      }
      // row p - 1 is complete
      const int q = p - 1;
      if (q >= r0 && q < r0 + COL_R && q < ny && out_lane && !in_block(q)) {
        const int sq = brow(q) + bx;
        const float drx = EDGE ? sdr[sq] : dA;
        float drn, un, vn;
        int nxo = 0, nyo = 0;
        const int cls = EDGE ? node_class(g, i, q, nxo, nyo) : C_INTERIOR;
        const float* fk = X;
        if (cls == C_INTERIOR) {
          gather9(fk, drx, sbi[sq], drn, un, vn);
        } else {
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
            const int jn = (q == 0) ? 1 : ny - 2;
            drn = sdr[brow(jn) + bx];
            un = vn = 0.f;
          } else if (cls == C_VELOCITY) {
            un = 0.f;
            if (i == 0 && q >= g.in_y0 && q <= g.in_y1) {
              const double H = (double)(g.in_y1 - g.in_y0), y = (double)(q - g.in_y0);
              un = a.u_in * (float)(4.0 * y * (H - y) / (H * H));
            }
            vn = 0.f;
            drn = __fadd_rn(drx, __fsub_rn(__fmaf_rn(2.f, sp, s0), __fmaf_rn(vn, (float)nyo, __fmul_rn(un, (float)nxo))));
          } else {
            drn = c.drho_out;
            const float unorm = __fadd_rn(__fmaf_rn(2.f, sp, s0), __fsub_rn(drx, c.drho_out));
            un = __fmul_rn(unorm, (float)nxo);
            vn = __fmul_rn(unorm, (float)nyo);
          }
        }
        const size_t o = (size_t)q * nx + i;
        a.out[0][o] = drn;
        a.out[1][o] = un;
        a.out[2][o] = vn;
        if (a.traj_u) {
          a.traj_u[o] = un;
          a.traj_v[o] = vn;
        }
        if (bad_velocity(un, vn)) raise_status(a.status, 4);
      }
      // rotate the rows
#pragma unroll
      for (int k = 0; k < 9; ++k) {
        X[k] = Y[k];
        Y[k] = Z[k];
        Z[k] = 0.f;
      }
      if (!EDGE) {
        dA = dB, uA = uB, vA = vB;
        dB = dC, uB = uC, vB = vC;
        if (p + 2 <= r0 + COL_R + 1) {
          const int o = brow(p + 2) + bx;
          dC = sdr[o], uC = su[o], vC = sv[o];
        }
      }
    }
  };
  // Interior tiles: the same march unrolled by three rows, so that the three-row
  // register rings rotate by renaming; each row's neighbour values are shuffled
  // once, when the row is loaded.
  struct Row {
    float d, u, v, dl, dr;  // drho, u, v of the lane's column and drho of the columns left and right
  };
  auto load_row = [&](Row& R, int y) {
    const int o = brow(y) + bx;
    R.d = sdr[o];
    R.u = su[o];
    R.v = sv[o];
    R.dl = __shfl_up_sync(0xffffffffu, R.d, 1);
    R.dr = __shfl_down_sync(0xffffffffu, R.d, 1);
  };
  // One row p of the march: A, B, C hold rows p-1, p, p+1; X, Y, Z collect the
  // populations of destination rows p-1, p, p+1.  Row p+2 is loaded into A.
  auto step = [&](int p, Row& A, Row& B, Row& C, float* X, float* Y, float* Z) {
    const float uL = __shfl_up_sync(0xffffffffu, B.u, 1), uR = __shfl_down_sync(0xffffffffu, B.u, 1);
    const float vL = __shfl_up_sync(0xffffffffu, B.v, 1), vR = __shfl_down_sync(0xffffffffu, B.v, 1);
    const float uu = B.u, vv = B.v;
    const float dr = B.d;
    float F[9];
    {
      const float dn[9] = {0.f, B.dr, C.d, B.dl, A.d, C.dr, C.dl, A.dl, A.dr};
      push9(dr, dn, uu, vv, cdiff(uR, uL), cdiff(C.u, A.u), cdiff(vR, vL), cdiff(C.v, A.v), c.A, F);
    }
    const int s2 = brow(p) + bx;
    if (a.J_partial && out_lane && p >= r0 && p < r0 + COL_R) {
      jloc += (double)jo_flow<BW>(su, sv, s2, c.nu, sbi[s2], uu, vv);
    }
    X[4] = F[4];
    X[7] = __shfl_down_sync(0xffffffffu, F[7], 1);
    X[8] = __shfl_up_sync(0xffffffffu, F[8], 1);
    Y[0] = F[0];
    Y[1] = __shfl_up_sync(0xffffffffu, F[1], 1);
    Y[3] = __shfl_down_sync(0xffffffffu, F[3], 1);
    Z[2] = F[2];
    Z[5] = __shfl_up_sync(0xffffffffu, F[5], 1);
    Z[6] = __shfl_down_sync(0xffffffffu, F[6], 1);
    const int q = p - 1;
    if (q >= r0 && out_lane) {  // row p - 1 is complete
      float drn, un, vn;
      gather9(X, A.d, sbi[s2 - BW], drn, un, vn);
      const size_t o = (size_t)q * nx + i;
      a.out[0][o] = drn;
      a.out[1][o] = un;
      a.out[2][o] = vn;
      if (a.traj_u) {
        a.traj_u[o] = un;
        a.traj_v[o] = vn;
      }
      if (bad_velocity(un, vn)) raise_status(a.status, 4);
    }
    if (p + 2 <= r0 + COL_R + 1) load_row(A, p + 2);
  };
  if (fast) {
    Row R0, R1, R2;
    float X0[9], X1[9], X2[9];
    load_row(R0, r0 - 2);
    load_row(R1, r0 - 1);
    load_row(R2, r0);
    static_assert((COL_R + 2) % 3 == 0, "the unrolled march covers COL_R + 2 rows in threes");
#pragma unroll 1
    for (int p = r0 - 1; p <= r0 + COL_R; p += 3) {
      step(p, R0, R1, R2, X0, X1, X2);
      step(p + 1, R1, R2, R0, X1, X2, X0);
      step(p + 2, R2, R0, R1, X2, X0, X1);
    }
  } else {
    march(std::true_type{});
  }
  if (a.J_partial) {
    const double s = block_sum<COL_NT>(jloc, red);
    if (threadIdx.x == 0) a.J_partial[blockIdx.x] += s;
  }
}


// ---------------------------------------------------------------------------------
// Warp-column forward with two columns per lane (interior block of the lattice)
// ---------------------------------------------------------------------------------
// Lane l owns the columns x0 - 2 + 2l and x0 - 1 + 2l and marches down R rows like
// fwd_col_kernel.  Neighbours inside the lane pair need no shuffle; a row costs two
// shuffles per field crossing the lane boundary and six for the populations moving
// to the neighbour lanes, and its loads and stores are 8-byte vectors.  Lanes 1..30
// write, so a warp covers 60 columns.  Every tile lies at least two nodes inside the
// lattice: the tile grid starts at (xa, ya) and the host sizes it so; the frame
// around it runs fwd_col_kernel.  The per-node arithmetic is push9 / gather9, as in
// the other FP32 staged kernels.
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
constexpr int C2_R = 16;

struct Col2Args {
  float* out[3];      // drho, u, v of the new level
  float* traj_u;      // optional trajectory copies of u, v
  float* traj_v;
  double* J_partial;  // per-tile accumulator of J_O(old state), or null
  int* status;
  float u_in;         // unused: no inlet node lies in the block
  int ntx;            // tiles along x
  int xa, ya;         // lattice origin of the tile grid
};

template <int R>
__global__ void __launch_bounds__(COL_NT) fwd_col2_kernel(const __grid_constant__ TmaMaps<4> maps,
                                                          const __grid_constant__ Col2Args a,
                                                          const __grid_constant__ Geom g,
                                                          const __grid_constant__ Coef<float> c) {
  using G2 = Col2Geo<R>;
  constexpr int BW = C2_BW, FS = G2::FS;
  extern __shared__ unsigned char smem_raw[];
  float* box = reinterpret_cast<float*>(smem_base128(smem_raw));  // [drho, u, v, 1/(1+alpha)][FS]
  uint64_t* bar = reinterpret_cast<uint64_t*>(box + 4 * FS);
  double* red = reinterpret_cast<double*>(bar + 1);
  if (timed_out_before(a.status)) return;
  if (!tma_layout_ok(box, bar, a.status)) return;
  const int nx = g.nx;
  const int x0 = a.xa + (int)(blockIdx.x % a.ntx) * C2_W, y0 = a.ya + (int)(blockIdx.x / a.ntx) * G2::H;
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
  const float* sdr = box;
  const float* su = box + FS;
  const float* sv = box + 2 * FS;
  const float* sbi = box + 3 * FS;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int i0 = x0 - 2 + 2 * lane;            // the lane's first lattice column
  const int bx = TMA_BXPAD - 2 + 2 * lane;     // its column in the box (even: 8-byte aligned)
  const int r0 = y0 + warp * R;
  const bool out_lane = lane >= 1 && lane <= 30;
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
  // Destination row of the march: the nine populations arriving at each column.
  struct Dst {
    float a[9], b[9];
  };
  // Row p: A, B, C hold rows p-1, p, p+1; X, Y, Z collect destination rows p-1, p,
  // p+1.  Row p-1 is complete afterwards and is written; row p+2 is loaded into A.
  auto step = [&](int p, Row& A, Row& B, Row& C, Dst& X, Dst& Y, Dst& Z) {
    const float uL = __shfl_up_sync(0xffffffffu, B.u.y, 1), uR = __shfl_down_sync(0xffffffffu, B.u.x, 1);
    const float vL = __shfl_up_sync(0xffffffffu, B.v.y, 1), vR = __shfl_down_sync(0xffffffffu, B.v.x, 1);
    float F0[9], F1[9];
    {
      const float dn[9] = {0.f, B.d.y, C.d.x, B.dl, A.d.x, C.d.y, C.dl, A.dl, A.d.y};
      push9(B.d.x, dn, B.u.x, B.v.x, cdiff(B.u.y, uL), cdiff(C.u.x, A.u.x), cdiff(B.v.y, vL), cdiff(C.v.x, A.v.x),
            c.A, F0);
    }
    {
      const float dn[9] = {0.f, B.dr, C.d.y, B.d.x, A.d.y, C.dr, C.d.x, A.d.x, A.dr};
      push9(B.d.y, dn, B.u.y, B.v.y, cdiff(uR, B.u.x), cdiff(C.u.y, A.u.y), cdiff(vR, B.v.x), cdiff(C.v.y, A.v.y),
            c.A, F1);
    }
    if (a.J_partial && out_lane && p >= r0 && p < r0 + R) {
      const int s2 = brow(p) + bx;
      const float2 inv = *reinterpret_cast<const float2*>(sbi + s2);
      jloc += (double)jo_flow<BW>(su, sv, s2, c.nu, inv.x, B.u.x, B.v.x);
      jloc += (double)jo_flow<BW>(su, sv, s2 + 1, c.nu, inv.y, B.u.y, B.v.y);
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
    if (q >= r0 && out_lane) {
      const float2 inv = *reinterpret_cast<const float2*>(sbi + brow(q) + bx);
      float2 dn, un, vn;
      gather9(X.a, A.d.x, inv.x, dn.x, un.x, vn.x);
      gather9(X.b, A.d.y, inv.y, dn.y, un.y, vn.y);
      const size_t o = (size_t)q * nx + i0;
      *reinterpret_cast<float2*>(a.out[0] + o) = dn;
      *reinterpret_cast<float2*>(a.out[1] + o) = un;
      *reinterpret_cast<float2*>(a.out[2] + o) = vn;
      if (a.traj_u) {
        *reinterpret_cast<float2*>(a.traj_u + o) = un;
        *reinterpret_cast<float2*>(a.traj_v + o) = vn;
      }
      bad |= bad_velocity(un.x, vn.x) | bad_velocity(un.y, vn.y);
    }
    if (p + 2 <= r0 + R + 1) load_row(A, p + 2);
  };
  Row R0, R1, R2;
  Dst X0, X1, X2;
  load_row(R0, r0 - 2);
  load_row(R1, r0 - 1);
  load_row(R2, r0);
#pragma unroll 1
  for (int p = r0 - 1; p <= r0 + R; p += 3) {
    step(p, R0, R1, R2, X0, X1, X2);
    step(p + 1, R1, R2, R0, X1, X2, X0);
    step(p + 2, R2, R0, R1, X2, X0, X1);
  }
  if (bad) raise_status(a.status, 4);
  if (a.J_partial) {
    const double s = block_sum<COL_NT>(jloc, red);
    if (threadIdx.x == 0) a.J_partial[blockIdx.x] += s;
  }
}


// ---------------------------------------------------------------------------------
// Warp-column ALKS step (FP32, non-thermal, one lattice)
// ---------------------------------------------------------------------------------
// The same march for the adjoint: a lane computes P + c_k . V (Eq. afeq) of its node
// for the nine links and the strain of the level-t state, hands the values a
// neighbouring column gathers to it by shuffle, and completes the moments of a row
// once the row below has been computed.  Tiles of 28 x 32 outputs (four warps of
// eight rows); the per-node arithmetic is that of adj_tma_kernel, term for term.
constexpr int ACOL_R = 8;
constexpr int ACOL_H = COL_WARPS * ACOL_R;
constexpr int ACOL_BH = ACOL_H + 4, ACOL_BOX = COL_BW * ACOL_BH;
constexpr int ACOL_FS = (ACOL_BOX * 4 + 127) / 128 * 128 / 4;

__host__ __device__ constexpr int acol_nf(bool same) { return same ? 10 : 12; }
__host__ __device__ constexpr size_t acol_smem_bytes(bool same) {
  return (size_t)acol_nf(same) * ACOL_FS * 4 + 128 + 8;
}

struct AdjColArgs {
  float* m0[6];       // adjoint moments at level t
  const float* gamma;
  const float* emap;  // 9 classes x 6 x 10
  float* sens;        // optional sensitivity accumulator
  int sens_flow;
  int* status;
  int ntx;
};

// Staged fields: rho~, u~x, u~y, s~xx, s~xy, s~yy, u1, v1, [u0, v0], alpha, 1/(1+alpha).
template <bool SAME>
__global__ void __launch_bounds__(COL_NT) adj_col_kernel(const __grid_constant__ TmaMaps<acol_nf(SAME)> maps,
                                                         const __grid_constant__ AdjColArgs a,
                                                         const __grid_constant__ Geom g,
                                                         const __grid_constant__ Coef<float> c) {
  constexpr int NF = acol_nf(SAME);
  constexpr int FU0 = SAME ? 6 : 8, FAL = SAME ? 8 : 10, FBI = FAL + 1;
  constexpr int BW = COL_BW;
  extern __shared__ unsigned char smem_raw[];
  float* box = reinterpret_cast<float*>(smem_base128(smem_raw));
  uint64_t* bar = reinterpret_cast<uint64_t*>(box + NF * ACOL_FS);
  if (timed_out_before(a.status)) return;
  if (!tma_layout_ok(box, bar, a.status)) return;
  const int nx = g.nx, ny = g.ny;
  const int x0 = (blockIdx.x % a.ntx) * COL_W, y0 = (blockIdx.x / a.ntx) * ACOL_H;
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
    fence_proxy_async();
    mbar_expect_tx(bar, NF * ACOL_BOX * 4);
    for (int f = 0; f < NF; ++f) tma_load_2d(box + f * ACOL_FS, &maps.m[f], x0 - TMA_BXPAD, y0 - 2, bar);
  }
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
  const bool fast = x0 >= 2 && x0 + COL_W + 2 <= nx && y0 >= 2 && y0 + ACOL_H + 2 <= ny;
  auto brow = [&](int y) { return (y - y0 + 2) * BW; };

  auto march = [&](auto edge_tag) {
    constexpr bool EDGE = decltype(edge_tag)::value;
    float X[9], Y[9], Z[9];  // gathered P + c.V of output rows p-1, p, p+1
#pragma unroll
    for (int k = 0; k < 9; ++k) X[k] = Y[k] = Z[k] = 0.f;
    float S0m = 0.f, S1m = 0.f, S2m = 0.f;  // strain of the level-t state, rows p-2 (m), p-1 (c), p (p)
    float S0c = 0.f, S1c = 0.f, S2c = 0.f;
    for (int p = r0 - 1; p <= r0 + ACOL_R; ++p) {
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
            const size_t gi = (size_t)q * nx + i;
            const float gm = __ldg(a.gamma + gi);
            float sacc = 0.f;
            if (a.sens_flow) sacc = __fadd_rn(sacc, sens_flow_term(c, gm, uu0, vv0, m[1], m[2]));
            a.sens[gi] += sacc;
          }
        } else {
#pragma unroll
          for (int k = 0; k < 9; ++k) {
            const int gi = i + cxk(k), gj = q + cyk(k);
            if (gi < 0 || gi >= nx || gj < 0 || gj >= ny) ft[k] = 0.f;
          }
          const float* M = a.emap + edge_class(g, i, q) * 60;
#pragma unroll
          for (int r = 0; r < 6; ++r) m[r] = adj_edge_row(M + r * 10, ft, 0.f);
        }
        (void)sq;
        const size_t o = (size_t)q * nx + i;
#pragma unroll
        for (int f = 0; f < 6; ++f) a.m0[f][o] = m[f];
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
    }
  };
  if (fast) march(std::false_type{});
  else march(std::true_type{});
}

}  // namespace lks
