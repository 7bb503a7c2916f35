// lks_tma.cuh -- TMA-staged, software-pipelined forms of the one-launch-per-step LKS
// and ALKS kernels (FP32) for lattices too large to stay resident.
//
// Each CTA is persistent over a static list of tiles.  Thread 0 issues 2-D tensor
// copies (cp.async.bulk.tensor) of every field the step reads, for the tile's box
// with a two-node halo, into one of two shared-memory stages; an mbarrier with a
// transaction count signals arrival.  While the CTA computes tile k from one stage,
// the copies of tile k+1 fill the other.  Out-of-lattice parts of a box arrive as
// zeros (tensor-map fill), so no thread computes a load address.  The material
// fields 1/(1 + alpha_gamma), alpha_gamma and B_gamma are computed once per march
// (material_kernel) and staged like the state, so the step kernels read no
// per-node global memory and divide nothing.
//
// Tiles whose two-node halo stays clear of the domain edge take a path without
// any edge test; edge tiles take the general path with the edge rules.
//
// TMA alignment: the box starts at x0 - 4 (a multiple of four floats, 16 bytes) and
// is TX + 8 floats wide; rows are nx floats apart, so the lattice needs nx % 4 == 0
// (the host falls back to the plain kernels otherwise).  Shared stages are
// 128-byte aligned (checked before the first copy).  Waits on an mbarrier are
// bounded; on timeout the kernel records LKS_ERR_TIMEOUT, waits (bounded) for its
// own copies and returns.
//
// The arithmetic per node is that of fwd_step_kernel / adj_step_kernel, in push
// form (each halo-1 node first writes the nine values it streams; an output node
// sums nine shared-memory values).
#pragma once
#include <cuda.h>

#include <type_traits>

#include "lks_kernels.cuh"

namespace lks {

constexpr int TMA_BXPAD = 4;  // left pad of a box (floats), keeps x aligned to 16 B

template <int NF>
struct TmaMaps {
  CUtensorMap m[NF];
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// A launch that follows a timed-out wait returns at once (status word already 6).
__device__ __forceinline__ bool timed_out_before(const int* status) {
  return status && *reinterpret_cast<const volatile int*>(status) == 6;
}
// Dynamic shared memory rounded up to 128 bytes (tensor copies need a 128-byte
// aligned shared destination); the kernels declare no static shared memory.  The
// offset is added to the shared array itself, not through an integer round trip,
// so that the compiler keeps every access derived from it in the shared space.
__device__ __forceinline__ unsigned char* smem_base128(unsigned char* raw) {
  return raw + ((128u - (smem_u32(raw) & 127u)) & 127u);
}
// Self-check before any copy: the stages 128-byte and the mbarriers 8-byte aligned.
__device__ __forceinline__ bool tma_layout_ok(const void* stage, const void* bar, int* status) {
  const bool ok = (smem_u32(stage) & 127u) == 0 && (smem_u32(bar) & 7u) == 0;
  if (!ok && threadIdx.x == 0) raise_status(status, 3);
  return ok;
}
// Bounded wait for an mbarrier phase.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  for (long long it = 0; it < (1ll << 20); ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if (it > 16) __nanosleep(20);
  }
  return false;
}
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void tma_store_2d(const CUtensorMap* map, int x, int y, const void* src) {
  asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"(
                   reinterpret_cast<uint64_t>(map)),
               "r"(x), "r"(y), "r"(smem_u32(src))
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read0() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait0() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }


// ---------------------------------------------------------------------------------
// Per-node arithmetic of the FP32 staged kernels, written with explicit rounding
// (every product and sum named, no contraction left to the compiler), so that the
// per-tile, batched and warp-column kernels give bit-identical results.
// ---------------------------------------------------------------------------------
// Central difference (f[+1] - f[-1]) / 2.
__device__ __forceinline__ float cdiff(float fp, float fm) { return __fmul_rn(__fsub_rn(fp, fm), 0.5f); }

// Local objective of one interior node (Eq. obj): nu/2 S:S + alpha |u|^2, with the
// strain S_ab = d_b u_a + d_a u_b from central differences; s2 indexes the node in
// staged u (su) and v (sv) arrays of row length BW, inv is 1 / (1 + alpha).
template <int BW>
__device__ __forceinline__ float jo_flow(const float* su, const float* sv, int s2, float nu, float inv, float uu,
                                         float vv) {
  const float Sxx = __fmul_rn(2.f, cdiff(su[s2 + 1], su[s2 - 1]));
  const float Syy = __fmul_rn(2.f, cdiff(sv[s2 + BW], sv[s2 - BW]));
  const float Sxy = __fadd_rn(cdiff(su[s2 + BW], su[s2 - BW]), cdiff(sv[s2 + 1], sv[s2 - 1]));
  const float SS = __fmaf_rn(Syy, Syy, __fmaf_rn(__fmul_rn(2.f, Sxy), Sxy, __fmul_rn(Sxx, Sxx)));
  const float al = __fsub_rn(__fdiv_rn(1.f, inv), 1.f);
  return __fmaf_rn(al, __fmaf_rn(vv, vv, __fmul_rn(uu, uu)), __fmul_rn(__fmul_rn(0.5f, nu), SS));
}

// The nine pushed populations of one node (Eq. feq2, increment form): F_k is sent
// to x + c_k and carries w_k [(drho(x) - drho(x + c_k)) + e0 + c_k.b + c_k c_k : Q]
// with e0 = -3/2 |u|^2, b = 3u, Q_ab = 9/2 u_a u_b + A (d_b u_a + d_a u_b).
// d[k] = drho(x + c_k) for k = 1..8 (d[0] unused).  Evaluated as
// F_k = G_k - w_k d[k] with G_k = w_k (drho(x) + e0 + c_k c_k : Q) + w_k c_k.b, the
// partial sums shared between the links.
__device__ __forceinline__ void push9(float dr, const float* d, float uu, float vv, float dudx, float dudy,
                                      float dvdx, float dvdy, float A, float* F) {
  constexpr float w1 = 1.f / 9.f, w5 = 1.f / 36.f;
  const float uu2 = __fmul_rn(uu, uu), vv2 = __fmul_rn(vv, vv);
  const float e0 = __fmul_rn(-1.5f, __fadd_rn(uu2, vv2));
  const float A2 = __fmul_rn(2.f, A);
  const float qxx = __fmaf_rn(4.5f, uu2, __fmul_rn(A2, dudx));
  const float qyy = __fmaf_rn(4.5f, vv2, __fmul_rn(A2, dvdy));
  const float qxy = __fmaf_rn(__fmul_rn(9.f, uu), vv, __fmul_rn(A2, __fadd_rn(dudy, dvdx)));
  const float p0 = __fadd_rn(dr, e0);
  const float px = __fadd_rn(p0, qxx), py = __fadd_rn(p0, qyy);
  const float pd = __fadd_rn(px, qyy);  // drho + e0 + Q_xx + Q_yy
  const float q1 = __fadd_rn(pd, qxy), q2 = __fsub_rn(pd, qxy);
  const float wbx = __fmul_rn(1.f / 3.f, uu), wby = __fmul_rn(1.f / 3.f, vv);  // w1 b_x, w1 b_y
  const float wsp = __fmul_rn(1.f / 12.f, __fadd_rn(uu, vv));                   // w5 (b_x + b_y)
  const float wsm = __fmul_rn(1.f / 12.f, __fsub_rn(uu, vv));                   // w5 (b_x - b_y)
  F[0] = __fmul_rn(e0, 4.f / 9.f);
  F[1] = __fmaf_rn(-w1, d[1], __fmaf_rn(w1, px, wbx));
  F[3] = __fmaf_rn(-w1, d[3], __fmaf_rn(w1, px, -wbx));
  F[2] = __fmaf_rn(-w1, d[2], __fmaf_rn(w1, py, wby));
  F[4] = __fmaf_rn(-w1, d[4], __fmaf_rn(w1, py, -wby));
  F[5] = __fmaf_rn(-w5, d[5], __fmaf_rn(w5, q1, wsp));
  F[7] = __fmaf_rn(-w5, d[7], __fmaf_rn(w5, q1, -wsp));
  F[6] = __fmaf_rn(-w5, d[6], __fmaf_rn(w5, q2, -wsm));
  F[8] = __fmaf_rn(-w5, d[8], __fmaf_rn(w5, q2, wsm));
}

// The thermal pushed populations of one node (Eq. geq2, increment form): G_k is sent
// to x + c_k and carries w_k [(T(x) - T(x + c_k)) + c_k . (3 T u + B grad T)];
// t[k] = T(x + c_k) for k = 1..8 (G_0 = 0).
__device__ __forceinline__ void gpush9(float TT, const float* t, float uu, float vv, float dTx, float dTy,
                                       float Bn, float* G) {
  const float T3 = __fmul_rn(3.f, TT);
  const float qx = __fmaf_rn(T3, uu, __fmul_rn(Bn, dTx));
  const float qy = __fmaf_rn(T3, vv, __fmul_rn(Bn, dTy));
  G[0] = 0.f;
  G[1] = __fmul_rn(__fadd_rn(__fsub_rn(TT, t[1]), qx), 1.f / 9.f);
  G[3] = __fmul_rn(__fsub_rn(__fsub_rn(TT, t[3]), qx), 1.f / 9.f);
  G[2] = __fmul_rn(__fadd_rn(__fsub_rn(TT, t[2]), qy), 1.f / 9.f);
  G[4] = __fmul_rn(__fsub_rn(__fsub_rn(TT, t[4]), qy), 1.f / 9.f);
  G[5] = __fmul_rn(__fadd_rn(__fadd_rn(__fsub_rn(TT, t[5]), qx), qy), 1.f / 36.f);
  G[6] = __fmul_rn(__fadd_rn(__fsub_rn(__fsub_rn(TT, t[6]), qx), qy), 1.f / 36.f);
  G[7] = __fmul_rn(__fsub_rn(__fsub_rn(__fsub_rn(TT, t[7]), qx), qy), 1.f / 36.f);
  G[8] = __fmul_rn(__fsub_rn(__fadd_rn(__fsub_rn(TT, t[8]), qx), qy), 1.f / 36.f);
}
// Interior thermal gather: T(x) + sum over k = 1..8 of G_k(x - c_k).
__device__ __forceinline__ float tgather8(float TT, const float* gk) {
  float gs = gk[1];
#pragma unroll
  for (int k = 2; k < 9; ++k) gs = __fadd_rn(gs, gk[k]);
  return __fadd_rn(TT, gs);
}
// Heat-flux edge (Sec. 2.4 edge rule): (T + g0 + 2 gp + q_w) / (1 + u_n), with g0 / gp
// the known tangential / inward populations and u_n the new normal velocity.
__device__ __forceinline__ float tflux_edge(float TT, float g0, float gp, float qw, float un, float vn, int nxo,
                                            int nyo) {
  const float num = __fadd_rn(__fadd_rn(__fadd_rn(TT, g0), __fmul_rn(2.f, gp)), qw);
  const float den = __fadd_rn(__fadd_rn(1.f, __fmul_rn(un, (float)nxo)), __fmul_rn(vn, (float)nyo));
  return __fdiv_rn(num, den);
}

// Interior gather of one node: drho, and u, v before / after the implicit Brinkman
// division (fk[k] = F_k(x - c_k)).
__device__ __forceinline__ void gather9(const float* fk, float drx, float inv, float& drn, float& un, float& vn) {
  drn = __fadd_rn(drx, __fadd_rn(__fadd_rn(__fadd_rn(__fadd_rn(fk[0], fk[1]), __fadd_rn(fk[2], fk[3])),
                                           __fadd_rn(__fadd_rn(fk[4], fk[5]), __fadd_rn(fk[6], fk[7]))),
                                 fk[8]));
  const float a57 = __fsub_rn(fk[5], fk[7]), b86 = __fsub_rn(fk[8], fk[6]);
  un = __fmul_rn(__fadd_rn(__fadd_rn(__fsub_rn(fk[1], fk[3]), a57), b86), inv);
  vn = __fmul_rn(__fsub_rn(__fadd_rn(__fsub_rn(fk[2], fk[4]), a57), b86), inv);
}

// Adjoint equilibrium coefficients of one node (Eq. afeq): Pq[k] = P + c_k . V with
// P = rho~, V_a = 3 (u~_a + 3 s~_ab u_b - rho~ u_a) - A D_a.
__device__ __forceinline__ void adj_pv9(float rt, float ux, float uy, float sxx, float sxy, float syy, float uu,
                                        float vv, float Dx, float Dy, float A, float* Pq) {
  const float tx = __fsub_rn(__fmaf_rn(3.f, __fmaf_rn(sxy, vv, __fmul_rn(sxx, uu)), ux), __fmul_rn(rt, uu));
  const float ty = __fsub_rn(__fmaf_rn(3.f, __fmaf_rn(syy, vv, __fmul_rn(sxy, uu)), uy), __fmul_rn(rt, vv));
  const float Vx = __fsub_rn(__fmul_rn(3.f, tx), __fmul_rn(A, Dx));
  const float Vy = __fsub_rn(__fmul_rn(3.f, ty), __fmul_rn(A, Dy));
  const float rp = __fadd_rn(rt, Vx), rm = __fsub_rn(rt, Vx);
  Pq[0] = rt;
  Pq[1] = rp;
  Pq[3] = rm;
  Pq[2] = __fadd_rn(rt, Vy);
  Pq[4] = __fsub_rn(rt, Vy);
  Pq[5] = __fadd_rn(rp, Vy);
  Pq[6] = __fadd_rn(rm, Vy);
  Pq[7] = __fsub_rn(rm, Vy);
  Pq[8] = __fsub_rn(rp, Vy);
}
// D_x = 2 (d_x s~xx + d_y s~xy), D_y = 2 (d_x s~xy + d_y s~yy) from the four derivatives.
__device__ __forceinline__ float adj_div2(float d1, float d2) { return __fmul_rn(2.f, __fadd_rn(d1, d2)); }

// Interior adjoint moments (rho~, u~*, s~) of the gathered f~ (ft[k] = P + c_k.V at x + c_k).
__device__ __forceinline__ void adj_moments6(const float* ft, float* m) {
  const float w0 = 4.f / 9.f, w1 = 1.f / 9.f, w5 = 1.f / 36.f;
  const float ax = __fadd_rn(ft[1], ft[3]), ay = __fadd_rn(ft[2], ft[4]);
  const float dg = __fadd_rn(__fadd_rn(__fadd_rn(ft[5], ft[6]), ft[7]), ft[8]);
  m[0] = __fmaf_rn(w5, dg, __fmaf_rn(w1, __fadd_rn(ax, ay), __fmul_rn(w0, ft[0])));
  m[1] = __fmaf_rn(w5, __fadd_rn(__fsub_rn(__fsub_rn(ft[5], ft[6]), ft[7]), ft[8]), __fmul_rn(w1, __fsub_rn(ft[1], ft[3])));
  m[2] = __fmaf_rn(w5, __fsub_rn(__fsub_rn(__fadd_rn(ft[5], ft[6]), ft[7]), ft[8]), __fmul_rn(w1, __fsub_rn(ft[2], ft[4])));
  m[3] = __fmaf_rn(w5, dg, __fmul_rn(w1, ax));
  m[4] = __fmul_rn(w5, __fsub_rn(__fadd_rn(__fsub_rn(ft[5], ft[6]), ft[7]), ft[8]));
  m[5] = __fmaf_rn(w5, dg, __fmul_rn(w1, ay));
}
// Objective source of one velocity component: nu (sum of strain differences) + 2 alpha u.
__device__ __forceinline__ float adj_jsrc(float nu, float diff, float al, float u0) {
  return __fmaf_rn(__fmul_rn(2.f, al), u0, __fmul_rn(nu, diff));
}
// Implicit adjoint Brinkman: (m - j/3 + coupling) / (1 + alpha).
__device__ __forceinline__ float adj_brinkman(float m, float j, float cp, float inv) {
  return __fmul_rn(__fadd_rn(__fsub_rn(m, __fmul_rn(j, 1.f / 3.f)), cp), inv);
}
// Edge-node moment r from a 6 x 10 map row and the gathered f~ (unknown entries zero).
__device__ __forceinline__ float adj_edge_row(const float* Mr, const float* ft, float kT) {
  float acc = 0.f;
#pragma unroll
  for (int k = 0; k < 9; ++k) acc = __fmaf_rn(Mr[k], ft[k], acc);
  return __fmaf_rn(Mr[9], kT, acc);
}
// Flow sensitivity of one level: alpha' |u|^2 + 3 alpha' u.u~.
__device__ __forceinline__ float sens_flow_term(const Coef<float>& c, float gm, float uu0, float vv0, float m1,
                                                float m2) {
  const float dd = __fadd_rn(c.q_alpha, gm);
  const float da = __fdividef(-c.alpha_bar * c.q_alpha * (1.f + c.q_alpha), __fmul_rn(dd, dd));
  const float uuu = __fmaf_rn(vv0, vv0, __fmul_rn(uu0, uu0));
  const float uut = __fmaf_rn(vv0, m2, __fmul_rn(uu0, m1));
  return __fmaf_rn(__fmul_rn(3.f, da), uut, __fmul_rn(da, uuu));
}

// Material fields of one march: 1 / (1 + alpha_gamma), alpha_gamma (Eq. brinkman)
// and B_gamma (Eqs. conductivity, B), one float each per node.
static __global__ void material_kernel(const float* __restrict__ gamma, size_t n, Coef<float> c, float* __restrict__ binv,
                                float* __restrict__ alpha, float* __restrict__ B) {
  for (size_t o = (size_t)blockIdx.x * blockDim.x + threadIdx.x; o < n; o += (size_t)gridDim.x * blockDim.x) {
    const float gm = gamma[o];
    const float al = alpha_of(c, gm);
    binv[o] = 1.f / (1.f + al);
    alpha[o] = al;
    if (B) B[o] = B_of(c, gm);
  }
}

// Interior test of a tile: every node of its halo-1 ring is a non-edge node, so the
// central differences and the interior update apply everywhere.
__device__ __forceinline__ bool tile_is_interior(int x0, int y0, int tx_, int ty_, int nx, int ny) {
  return x0 >= 2 && y0 >= 2 && x0 + tx_ + 2 <= nx && y0 + ty_ + 2 <= ny;
}

// ---------------------------------------------------------------------------------
// Batched form: several lattices of unequal size packed into one arena (one 2-D
// array per field, row pitch `pitch`).  Each design owns a rectangle of the arena
// whose origin and extent are multiples of the tile shape, so the tensor maps of the
// arena serve every design and a tile's output box never leaves its design's
// rectangle.  A work list names every (design, tile) pair; each CTA walks it with the
// same static stride as the single-lattice kernels.  The per-node arithmetic is that
// of the single-lattice form, with the design's own geometry and coefficients.
// ---------------------------------------------------------------------------------
struct BatchDesign {
  Geom g;
  Coef<float> c;
  int ax, ay;  // arena origin of the design's node (0, 0)
};
struct __align__(16) BatchTile {
  int d;         // design index
  int x0, y0;    // tile origin in the design's lattice
  int interior;  // 1 when the tile's two-node halo lies inside the lattice
};

// Arena coordinates of a tile's output origin.
template <bool BATCH, int TX_, int TY_>
__device__ __forceinline__ void tile_arena_origin(int tile, int ntx, const BatchTile* work,
                                                  const BatchDesign* designs, int& gx, int& gy) {
  if constexpr (BATCH) {
    const BatchTile w = work[tile];
    gx = designs[w.d].ax + w.x0;
    gy = designs[w.d].ay + w.y0;
  } else {
    gx = (tile % ntx) * TX_;
    gy = (tile / ntx) * TY_;
  }
}

// Everything a CTA needs to know about the tile it works on.
// Geometry and coefficients are read in place (kernel parameters of the single-lattice
// form, the design table of the batched form), never copied to local memory.
template <bool BATCH>
struct TileCtx {
  const Geom* g;
  const Coef<float>* c;
  int d, x0, y0, gx, gy;  // design, origin in the design's lattice, origin in the arena
  bool interior;
  __device__ __forceinline__ TileCtx(int tile, int ntx, int tx_, int ty_, const BatchTile* work,
                                     const BatchDesign* designs, const Geom& g0, const Coef<float>& c0) {
    if constexpr (BATCH) {
      const BatchTile w = work[tile];
      const BatchDesign& bd = designs[w.d];
      g = &bd.g;
      c = &bd.c;
      d = w.d;
      x0 = w.x0;
      y0 = w.y0;
      gx = bd.ax + x0;
      gy = bd.ay + y0;
      interior = w.interior != 0;
    } else {
      g = &g0;
      c = &c0;
      d = 0;
      x0 = (tile % ntx) * tx_;
      y0 = (tile / ntx) * ty_;
      gx = x0;
      gy = y0;
      interior = tile_is_interior(x0, y0, tx_, ty_, g0.nx, g0.ny);
    }
  }
};

// ---------------------------------------------------------------------------------
// Forward
// ---------------------------------------------------------------------------------
// Output tensor maps of the forward kernel (boxes TX x TY, no halo): new drho, u, v
// (, T), then the trajectory copies u, v (, T) when stored.
template <bool TH>
struct FwdOutMaps {
  CUtensorMap m[TH ? 7 : 5];
};

template <bool TH>
struct FwdTmaArgs {
  float* drho_n;
  float* u_n;
  float* v_n;
  float* T_n;
  const float* gamma;
  float u_in;
  double* J_partial;   // per-CTA accumulator of J_O(old state), or null
  int* status;
  float* traj_u;
  float* traj_v;
  float* traj_T;
  int ntx, ntiles;
  // batched form only
  const BatchTile* work;
  const BatchDesign* designs;
  const float* u_in_d;  // inlet amplitude of each design at the new level
};

// fields staged per stage: drho, u, v, 1/(1+alpha) (, T, B)
__host__ __device__ constexpr int fwd_tma_nf(bool th) { return th ? 6 : 4; }
template <bool TH, int TX_, int TY_>
constexpr int fwd_tma_smem_bytes() {
  return 2 * fwd_tma_nf(TH) * (TX_ + 8) * (TY_ + 4) * 4 + (TH ? 18 : 9) * (TX_ + 2) * (TY_ + 2) * 4 +
         (TH ? 4 : 3) * TX_ * TY_ * 4 + 384;
}

template <bool TH, bool BATCH, int TX_, int TY_, int NT>
__global__ void __launch_bounds__(NT) fwd_tma_kernel(const __grid_constant__ TmaMaps<fwd_tma_nf(TH)> maps,
                                                     const __grid_constant__ FwdOutMaps<TH> omaps,
                                                     FwdTmaArgs<TH> a, const __grid_constant__ Geom g0,
                                                     const __grid_constant__ Coef<float> c0) {
  constexpr int NF = fwd_tma_nf(TH);
  constexpr int NO = TH ? 4 : 3;
  constexpr int BW = TX_ + 8, BH = TY_ + 4, BOX = BW * BH;
  constexpr int LX1 = TX_ + 2, LY1 = TY_ + 2, A1 = LX1 * LY1;
  extern __shared__ unsigned char smem_raw[];
  float* stage = reinterpret_cast<float*>(smem_base128(smem_raw));  // [2][NF][BOX]
  float* sout = stage + 2 * NF * BOX;                                // [NO][TX*TY] output tile
  float* F = sout + NO * TX_ * TY_;                                  // [9][A1]
  float* Gp = F + 9 * A1;                                            // thermal [9][A1]
  uint64_t* bar = reinterpret_cast<uint64_t*>(Gp + (TH ? 9 * A1 : 0));
  double* red = reinterpret_cast<double*>(bar + 2);                  // NT / 32 doubles

  if (timed_out_before(a.status)) return;
  if (!tma_layout_ok(stage, bar, a.status)) return;
  auto issue = [&](int tile, int st) {
    int gx, gy;
    tile_arena_origin<BATCH, TX_, TY_>(tile, a.ntx, a.work, a.designs, gx, gy);
    mbar_expect_tx(&bar[st], NF * BOX * 4);
    for (int f = 0; f < NF; ++f)
      tma_load_2d(stage + (st * NF + f) * BOX, &maps.m[f], gx - TMA_BXPAD, gy - 2, &bar[st]);
  };
  if (threadIdx.x == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_mbar_init();
    fence_proxy_async();
    if ((int)blockIdx.x < a.ntiles) issue(blockIdx.x, 0);
  }
  __syncthreads();

  double jloc = 0.0;
  int it = 0;
  for (int tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x, ++it) {
    const int st = it & 1;
    if (threadIdx.x == 0 && tile + (int)gridDim.x < a.ntiles) issue(tile + gridDim.x, st ^ 1);
    if (!mbar_wait(&bar[st], (it >> 1) & 1)) {
      raise_status(a.status, 6);
      if (threadIdx.x == 0) {
        mbar_wait(&bar[st ^ 1], ((it + 1) >> 1) & 1);
        bulk_wait0();
      }
      return;
    }
    const float* sdr = stage + (st * NF + 0) * BOX;
    const float* su = stage + (st * NF + 1) * BOX;
    const float* sv = stage + (st * NF + 2) * BOX;
    const float* sbi = stage + (st * NF + 3) * BOX;  // 1 / (1 + alpha)
    const float* sT = stage + (st * NF + 4) * BOX;   // thermal
    const float* sB = stage + (st * NF + 5) * BOX;   // thermal
    TileCtx<BATCH> tc(tile, a.ntx, TX_, TY_, a.work, a.designs, g0, c0);
    const Geom& g = *tc.g;
    const Coef<float>& c = *tc.c;
    const int nx = g.nx, ny = g.ny, x0 = tc.x0, y0 = tc.y0;
    const float u_in = BATCH ? a.u_in_d[tc.d] : a.u_in;

    // push values on the halo-1 region
    auto phase_a = [&](auto edge_tag) {
      constexpr bool EDGE = decltype(edge_tag)::value;
      for (int q = threadIdx.x; q < A1; q += NT) {
        const int ly = q / LX1, lx = q - ly * LX1;
        const int i = x0 - 1 + lx, j = y0 - 1 + ly;
        if (EDGE && (i < 0 || i >= nx || j < 0 || j >= ny)) {
#pragma unroll
          for (int k = 0; k < 9; ++k) {
            F[k * A1 + q] = 0.f;
            if (TH) Gp[k * A1 + q] = 0.f;
          }
          continue;
        }
        const int sx = lx + TMA_BXPAD - 1, sy = ly + 1, s2 = sy * BW + sx;
        const float uu = su[s2], vv = sv[s2];
        float dudx, dudy, dvdx, dvdy;
        if (EDGE) {
          dudx = dfdx<float, BW>(su, sx, sy, i, nx);
          dudy = dfdy<float, BW>(su, sx, sy, j, ny);
          dvdx = dfdx<float, BW>(sv, sx, sy, i, nx);
          dvdy = dfdy<float, BW>(sv, sx, sy, j, ny);
          const bool xe = (i == 0 || i == nx - 1), ye = (j == 0 || j == ny - 1);
          if (xe && ye) {
            dudx = 0.f;
            dvdy = 0.f;
          } else if (xe) {
            dudx = -dvdy;
          } else if (ye) {
            dvdy = -dudx;
          }
        } else {
          dudx = cdiff(su[s2 + 1], su[s2 - 1]);
          dudy = cdiff(su[s2 + BW], su[s2 - BW]);
          dvdx = cdiff(sv[s2 + 1], sv[s2 - 1]);
          dvdy = cdiff(sv[s2 + BW], sv[s2 - BW]);
        }
        const float dr = sdr[s2];
        {
          const float dn[9] = {0.f,           sdr[s2 + 1],      sdr[s2 + BW],     sdr[s2 - 1],     sdr[s2 - BW],
                               sdr[s2 + BW + 1], sdr[s2 + BW - 1], sdr[s2 - BW - 1], sdr[s2 - BW + 1]};
          float Fn[9];
          push9(dr, dn, uu, vv, dudx, dudy, dvdx, dvdy, c.A, Fn);
#pragma unroll
          for (int k = 0; k < 9; ++k) F[k * A1 + q] = Fn[k];
        }
        if (TH) {
          const float TT = sT[s2];
          const float dTx = EDGE ? dfdx<float, BW>(sT, sx, sy, i, nx) : cdiff(sT[s2 + 1], sT[s2 - 1]);
          const float dTy = EDGE ? dfdy<float, BW>(sT, sx, sy, j, ny) : cdiff(sT[s2 + BW], sT[s2 - BW]);
          const float tn[9] = {0.f, sT[s2 + 1], sT[s2 + BW], sT[s2 - 1], sT[s2 - BW], sT[s2 + BW + 1], sT[s2 + BW - 1],
                               sT[s2 - BW - 1], sT[s2 - BW + 1]};
          float G[9];
          gpush9(TT, tn, uu, vv, dTx, dTy, sB[s2], G);
#pragma unroll
          for (int k = 0; k < 9; ++k) Gp[k * A1 + q] = G[k];
        }
        // objective of the old state at interior tile nodes (unsteady accumulation)
        if (a.J_partial && lx >= 1 && lx <= TX_ && ly >= 1 && ly <= TY_ &&
            (!EDGE || (i > 0 && j > 0 && i < nx - 1 && j < ny - 1))) {
          jloc += (double)jo_flow<BW>(su, sv, s2, c.nu, sbi[s2], uu, vv);
          if (TH) jloc += (double)__fmul_rn(c.kappa_T, sT[s2]);
          if constexpr (TH && !BATCH)
            if (c.kappa_Q != 0.f) jloc += (double)heat_objective(c, __ldg(a.gamma + (size_t)j * nx + i), sT[s2]);
        }
      }
    };

    auto phase_b = [&](auto edge_tag) {
      constexpr bool EDGE = decltype(edge_tag)::value;
      for (int q = threadIdx.x; q < TX_ * TY_; q += NT) {
        const int oy = q / TX_, ox = q - oy * TX_;
        const int i = x0 + ox, j = y0 + oy;
        if (EDGE && (i >= nx || j >= ny)) {  // outside the lattice: the output box carries zeros
#pragma unroll
          for (int f = 0; f < NO; ++f) sout[f * TX_ * TY_ + q] = 0.f;
          continue;
        }
        const int q1 = (oy + 1) * LX1 + (ox + 1);
        const int s2 = (oy + 2) * BW + (ox + TMA_BXPAD);
        int nxo = 0, nyo = 0;
        const int cls = EDGE ? node_class(g, i, j, nxo, nyo) : C_INTERIOR;
        const float drx = sdr[s2];
        float fk[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) fk[k] = F[k * A1 + q1 - cxk(k) - cyk(k) * LX1];
        float drn, un, vn, Tn = 0.f;
        if (cls == C_INTERIOR) {
          gather9(fk, drx, sbi[s2], drn, un, vn);
          if (TH) {
            float gk[9];
#pragma unroll
            for (int k = 1; k < 9; ++k) gk[k] = Gp[k * A1 + q1 - cxk(k) - cyk(k) * LX1];
            Tn = tgather8(sT[s2], gk);
            if constexpr (!BATCH)
              if (has_thermal_sources(c)) thermal_sources(c, __ldg(a.gamma + (size_t)j * nx + i), sbi[s2], Tn, un, vn);
          }
        } else {
          float s0 = 0.f, sp = 0.f, g0 = 0.f, gp = 0.f;
#pragma unroll
          for (int k = 0; k < 9; ++k) {
            const int cx = cxk(k), cy = cyk(k);
            const int si = i - cx, sj = j - cy;
            if (si < 0 || si >= nx || sj < 0 || sj >= ny) continue;
            const int cn = cx * nxo + cy * nyo;
            if (cn == 0) s0 += fk[k];
            else if (cn > 0) sp += fk[k];
            if (TH) {
              const float gk = Gp[k * A1 + q1 - cx - cy * LX1];
              if (cn == 0) g0 += gk;
              else if (cn > 0) gp += gk;
            }
          }
          if (cls == C_CORNER) {
            const int jn = (j == 0) ? 1 : ny - 2;
            drn = sdr[(jn - y0 + 2) * BW + (ox + TMA_BXPAD)];
            un = vn = 0.f;
          } else if (cls == C_VELOCITY) {
            un = 0.f;
            if (i == 0 && j >= g.in_y0 && j <= g.in_y1) {
              un = u_in * inlet_profile<float>(g, j);
            }
            vn = 0.f;
            drn = __fadd_rn(drx, __fsub_rn(__fmaf_rn(2.f, sp, s0), __fmaf_rn(vn, (float)nyo, __fmul_rn(un, (float)nxo))));
          } else {
            drn = c.drho_out;
            const float unorm = __fadd_rn(__fmaf_rn(2.f, sp, s0), __fsub_rn(drx, c.drho_out));
            un = __fmul_rn(unorm, (float)nxo);
            vn = __fmul_rn(unorm, (float)nyo);
          }
          if (TH) {
            const int e = thermal_edge(g, i, j);
            if (g.t_kind[e] == 0) {
              Tn = c.t_val[e];
            } else if (cls == C_CORNER) {
              const int jn = (j == 0) ? 1 : ny - 2;
              Tn = sT[(jn - y0 + 2) * BW + (ox + TMA_BXPAD)];
            } else {
              Tn = tflux_edge(sT[s2], g0, gp, flux_value(g, c, e, i), un, vn, nxo, nyo);
            }
          }
        }
        sout[q] = drn;
        sout[TX_ * TY_ + q] = un;
        sout[2 * TX_ * TY_ + q] = vn;
        if (TH) sout[3 * TX_ * TY_ + q] = Tn;
        if (bad_velocity(un, vn)) raise_status(a.status, 4);
      }
    };

    if (threadIdx.x == 0) bulk_wait_read0();  // the previous tile's output copies have left sout
    if (tc.interior) {
      phase_a(std::false_type{});
      __syncthreads();
      phase_b(std::false_type{});
    } else {
      phase_a(std::true_type{});
      __syncthreads();
      phase_b(std::true_type{});
    }
    fence_proxy_async();  // make this thread's sout writes visible to the bulk copies
    __syncthreads();      // stage st and the push arrays are free again; sout complete
    if (threadIdx.x == 0) {
      for (int f = 0; f < NO; ++f) tma_store_2d(&omaps.m[f], tc.gx, tc.gy, sout + f * TX_ * TY_);
      if (a.traj_u) {
        tma_store_2d(&omaps.m[NO], tc.gx, tc.gy, sout + TX_ * TY_);
        tma_store_2d(&omaps.m[NO + 1], tc.gx, tc.gy, sout + 2 * TX_ * TY_);
        if (TH) tma_store_2d(&omaps.m[NO + 2], tc.gx, tc.gy, sout + 3 * TX_ * TY_);
      }
      bulk_commit();
    }
    if (BATCH && a.J_partial) {  // per-tile objective partial (each tile has one owner CTA)
      const double s = block_sum<NT>(jloc, red);
      if (threadIdx.x == 0) a.J_partial[tile] += s;
      jloc = 0.0;
    }
  }
  if (threadIdx.x == 0) bulk_wait0();
  if (!BATCH && a.J_partial) {
    const double s = block_sum<NT>(jloc, red);
    if (threadIdx.x == 0) a.J_partial[blockIdx.x] += s;
  }
}

// ---------------------------------------------------------------------------------
// Adjoint
// ---------------------------------------------------------------------------------
// Output tensor maps of the adjoint kernel (boxes TX x TY): the 6 (9) moments.
template <bool TH>
struct AdjOutMaps {
  CUtensorMap m[TH ? 9 : 6];
};

template <bool TH>
struct AdjTmaArgs {
  float* m0[9];       // adjoint moments at level t
  const float* gamma;
  const float* emap;  // 9 classes x 6 x 10
  float* sens;        // optional sensitivity accumulator
  int sens_flow, sens_thermal;
  int* status;
  int ntx, ntiles;
  // batched form only (gamma, sens and emap then cover every design: gamma and sens
  // with row pitch `pitch` in arena coordinates, emap with 9 x 60 entries per design)
  const BatchTile* work;
  const BatchDesign* designs;
  int pitch;
};

// Staged fields: 6 adjoint (+3 thermal), u1, v1, [u0, v0], alpha, 1/(1+alpha),
// thermal: T0, B.
__host__ __device__ constexpr int adj_tma_nf(bool th, bool same) {
  return (th ? 9 : 6) + 2 + (same ? 0 : 2) + 2 + (th ? 2 : 0);
}
template <bool TH, bool SAME, int TX_, int TY_>
constexpr int adj_tma_smem_bytes() {
  return 2 * adj_tma_nf(TH, SAME) * (TX_ + 8) * (TY_ + 4) * 4 + (9 + 3 + (TH ? 1 : 0)) * (TX_ + 2) * (TY_ + 2) * 4 +
         (TH ? 9 : 6) * TX_ * TY_ * 4 + 256;
}

template <bool TH, bool SAME, bool BATCH, int TX_, int TY_, int NT>
__global__ void __launch_bounds__(NT) adj_tma_kernel(const __grid_constant__ TmaMaps<adj_tma_nf(TH, SAME)> maps,
                                                     const __grid_constant__ AdjOutMaps<TH> omaps,
                                                     AdjTmaArgs<TH> a, const __grid_constant__ Geom g0,
                                                     const __grid_constant__ Coef<float> c0) {
  constexpr int NF = adj_tma_nf(TH, SAME);
  constexpr int NA = TH ? 9 : 6;
  constexpr int BW = TX_ + 8, BH = TY_ + 4, BOX = BW * BH;
  constexpr int LX1 = TX_ + 2, LY1 = TY_ + 2, A1 = LX1 * LY1;
  // stage field indices
  constexpr int FU1 = NA, FV1 = NA + 1, FU0 = SAME ? NA : NA + 2, FV0 = SAME ? NA + 1 : NA + 3;
  constexpr int FAL = SAME ? NA + 2 : NA + 4, FBI = FAL + 1, FT0 = FAL + 2, FB = FAL + 3;
  extern __shared__ unsigned char smem_raw[];
  float* stage = reinterpret_cast<float*>(smem_base128(smem_raw));  // [2][NF][BOX]
  float* sout = stage + 2 * NF * BOX;                                // [NA][TX*TY] output tile
  float* Pq = sout + NA * TX_ * TY_;                                 // [9][A1] push values P + c_k.V
  float* cS = Pq + 9 * A1;                                           // [3][A1] strain of the level-t state
  float* cG = cS + 3 * A1;                                           // thermal: G~ on the halo-1 region
  uint64_t* bar = reinterpret_cast<uint64_t*>(cG + (TH ? A1 : 0));

  if (timed_out_before(a.status)) return;
  if (!tma_layout_ok(stage, bar, a.status)) return;
  auto issue = [&](int tile, int st) {
    int gx, gy;
    tile_arena_origin<BATCH, TX_, TY_>(tile, a.ntx, a.work, a.designs, gx, gy);
    mbar_expect_tx(&bar[st], NF * BOX * 4);
    for (int f = 0; f < NF; ++f)
      tma_load_2d(stage + (st * NF + f) * BOX, &maps.m[f], gx - TMA_BXPAD, gy - 2, &bar[st]);
  };
  if (threadIdx.x == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_mbar_init();
    fence_proxy_async();
    if ((int)blockIdx.x < a.ntiles) issue(blockIdx.x, 0);
  }
  __syncthreads();

  int it = 0;
  for (int tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x, ++it) {
    const int st = it & 1;
    if (threadIdx.x == 0 && tile + (int)gridDim.x < a.ntiles) issue(tile + gridDim.x, st ^ 1);
    if (!mbar_wait(&bar[st], (it >> 1) & 1)) {
      raise_status(a.status, 6);
      if (threadIdx.x == 0) {
        mbar_wait(&bar[st ^ 1], ((it + 1) >> 1) & 1);
        bulk_wait0();
      }
      return;
    }
    const float* S = stage + st * NF * BOX;
    const float* sa0 = S + 0 * BOX;
    const float* sa3 = S + 3 * BOX;
    const float* sa4 = S + 4 * BOX;
    const float* sa5 = S + 5 * BOX;
    const float* su1 = S + FU1 * BOX;
    const float* sv1 = S + FV1 * BOX;
    const float* su0 = S + FU0 * BOX;
    const float* sv0 = S + FV0 * BOX;
    const float* sal = S + FAL * BOX;
    const float* sbi = S + FBI * BOX;
    const float* sT0 = S + FT0 * BOX;  // thermal
    const float* sB = S + FB * BOX;    // thermal
    TileCtx<BATCH> tc(tile, a.ntx, TX_, TY_, a.work, a.designs, g0, c0);
    const Geom& g = *tc.g;
    const Coef<float>& c = *tc.c;
    const int nx = g.nx, ny = g.ny, x0 = tc.x0, y0 = tc.y0;
    // global index of node (i, j): gbase + j * gpitch + i
    const int gpitch = BATCH ? a.pitch : nx;
    const size_t gbase = BATCH ? (size_t)(tc.gy - y0) * a.pitch + (size_t)(tc.gx - x0) : 0;
    const float* emap = BATCH ? a.emap + (size_t)tc.d * 540 : a.emap;

    auto phase_a = [&](auto edge_tag) {
      constexpr bool EDGE = decltype(edge_tag)::value;
      for (int q = threadIdx.x; q < A1; q += NT) {
        const int ly = q / LX1, lx = q - ly * LX1;
        const int i = x0 - 1 + lx, j = y0 - 1 + ly;
        if (EDGE && (i < 0 || i >= nx || j < 0 || j >= ny)) {
#pragma unroll
          for (int k = 0; k < 9; ++k) Pq[k * A1 + q] = 0.f;
          cS[q] = cS[A1 + q] = cS[2 * A1 + q] = 0.f;
          if (TH) cG[q] = 0.f;
          continue;
        }
        const int sx = lx + TMA_BXPAD - 1, sy = ly + 1, s2 = sy * BW + sx;
        const float rt = sa0[s2], ux = S[BOX + s2], uy = S[2 * BOX + s2];
        const float sxx = sa3[s2], sxy = sa4[s2], syy = sa5[s2];
        const float uu = su1[s2], vv = sv1[s2];
        float Dx, Dy;
        if (EDGE) {
          Dx = adj_div2(dfdx<float, BW>(sa3, sx, sy, i, nx), dfdy<float, BW>(sa4, sx, sy, j, ny));
          Dy = adj_div2(dfdx<float, BW>(sa4, sx, sy, i, nx), dfdy<float, BW>(sa5, sx, sy, j, ny));
        } else {
          Dx = adj_div2(cdiff(sa3[s2 + 1], sa3[s2 - 1]), cdiff(sa4[s2 + BW], sa4[s2 - BW]));
          Dy = adj_div2(cdiff(sa4[s2 + 1], sa4[s2 - 1]), cdiff(sa5[s2 + BW], sa5[s2 - BW]));
        }
        {
          float Pn[9];
          adj_pv9(rt, ux, uy, sxx, sxy, syy, uu, vv, Dx, Dy, c.A, Pn);
#pragma unroll
          for (int k = 0; k < 9; ++k) Pq[k * A1 + q] = Pn[k];
        }
        if (!EDGE || (i > 0 && j > 0 && i < nx - 1 && j < ny - 1)) {
          cS[q] = __fmul_rn(2.f, cdiff(su0[s2 + 1], su0[s2 - 1]));
          cS[A1 + q] = __fadd_rn(cdiff(su0[s2 + BW], su0[s2 - BW]), cdiff(sv0[s2 + 1], sv0[s2 - 1]));
          cS[2 * A1 + q] = __fmul_rn(2.f, cdiff(sv0[s2 + BW], sv0[s2 - BW]));
        } else {
          cS[q] = cS[A1 + q] = cS[2 * A1 + q] = 0.f;
        }
        if (TH) {
          const float* sTt = S + 6 * BOX;
          const float* sqx = S + 7 * BOX;
          const float* sqy = S + 8 * BOX;
          const float qx = sqx[s2], qy = sqy[s2];
          float divq, dBx, dBy;
          if (EDGE) {
            divq = dfdx<float, BW>(sqx, sx, sy, i, nx) + dfdy<float, BW>(sqy, sx, sy, j, ny);
            dBx = dfdx<float, BW>(sB, sx, sy, i, nx);
            dBy = dfdy<float, BW>(sB, sx, sy, j, ny);
          } else {
            divq = (sqx[s2 + 1] - sqx[s2 - 1]) * 0.5f + (sqy[s2 + BW] - sqy[s2 - BW]) * 0.5f;
            dBx = (sB[s2 + 1] - sB[s2 - 1]) * 0.5f;
            dBy = (sB[s2 + BW] - sB[s2 - BW]) * 0.5f;
          }
          cG[q] = sTt[s2] + 3.f * (qx * uu + qy * vv) - sB[s2] * divq - (dBx * qx + dBy * qy);
        }
      }
    };

    auto phase_b = [&](auto edge_tag) {
      constexpr bool EDGE = decltype(edge_tag)::value;
      for (int q = threadIdx.x; q < TX_ * TY_; q += NT) {
        const int oy = q / TX_, ox = q - oy * TX_;
        const int i = x0 + ox, j = y0 + oy;
        if (EDGE && (i >= nx || j >= ny)) {  // outside the lattice: the output box carries zeros
#pragma unroll
          for (int f = 0; f < NA; ++f) sout[f * TX_ * TY_ + q] = 0.f;
          continue;
        }
        const int q1 = (oy + 1) * LX1 + (ox + 1);
        const int s2 = (oy + 2) * BW + (ox + TMA_BXPAD);
        const bool interior = !EDGE || (i > 0 && j > 0 && i < nx - 1 && j < ny - 1);
        // the node's gamma and sensitivity, loaded before the gather so that their
        // latency overlaps it (each node belongs to one tile: no other writer)
        const size_t gi = gbase + (size_t)j * gpitch + i;
        float gm = 0.f, sold = 0.f;
        if (a.sens && interior) {
          gm = __ldg(a.gamma + gi);
          sold = a.sens[gi];
        }
        float ft[9], gt[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) {
          const int qg = q1 + cxk(k) + cyk(k) * LX1;
          ft[k] = Pq[k * A1 + qg];
          if (TH) gt[k] = cG[qg];
        }
        float m[9];
        if (interior) {
          const float w0 = 4.f / 9.f, w1 = 1.f / 9.f, w5 = 1.f / 36.f;
          adj_moments6(ft, m);
          const float al = sal[s2];
          const float uu0 = su0[s2], vv0 = sv0[s2];
          const float ju = adj_jsrc(
              c.nu, __fsub_rn(__fadd_rn(__fsub_rn(cS[q1 - 1], cS[q1 + 1]), cS[A1 + q1 - LX1]), cS[A1 + q1 + LX1]), al,
              uu0);
          const float jv = adj_jsrc(
              c.nu,
              __fsub_rn(__fadd_rn(__fsub_rn(cS[2 * A1 + q1 - LX1], cS[2 * A1 + q1 + LX1]), cS[A1 + q1 - 1]),
                        cS[A1 + q1 + 1]),
              al, vv0);
          float cpx = 0.f, cpy = 0.f;
          if (TH) {
            const float gx = gt[1] + gt[3], gy = gt[2] + gt[4], gd = gt[5] + gt[6] + gt[7] + gt[8];
            m[6] = w0 * gt[0] + w1 * (gx + gy) + w5 * gd - c.kappa_T;
            m[7] = w1 * (gt[1] - gt[3]) + w5 * (gt[5] - gt[6] - gt[7] + gt[8]);
            m[8] = w1 * (gt[2] - gt[4]) + w5 * (gt[5] + gt[6] - gt[7] - gt[8]);
            const float T0 = sT0[s2];
            cpx = T0 * m[7];
            cpy = T0 * m[8];
          }
          const float inv = sbi[s2];
          m[1] = adj_brinkman(m[1], ju, cpx, inv);
          m[2] = adj_brinkman(m[2], jv, cpy, inv);
          if constexpr (TH && !BATCH)
            if (has_thermal_sources(c)) {
              if (!a.sens) gm = __ldg(a.gamma + gi);
              m[6] = adj_thermal_T(c, gm, m[6] + c.kappa_T, m[1], m[2]);
            }
          if (a.sens) {
            float sacc = 0.f;
            if (a.sens_flow) sacc = __fadd_rn(sacc, sens_flow_term(c, gm, uu0, vv0, m[1], m[2]));
            if constexpr (TH && !BATCH)
              if (a.sens_flow) sacc += heat_sensitivity(c, gm, sT0[s2], m[6]);
            if (TH && a.sens_thermal) {
              const float dTx = (sT0[s2 + 1] - sT0[s2 - 1]) * 0.5f;
              const float dTy = (sT0[s2 + BW] - sT0[s2 - BW]) * 0.5f;
              sacc -= dB_of(c, gm) * (dTx * m[7] + dTy * m[8]);
            }
            a.sens[gi] = sold + sacc;
          }
        } else {
#pragma unroll
          for (int k = 0; k < 9; ++k) {
            const int gi = i + cxk(k), gj = j + cyk(k);
            if (gi < 0 || gi >= nx || gj < 0 || gj >= ny) {
              ft[k] = 0.f;
              gt[k] = 0.f;
            }
          }
          float kT = 0.f;
          if (TH) {
            int nxo, nyo;
            node_class(g, i, j, nxo, nyo);
            const int e = thermal_edge(g, i, j);
            const bool flux = g.t_kind[e] != 0;
            const float un = su0[s2] * (float)nxo + sv0[s2] * (float)nyo;
            const float kap = thermal_edge_solve<float>(nxo, nyo, sB[s2], flux, un, gt);
            float T_ = 0.f, qx_ = 0.f, qy_ = 0.f;
#pragma unroll
            for (int k = 0; k < 9; ++k) {
              const float gk = gt[k] * wk<float>(k);
              T_ += gk;
              qx_ += (float)cxk(k) * gk;
              qy_ += (float)cyk(k) * gk;
            }
            m[6] = T_;
            m[7] = qx_;
            m[8] = qy_;
            if (flux) kT = kap * sT0[s2];
          }
          const int ec = edge_class(g, i, j);
          const float* M = emap + ec * 60;
#pragma unroll
          for (int r = 0; r < 6; ++r) m[r] = adj_edge_row(M + r * 10, ft, kT);
          if constexpr (!BATCH) {  // the static pressure drop (steady single lattices only)
            const float jb = edge_objective_term(g, c, ec, j);
            if (jb != 0.f)
#pragma unroll
              for (int r = 0; r < 6; ++r) m[r] = __fmaf_rn(jb, emap[540 + ec * 6 + r], m[r]);
          }
        }
#pragma unroll
        for (int f = 0; f < NA; ++f) sout[f * TX_ * TY_ + q] = m[f];
        if (!(m[1] * m[1] + m[2] * m[2] < 1e30f)) raise_status(a.status, 4);
      }
    };

    if (threadIdx.x == 0) bulk_wait_read0();  // the previous tile's output copies have left sout
    if (tc.interior) {
      phase_a(std::false_type{});
      __syncthreads();
      phase_b(std::false_type{});
    } else {
      phase_a(std::true_type{});
      __syncthreads();
      phase_b(std::true_type{});
    }
    fence_proxy_async();
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int f = 0; f < NA; ++f) tma_store_2d(&omaps.m[f], tc.gx, tc.gy, sout + f * TX_ * TY_);
      bulk_commit();
    }
  }
  if (threadIdx.x == 0) bulk_wait0();
}

}  // namespace lks
