// lks_resident.cuh -- persistent, shared-memory-resident forms of the LKS and ALKS
// steady marches for lattices whose tiles fit one CTA per tile on the GPU at once.
//
// A cooperative launch makes every tile's CTA resident for the whole march.  Each
// CTA keeps its tile plus a two-node halo in shared memory and runs all time steps
// itself.  After each step it writes the tile's new values to a double-buffered
// global array (L2-resident at these sizes), publishes the step number in its
// tile flag (release), waits for the flags of its eight neighbours (acquire,
// bounded spin) and reloads only the halo ring.  No kernel launch and no grid-wide
// barrier per step.
//
// The arithmetic per node is the one of fwd_step_kernel / adj_step_kernel in
// lks_kernels.cuh (same helpers, same order of operations).
#pragma once
#include "lks_kernels.cuh"

namespace lks {

constexpr long long kSpinLimit = 1ll << 22;  // ~0.3 s with the back-off below

__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(int* p, int v) {
  asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Bounded wait until *flag >= target.  On timeout records LKS_ERR_TIMEOUT (6) in the
// status word and returns false.
__device__ __forceinline__ bool wait_flag(const int* flag, int target, int* status) {
  for (long long it = 0; it < kSpinLimit; ++it) {
    if (ld_acquire(flag) >= target) return true;
    if (it > 32) __nanosleep(64);
  }
  raise_status(status, 6);
  return false;
}

template <typename R>
struct ResArgs {
  R* buf[2][9];      // double-buffered global fields (state: drho,u,v[,T]; adjoint: 6 or 9)
  int cur;           // buffer holding the starting level
  const R* u;        // adjoint: frozen state u, v (steady)
  const R* v;
  const R* gamma;
  const R* emap;     // adjoint edge maps (9 x 6 x 10)
  int* flags;        // one per tile, zero at launch
  int* status;
  int n_steps;
  int t0;            // forward: time level of the starting state
  R u_in;            // forward: inlet peak velocity (steady)
  int ntx;           // tiles along x
};

// Load a field's halo-2 region for a tile; only_ring = true skips the tile interior.
template <typename R, int TXR, int TYR, int NT>
__device__ __forceinline__ void res_load(R* s, const R* g, int x0, int y0, int nx, int ny, bool only_ring) {
  constexpr int LX = TXR + 4, LY = TYR + 4;
  for (int q = threadIdx.x; q < LX * LY; q += NT) {
    const int ly = q / LX, lx = q - ly * LX;
    if (only_ring && lx >= 2 && lx < TXR + 2 && ly >= 2 && ly < TYR + 2) continue;
    const int i = x0 - 2 + lx, j = y0 - 2 + ly;
    R v = R(0);
    if (i >= 0 && i < nx && j >= 0 && j < ny) v = __ldcg(g + (size_t)j * nx + i);
    s[q] = v;
  }
}

// Publish this tile's step and wait for the neighbours; returns false on timeout.
__device__ __forceinline__ bool res_exchange(int* flags, int tile, int tx, int ty, int ntx, int nty, int step,
                                             int* status, int* s_abort) {
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) st_release(flags + tile, step);
  if (threadIdx.x < 9 && threadIdx.x != 4) {
    const int dx = (int)threadIdx.x % 3 - 1, dy = (int)threadIdx.x / 3 - 1;
    const int nxt = tx + dx, nyt = ty + dy;
    if (nxt >= 0 && nxt < ntx && nyt >= 0 && nyt < nty)
      if (!wait_flag(flags + nyt * ntx + nxt, step, status)) atomicExch(s_abort, 1);
  }
  __syncthreads();
  return *s_abort == 0;
}

template <bool TH, int TXR, int TYR>
constexpr int fwd_res_smem_elems() {
  return (TH ? 4 : 3) * (TXR + 4) * (TYR + 4) + (TH ? 9 : 6) * (TXR + 2) * (TYR + 2) + TXR * TYR;
}

// Steady forward march, resident form.  Buffers hold drho, u, v (, T).
template <typename R, bool TH, int TXR, int TYR, int NT>
__global__ void __launch_bounds__(NT, 1) fwd_resident_kernel(ResArgs<R> a, Geom g, Coef<R> c) {
  constexpr int LX2 = TXR + 4, LY2 = TYR + 4, LX1 = TXR + 2, LY1 = TYR + 2;
  constexpr int A2 = LX2 * LY2, A1 = LX1 * LY1;
  constexpr int NPT = (TXR * TYR + NT - 1) / NT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R* sm = reinterpret_cast<R*>(smem_raw);
  R* sdr = sm;
  R* su = sdr + A2;
  R* sv = su + A2;
  R* sT = sv + A2;                      // thermal only
  R* ca0 = sT + (TH ? A2 : 0);
  R* cbx = ca0 + A1;
  R* cby = cbx + A1;
  R* cqx = cby + A1;
  R* cqy = cqx + A1;
  R* cqxy = cqy + A1;
  R* ctx = cqxy + A1;                   // thermal only: tq_x, tq_y, B
  R* cty = ctx + (TH ? A1 : 0);
  R* cB = cty + (TH ? A1 : 0);
  R* sinv = cB + (TH ? A1 : 0);         // 1 / (1 + alpha) on the tile
  __shared__ int s_abort;

  const int nx = g.nx, ny = g.ny;
  const int tile = blockIdx.x, tx = tile % a.ntx, ty = tile / a.ntx;
  const int nty = gridDim.x / a.ntx;
  const int x0 = tx * TXR, y0 = ty * TYR;
  if (threadIdx.x == 0) s_abort = 0;
  const int nf = TH ? 4 : 3;
  R* sf[4] = {sdr, su, sv, sT};
  for (int f = 0; f < nf; ++f) res_load<R, TXR, TYR, NT>(sf[f], a.buf[a.cur][f], x0, y0, nx, ny, false);
  for (int q = threadIdx.x; q < TXR * TYR; q += NT) {
    const int ly = q / TXR, lx = q - ly * TXR, i = x0 + lx, j = y0 + ly;
    sinv[q] = (i < nx && j < ny) ? R(1) / (R(1) + alpha_of(c, __ldg(a.gamma + (size_t)j * nx + i))) : R(0);
  }
  if (TH)
    for (int q = threadIdx.x; q < A1; q += NT) {
      const int ly = q / LX1, lx = q - ly * LX1, i = x0 - 1 + lx, j = y0 - 1 + ly;
      cB[q] = (i >= 0 && i < nx && j >= 0 && j < ny) ? B_of(c, __ldg(a.gamma + (size_t)j * nx + i)) : R(0);
    }
  __syncthreads();

  for (int s = 0; s < a.n_steps; ++s) {
    // equilibrium coefficients on the halo-1 region
    for (int q = threadIdx.x; q < A1; q += NT) {
      const int ly = q / LX1, lx = q - ly * LX1;
      const int i = x0 - 1 + lx, j = y0 - 1 + ly;
      if (i < 0 || i >= nx || j < 0 || j >= ny) {
        ca0[q] = cbx[q] = cby[q] = cqx[q] = cqy[q] = cqxy[q] = R(0);
        if (TH) ctx[q] = cty[q] = R(0);
        continue;
      }
      const int sx = lx + 1, sy = ly + 1, s2 = sy * LX2 + sx;
      const R uu = su[s2], vv = sv[s2];
      R dudx = dfdx<R, LX2>(su, sx, sy, i, nx);
      const R dudy = dfdy<R, LX2>(su, sx, sy, j, ny);
      const R dvdx = dfdx<R, LX2>(sv, sx, sy, i, nx);
      R dvdy = dfdy<R, LX2>(sv, sx, sy, j, ny);
      const bool xe = (i == 0 || i == nx - 1), ye = (j == 0 || j == ny - 1);
      if (xe && ye) {
        dudx = R(0);
        dvdy = R(0);
      } else if (xe) {
        dudx = -dvdy;
      } else if (ye) {
        dvdy = -dudx;
      }
      ca0[q] = -R(1.5) * (uu * uu + vv * vv);
      cbx[q] = R(3) * uu;
      cby[q] = R(3) * vv;
      cqx[q] = R(4.5) * uu * uu + c.A * (R(2) * dudx);
      cqy[q] = R(4.5) * vv * vv + c.A * (R(2) * dvdy);
      cqxy[q] = R(9) * uu * vv + R(2) * c.A * (dudy + dvdx);
      if (TH) {
        const R TT = sT[s2];
        ctx[q] = R(3) * TT * uu + cB[q] * dfdx<R, LX2>(sT, sx, sy, i, nx);
        cty[q] = R(3) * TT * vv + cB[q] * dfdy<R, LX2>(sT, sx, sy, j, ny);
      }
    }
    __syncthreads();

    R out[NPT][4];
#pragma unroll
    for (int p = 0; p < NPT; ++p) {
      const int lin = threadIdx.x + p * NT;
      out[p][0] = out[p][1] = out[p][2] = out[p][3] = R(0);
      if (lin >= TXR * TYR) continue;
      const int oy = lin / TXR, ox = lin - oy * TXR;
      const int i = x0 + ox, j = y0 + oy;
      if (i >= nx || j >= ny) continue;
      const int q = (oy + 1) * LX1 + (ox + 1);
      const int s2 = (oy + 2) * LX2 + (ox + 2);
      int nxo, nyo;
      const int cls = node_class(g, i, j, nxo, nyo);
      const R drx = sdr[s2];
      R drn, un, vn, Tn = R(0);
      if (cls == C_INTERIOR) {
        const int W = q - 1, E = q + 1, S = q - LX1, N = q + LX1;
        const int SW = S - 1, SE = S + 1, NE = N + 1, NW = N - 1;
        const R f0 = ca0[q] * (R(4) / R(9));
        const R f1 = ((sdr[s2 - 1] - drx) + ca0[W] + cbx[W] + cqx[W]) * (R(1) / R(9));
        const R f3 = ((sdr[s2 + 1] - drx) + ca0[E] - cbx[E] + cqx[E]) * (R(1) / R(9));
        const R f2 = ((sdr[s2 - LX2] - drx) + ca0[S] + cby[S] + cqy[S]) * (R(1) / R(9));
        const R f4 = ((sdr[s2 + LX2] - drx) + ca0[N] - cby[N] + cqy[N]) * (R(1) / R(9));
        const R d5 = (sdr[s2 - LX2 - 1] - drx) + ca0[SW] + cqx[SW] + cqy[SW];
        const R d6 = (sdr[s2 - LX2 + 1] - drx) + ca0[SE] + cqx[SE] + cqy[SE];
        const R d7 = (sdr[s2 + LX2 + 1] - drx) + ca0[NE] + cqx[NE] + cqy[NE];
        const R d8 = (sdr[s2 + LX2 - 1] - drx) + ca0[NW] + cqx[NW] + cqy[NW];
        const R f5 = (d5 + cbx[SW] + cby[SW] + cqxy[SW]) * (R(1) / R(36));
        const R f6 = (d6 - cbx[SE] + cby[SE] - cqxy[SE]) * (R(1) / R(36));
        const R f7 = (d7 - cbx[NE] - cby[NE] + cqxy[NE]) * (R(1) / R(36));
        const R f8 = (d8 + cbx[NW] - cby[NW] - cqxy[NW]) * (R(1) / R(36));
        drn = drx + (f0 + f1 + f2 + f3 + f4 + f5 + f6 + f7 + f8);
        const R inv = sinv[oy * TXR + ox];
        un = (f1 - f3 + f5 - f6 - f7 + f8) * inv;
        vn = (f2 - f4 + f5 + f6 - f7 - f8) * inv;
        if (TH) {
          const R Tx = sT[s2];
          R Ts = ((sT[s2 - 1] - Tx) + ctx[W] + (sT[s2 + 1] - Tx) - ctx[E] + (sT[s2 - LX2] - Tx) + cty[S] +
                  (sT[s2 + LX2] - Tx) - cty[N]) * (R(1) / R(9));
          Ts += ((sT[s2 - LX2 - 1] - Tx) + ctx[SW] + cty[SW] + (sT[s2 - LX2 + 1] - Tx) - ctx[SE] + cty[SE] +
                 (sT[s2 + LX2 + 1] - Tx) - ctx[NE] - cty[NE] + (sT[s2 + LX2 - 1] - Tx) + ctx[NW] - cty[NW]) *
                (R(1) / R(36));
          Tn = Tx + Ts;
        }
      } else {
        R s0 = R(0), sp = R(0), g0 = R(0), gp = R(0);
#pragma unroll
        for (int k = 0; k < 9; ++k) {
          const int cx = cxk(k), cy = cyk(k);
          const int si = i - cx, sj = j - cy;
          if (si < 0 || si >= nx || sj < 0 || sj >= ny) continue;
          const int qs = q - cx - cy * LX1, ss = s2 - cx - cy * LX2;
          const R fk = wk<R>(k) * ((sdr[ss] - drx) + ca0[qs] + R(cx) * cbx[qs] + R(cy) * cby[qs] +
                                   R(cx * cx) * cqx[qs] + R(cy * cy) * cqy[qs] + R(cx * cy) * cqxy[qs]);
          const int cn = cx * nxo + cy * nyo;
          if (cn == 0) s0 += fk;
          else if (cn > 0) sp += fk;
          if (TH) {
            const R gk = wk<R>(k) * ((sT[ss] - sT[s2]) + R(cx) * ctx[qs] + R(cy) * cty[qs]);
            if (cn == 0) g0 += gk;
            else if (cn > 0) gp += gk;
          }
        }
        if (cls == C_CORNER) {
          const int jn = (j == 0) ? 1 : ny - 2;
          drn = sdr[(jn - y0 + 2) * LX2 + (ox + 2)];
          un = vn = R(0);
        } else if (cls == C_VELOCITY) {
          un = R(0);
          if (i == 0 && j >= g.in_y0 && j <= g.in_y1) {
            const double H = (double)(g.in_y1 - g.in_y0), y = (double)(j - g.in_y0);
            un = a.u_in * (R)(4.0 * y * (H - y) / (H * H));
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
            Tn = sT[(jn - y0 + 2) * LX2 + (ox + 2)];
          } else {
            Tn = (sT[s2] + g0 + R(2) * gp + c.t_val[e]) / (R(1) + un * R(nxo) + vn * R(nyo));
          }
        }
      }
      out[p][0] = drn;
      out[p][1] = un;
      out[p][2] = vn;
      out[p][3] = Tn;
      if (bad_velocity(un, vn)) raise_status(a.status, 4);
    }
    __syncthreads();  // every read of the old level is done

    const int nb = (a.cur + s + 1) & 1;
#pragma unroll
    for (int p = 0; p < NPT; ++p) {
      const int lin = threadIdx.x + p * NT;
      if (lin >= TXR * TYR) continue;
      const int oy = lin / TXR, ox = lin - oy * TXR;
      const int i = x0 + ox, j = y0 + oy;
      if (i >= nx || j >= ny) continue;
      const int s2 = (oy + 2) * LX2 + (ox + 2);
      const size_t o = (size_t)j * nx + i;
      for (int f = 0; f < nf; ++f) {
        sf[f][s2] = out[p][f];
        __stcg(a.buf[nb][f] + o, out[p][f]);
      }
    }
    if (!res_exchange(a.flags, tile, tx, ty, a.ntx, nty, s + 1, a.status, &s_abort)) return;
    for (int f = 0; f < nf; ++f) res_load<R, TXR, TYR, NT>(sf[f], a.buf[nb][f], x0, y0, nx, ny, true);
    __syncthreads();
  }
}

template <int TXR, int TYR>
constexpr int adj_res_smem_elems() {
  return 8 * (TXR + 4) * (TYR + 4) + 3 * (TXR + 2) * (TYR + 2) + 3 * TXR * TYR;
}

// Steady ALKS march, resident form (non-thermal).  Buffers hold the six adjoint
// moments; the state (u, v) is frozen.
template <typename R, int TXR, int TYR, int NT>
__global__ void __launch_bounds__(NT, 1) adj_resident_kernel(ResArgs<R> a, Geom g, Coef<R> c) {
  constexpr int LX2 = TXR + 4, LY2 = TYR + 4, LX1 = TXR + 2, LY1 = TYR + 2;
  constexpr int A2 = LX2 * LY2, A1 = LX1 * LY1;
  constexpr int NPT = (TXR * TYR + NT - 1) / NT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R* sm = reinterpret_cast<R*>(smem_raw);
  R* sa[6];
  for (int f = 0; f < 6; ++f) sa[f] = sm + f * A2;
  R* su = sm + 6 * A2;
  R* sv = su + A2;
  R* cP = sv + A2;
  R* cVx = cP + A1;
  R* cVy = cVx + A1;
  R* sju = cVy + A1;   // objective source dJ_O/du, dJ_O/dv on the tile
  R* sjv = sju + TXR * TYR;
  R* sinv = sjv + TXR * TYR;
  __shared__ int s_abort;

  const int nx = g.nx, ny = g.ny;
  const int tile = blockIdx.x, tx = tile % a.ntx, ty = tile / a.ntx;
  const int nty = gridDim.x / a.ntx;
  const int x0 = tx * TXR, y0 = ty * TYR;
  if (threadIdx.x == 0) s_abort = 0;
  for (int f = 0; f < 6; ++f) res_load<R, TXR, TYR, NT>(sa[f], a.buf[a.cur][f], x0, y0, nx, ny, false);
  res_load<R, TXR, TYR, NT>(su, a.u, x0, y0, nx, ny, false);
  res_load<R, TXR, TYR, NT>(sv, a.v, x0, y0, nx, ny, false);
  __syncthreads();
  // Strain of the frozen state on interior nodes (into cP / cVx / cVy for now),
  // then the objective source of every tile node.
  for (int q = threadIdx.x; q < A1; q += NT) {
    const int ly = q / LX1, lx = q - ly * LX1;
    const int i = x0 - 1 + lx, j = y0 - 1 + ly;
    R Sxx = R(0), Sxy = R(0), Syy = R(0);
    if (i > 0 && j > 0 && i < nx - 1 && j < ny - 1) {
      const int s2 = (ly + 1) * LX2 + lx + 1;
      Sxx = (su[s2 + 1] - su[s2 - 1]);
      Syy = (sv[s2 + LX2] - sv[s2 - LX2]);
      Sxy = (su[s2 + LX2] - su[s2 - LX2]) * R(0.5) + (sv[s2 + 1] - sv[s2 - 1]) * R(0.5);
    }
    cP[q] = Sxx;
    cVx[q] = Sxy;
    cVy[q] = Syy;
  }
  __syncthreads();
  for (int q = threadIdx.x; q < TXR * TYR; q += NT) {
    const int oy = q / TXR, ox = q - oy * TXR, i = x0 + ox, j = y0 + oy;
    R ju = R(0), jv = R(0), inv = R(0);
    if (i < nx && j < ny) {
      const int q1 = (oy + 1) * LX1 + ox + 1, s2 = (oy + 2) * LX2 + ox + 2;
      const R al = alpha_of(c, __ldg(a.gamma + (size_t)j * nx + i));
      ju = c.nu * (cP[q1 - 1] - cP[q1 + 1] + cVx[q1 - LX1] - cVx[q1 + LX1]) + R(2) * al * su[s2];
      jv = c.nu * (cVy[q1 - LX1] - cVy[q1 + LX1] + cVx[q1 - 1] - cVx[q1 + 1]) + R(2) * al * sv[s2];
      inv = R(1) / (R(1) + al);
    }
    sju[q] = ju;
    sjv[q] = jv;
    sinv[q] = inv;
  }
  __syncthreads();

  for (int s = 0; s < a.n_steps; ++s) {
    for (int q = threadIdx.x; q < A1; q += NT) {
      const int ly = q / LX1, lx = q - ly * LX1;
      const int i = x0 - 1 + lx, j = y0 - 1 + ly;
      if (i < 0 || i >= nx || j < 0 || j >= ny) {
        cP[q] = cVx[q] = cVy[q] = R(0);
        continue;
      }
      const int sx = lx + 1, sy = ly + 1, s2 = sy * LX2 + sx;
      const R rt = sa[0][s2], ux = sa[1][s2], uy = sa[2][s2];
      const R sxx = sa[3][s2], sxy = sa[4][s2], syy = sa[5][s2];
      const R uu = su[s2], vv = sv[s2];
      const R Dx = R(2) * (dfdx<R, LX2>(sa[3], sx, sy, i, nx) + dfdy<R, LX2>(sa[4], sx, sy, j, ny));
      const R Dy = R(2) * (dfdx<R, LX2>(sa[4], sx, sy, i, nx) + dfdy<R, LX2>(sa[5], sx, sy, j, ny));
      cP[q] = rt;
      cVx[q] = R(3) * (ux + R(3) * (sxx * uu + sxy * vv) - rt * uu) - c.A * Dx;
      cVy[q] = R(3) * (uy + R(3) * (sxy * uu + syy * vv) - rt * vv) - c.A * Dy;
    }
    __syncthreads();

    R out[NPT][6];
#pragma unroll
    for (int p = 0; p < NPT; ++p) {
      const int lin = threadIdx.x + p * NT;
#pragma unroll
      for (int f = 0; f < 6; ++f) out[p][f] = R(0);
      if (lin >= TXR * TYR) continue;
      const int oy = lin / TXR, ox = lin - oy * TXR;
      const int i = x0 + ox, j = y0 + oy;
      if (i >= nx || j >= ny) continue;
      const int q = (oy + 1) * LX1 + (ox + 1);
      const bool interior = i > 0 && j > 0 && i < nx - 1 && j < ny - 1;
      R ft[9];
#pragma unroll
      for (int k = 0; k < 9; ++k) {
        const int cx = cxk(k), cy = cyk(k);
        const int gi = i + cx, gj = j + cy;
        const bool in = gi >= 0 && gi < nx && gj >= 0 && gj < ny;
        const int qg = q + cx + cy * LX1;
        ft[k] = in ? cP[qg] + R(cx) * cVx[qg] + R(cy) * cVy[qg] : R(0);
      }
      if (interior) {
        const R w0 = R(4) / R(9), w1 = R(1) / R(9), w5 = R(1) / R(36);
        const R ax = ft[1] + ft[3], ay = ft[2] + ft[4], dg = ft[5] + ft[6] + ft[7] + ft[8];
        out[p][0] = w0 * ft[0] + w1 * (ax + ay) + w5 * dg;
        const R m1 = w1 * (ft[1] - ft[3]) + w5 * (ft[5] - ft[6] - ft[7] + ft[8]);
        const R m2 = w1 * (ft[2] - ft[4]) + w5 * (ft[5] + ft[6] - ft[7] - ft[8]);
        out[p][3] = w1 * ax + w5 * dg;
        out[p][4] = w5 * (ft[5] - ft[6] + ft[7] - ft[8]);
        out[p][5] = w1 * ay + w5 * dg;
        const int qt = oy * TXR + ox;
        const R inv = sinv[qt];
        out[p][1] = (m1 - sju[qt] * (R(1) / R(3))) * inv;
        out[p][2] = (m2 - sjv[qt] * (R(1) / R(3))) * inv;
      } else {
        const R* M = a.emap + edge_class(g, i, j) * 60;
#pragma unroll
        for (int r = 0; r < 6; ++r) {
          R acc = R(0);
#pragma unroll
          for (int k = 0; k < 9; ++k) acc += M[r * 10 + k] * ft[k];
          out[p][r] = acc;
        }
      }
      if (!(out[p][1] * out[p][1] + out[p][2] * out[p][2] < R(1e30))) raise_status(a.status, 4);
    }
    __syncthreads();

    const int nb = (a.cur + s + 1) & 1;
#pragma unroll
    for (int p = 0; p < NPT; ++p) {
      const int lin = threadIdx.x + p * NT;
      if (lin >= TXR * TYR) continue;
      const int oy = lin / TXR, ox = lin - oy * TXR;
      const int i = x0 + ox, j = y0 + oy;
      if (i >= nx || j >= ny) continue;
      const int s2 = (oy + 2) * LX2 + (ox + 2);
      const size_t o = (size_t)j * nx + i;
#pragma unroll
      for (int f = 0; f < 6; ++f) {
        sa[f][s2] = out[p][f];
        __stcg(a.buf[nb][f] + o, out[p][f]);
      }
    }
    if (!res_exchange(a.flags, tile, tx, ty, a.ntx, nty, s + 1, a.status, &s_abort)) return;
    for (int f = 0; f < 6; ++f) res_load<R, TXR, TYR, NT>(sa[f], a.buf[nb][f], x0, y0, nx, ny, true);
    __syncthreads();
  }
}

}  // namespace lks
