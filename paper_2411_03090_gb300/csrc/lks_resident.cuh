// lks_resident.cuh -- persistent, shared-memory-resident forms of the LKS and ALKS
// steady marches for lattices whose tiles fit one CTA per tile on the GPU at once.
//
// A cooperative launch makes every tile's CTA resident for the whole march.  Each
// CTA keeps its tile plus a two-node halo in shared memory and runs all time steps
// itself.  After each step it writes the tile's new values to a double-buffered
// global array (L2-resident at these sizes), publishes the step number in its tile
// flag (release) and, for the next step, first computes everything that needs no
// halo (the tile interior), then waits for its eight neighbours' flags (acquire,
// bounded spin), reloads only the two-node halo ring and finishes the tile band.
// Only the band (the two outer rows and columns the neighbours read) goes to global
// memory each step; the interior stays in shared memory until the last step.
// No kernel launch and no grid-wide barrier per step.
//
// Streaming is done in push form: each node first evaluates the nine values it
// sends (f_k^eq towards x + c_k for LKS, f~ towards x - c_k for ALKS); each output
// node then sums nine shared-memory values.  The arithmetic per node is the one of
// fwd_step_kernel / adj_step_kernel (the same terms; the order of the final sums
// may differ by rounding).
#pragma once
#include "lks_kernels.cuh"

namespace lks {

constexpr long long kSpinLimit = 1ll << 22;  // bounded wait (about a second at most)

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
    if (it > 64) __nanosleep(32);
  }
  raise_status(status, 6);
  return false;
}

template <typename R>
struct ResArgs {
  R* buf[2][9];      // double-buffered global fields (state: drho,u,v[,T]; adjoint: 6)
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

// Load a field's halo-2 region for a tile; only_ring skips the tile interior.
template <typename R, int TXR, int TYR, int NT>
__device__ __forceinline__ void res_load(R* s, const R* g, int x0, int y0, int nx, int ny, bool only_ring) {
  constexpr int LX = TXR + 4, LY = TYR + 4;
  if (!only_ring) {
    for (int q = threadIdx.x; q < LX * LY; q += NT) {
      const int ly = q / LX, lx = q - ly * LX;
      const int i = x0 - 2 + lx, j = y0 - 2 + ly;
      R v = R(0);
      if (i >= 0 && i < nx && j >= 0 && j < ny) v = __ldcg(g + (size_t)j * nx + i);
      s[q] = v;
    }
    return;
  }
  // ring: two rows at the bottom and top (full width), two columns left and right
  constexpr int NROW = 4 * LX, NCOL = 4 * TYR;
  for (int q = threadIdx.x; q < NROW + NCOL; q += NT) {
    int lx, ly;
    if (q < NROW) {
      const int r = q / LX;
      lx = q - r * LX;
      ly = r < 2 ? r : TYR + r;  // rows 0,1 and TYR+2, TYR+3
    } else {
      const int t = q - NROW, c = t / TYR;
      ly = 2 + (t - c * TYR);
      lx = c < 2 ? c : TXR + c;  // columns 0,1 and TXR+2, TXR+3
    }
    const int i = x0 - 2 + lx, j = y0 - 2 + ly;
    R v = R(0);
    if (i >= 0 && i < nx && j >= 0 && j < ny) v = __ldcg(g + (size_t)j * nx + i);
    s[ly * LX + lx] = v;
  }
}

// Ring of the halo-2 region (two rows below and above the tile at full width, two
// columns left and right of it) for nf fields at once: all loads are issued before
// any shared-memory store, so the ring costs one L2 round trip.
template <typename R, int TXR, int TYR, int NT, int NF>
__device__ __forceinline__ void res_load_ring(R* const* s, R* const* g, int nf, int x0, int y0, int nx,
                                              int ny) {
  constexpr int LX = TXR + 4, NROW = 4 * LX, NCOL = 4 * TYR, NR = NROW + NCOL;
  constexpr int PER = (NR + NT - 1) / NT;
  R v[PER][NF];
  int pos[PER];
#pragma unroll
  for (int p = 0; p < PER; ++p) {
    const int q = threadIdx.x + p * NT;
    pos[p] = -1;
    if (q >= NR) continue;
    int lx, ly;
    if (q < NROW) {
      const int r = q / LX;
      lx = q - r * LX;
      ly = r < 2 ? r : TYR + r;
    } else {
      const int t = q - NROW, c = t / TYR;
      ly = 2 + (t - c * TYR);
      lx = c < 2 ? c : TXR + c;
    }
    const int i = x0 - 2 + lx, j = y0 - 2 + ly;
    pos[p] = ly * LX + lx;
    const bool in = i >= 0 && i < nx && j >= 0 && j < ny;
    const size_t off = in ? (size_t)j * nx + i : 0;
#pragma unroll
    for (int f = 0; f < NF; ++f) v[p][f] = (in && f < nf) ? __ldcg(g[f] + off) : R(0);
  }
#pragma unroll
  for (int p = 0; p < PER; ++p) {
    if (pos[p] < 0) continue;
#pragma unroll
    for (int f = 0; f < NF; ++f)
      if (f < nf) s[f][pos[p]] = v[p][f];
  }
}

// Publish this tile's step: the CTA barrier orders every thread's global writes
// before thread 0's release store (the release is cumulative).
__device__ __forceinline__ void res_publish(int* flags, int tile, int step) {
  __syncthreads();
  if (threadIdx.x == 0) st_release(flags + tile, step);
}

// Wait for the eight neighbours to publish `step`; false on timeout (all threads).
__device__ __forceinline__ bool res_wait(const int* flags, int tx, int ty, int ntx, int nty, int step,
                                         int* status, int* s_abort) {
  if (threadIdx.x < 9 && threadIdx.x != 4) {
    const int dx = (int)threadIdx.x % 3 - 1, dy = (int)threadIdx.x / 3 - 1;
    const int nxt = tx + dx, nyt = ty + dy;
    if (nxt >= 0 && nxt < ntx && nyt >= 0 && nyt < nty)
      if (!wait_flag(flags + nyt * ntx + nxt, step, status)) atomicExch(s_abort, 1);
  }
  __syncthreads();
  return *s_abort == 0;
}

// Region helpers: positions of the halo-1 coefficient region (lx, ly in [0, TXR+2) x
// [0, TYR+2)) that need no halo data ("inner": 2 <= lx <= TXR-1, 2 <= ly <= TYR-1),
// and tile outputs (ox, oy) whose stencil stays inner (2 <= ox <= TXR-3, ...).
template <int TXR, int TYR>
__device__ __forceinline__ bool coef_inner(int lx, int ly) {
  return lx >= 2 && lx <= TXR - 1 && ly >= 2 && ly <= TYR - 1;
}
template <int TXR, int TYR>
__device__ __forceinline__ bool out_inner(int ox, int oy) {
  return ox >= 2 && ox <= TXR - 3 && oy >= 2 && oy <= TYR - 3;
}

// Positions of the halo-1 region outside the inner block, enumerated directly:
// rows 0, 1, TYR, TYR+1 at full width, then columns 0, 1, TXR, TXR+1 of rows
// 2 .. TYR-1.  Count 4 (TXR+2) + 4 (TYR-2).
template <int TXR, int TYR>
__device__ __forceinline__ void band_coef_pos(int t, int& lx, int& ly) {
  constexpr int LX1 = TXR + 2, LY1 = TYR + 2;
  if (t < 4 * LX1) {
    const int r = t / LX1;
    lx = t - r * LX1;
    ly = r < 2 ? r : LY1 - 4 + r;
  } else {
    const int u = t - 4 * LX1, r = u / 4, cidx = u - r * 4;
    ly = 2 + r;
    lx = cidx < 2 ? cidx : LX1 - 4 + cidx;
  }
}

template <bool TH, int TXR, int TYR>
constexpr int fwd_res_smem_elems() {
  return (TH ? 4 : 3) * (TXR + 4) * (TYR + 4) + (TH ? 19 : 9) * (TXR + 2) * (TYR + 2) + TXR * TYR;
}

// ---------------------------------------------------------------------------------
// Steady LKS march, resident form.  Buffers hold drho, u, v (, T).
// ---------------------------------------------------------------------------------
template <typename R, bool TH, int TXR, int TYR, int NT>
__global__ void __launch_bounds__(NT, 1) fwd_resident_kernel(ResArgs<R> a, Geom g, Coef<R> c) {
  constexpr int LX2 = TXR + 4, LY2 = TYR + 4, LX1 = TXR + 2, LY1 = TYR + 2;
  constexpr int A2 = LX2 * LY2, A1 = LX1 * LY1, NO = TXR * TYR;
  constexpr int NOI = (TXR - 4) * (TYR - 4), NOO = NO - NOI;
  constexpr int PI = (NOI + NT - 1) / NT, PO = (NOO + NT - 1) / NT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R* sm = reinterpret_cast<R*>(smem_raw);
  R* sdr = sm;
  R* su = sdr + A2;
  R* sv = su + A2;
  R* sT = sv + A2;                   // thermal only
  R* F = sT + (TH ? A2 : 0);         // push values f_k^eq, 9 x A1
  R* G = F + 9 * A1;                 // thermal push values g_k^eq, 9 x A1
  R* cB = G + (TH ? 9 * A1 : 0);     // thermal: B on the halo-1 region
  R* sinv = cB + (TH ? A1 : 0);      // 1 / (1 + alpha) on the tile
  __shared__ int s_abort;

  if (a.status && *reinterpret_cast<const volatile int*>(a.status) == 6) return;  // earlier timeout
  const int nx = g.nx, ny = g.ny;
  const int tile = blockIdx.x, tx = tile % a.ntx, ty = tile / a.ntx;
  const int nty = gridDim.x / a.ntx;
  const int x0 = tx * TXR, y0 = ty * TYR;
  if (threadIdx.x == 0) s_abort = 0;
  const int nf = TH ? 4 : 3;
  R* sf[4] = {sdr, su, sv, sT};
  for (int f = 0; f < nf; ++f) res_load<R, TXR, TYR, NT>(sf[f], a.buf[a.cur][f], x0, y0, nx, ny, false);
  for (int q = threadIdx.x; q < NO; q += NT) {
    const int ly = q / TXR, lx = q - ly * TXR, i = x0 + lx, j = y0 + ly;
    sinv[q] = (i < nx && j < ny) ? R(1) / (R(1) + alpha_of(c, __ldg(a.gamma + (size_t)j * nx + i))) : R(0);
  }
  if (TH)
    for (int q = threadIdx.x; q < A1; q += NT) {
      const int ly = q / LX1, lx = q - ly * LX1, i = x0 - 1 + lx, j = y0 - 1 + ly;
      cB[q] = (i >= 0 && i < nx && j >= 0 && j < ny) ? B_of(c, __ldg(a.gamma + (size_t)j * nx + i)) : R(0);
    }
  __syncthreads();

  // Push values of halo-1 node (lx, ly): f_k^eq towards x + c_k as an increment on
  // the destination's density (and temperature).
  auto coef = [&](int lx, int ly) {
    const int q = ly * LX1 + lx;
    const int i = x0 - 1 + lx, j = y0 - 1 + ly;
    if (i < 0 || i >= nx || j < 0 || j >= ny) {
#pragma unroll
      for (int k = 0; k < 9; ++k) {
        F[k * A1 + q] = R(0);
        if (TH) G[k * A1 + q] = R(0);
      }
      return;
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
    const R e0 = -R(1.5) * (uu * uu + vv * vv);
    const R bx = R(3) * uu, by = R(3) * vv;
    const R qxx = R(4.5) * uu * uu + c.A * (R(2) * dudx);
    const R qyy = R(4.5) * vv * vv + c.A * (R(2) * dvdy);
    const R qxy = R(9) * uu * vv + R(2) * c.A * (dudy + dvdx);
    const R dr = sdr[s2];
    F[q] = e0 * (R(4) / R(9));
    F[1 * A1 + q] = ((dr - sdr[s2 + 1]) + e0 + bx + qxx) * (R(1) / R(9));
    F[3 * A1 + q] = ((dr - sdr[s2 - 1]) + e0 - bx + qxx) * (R(1) / R(9));
    F[2 * A1 + q] = ((dr - sdr[s2 + LX2]) + e0 + by + qyy) * (R(1) / R(9));
    F[4 * A1 + q] = ((dr - sdr[s2 - LX2]) + e0 - by + qyy) * (R(1) / R(9));
    const R d0 = e0 + qxx + qyy;
    F[5 * A1 + q] = (((dr - sdr[s2 + LX2 + 1]) + d0) + bx + by + qxy) * (R(1) / R(36));
    F[6 * A1 + q] = (((dr - sdr[s2 + LX2 - 1]) + d0) - bx + by - qxy) * (R(1) / R(36));
    F[7 * A1 + q] = (((dr - sdr[s2 - LX2 - 1]) + d0) - bx - by + qxy) * (R(1) / R(36));
    F[8 * A1 + q] = (((dr - sdr[s2 - LX2 + 1]) + d0) + bx - by - qxy) * (R(1) / R(36));
    if (TH) {
      const R TT = sT[s2];
      const R tx_ = R(3) * TT * uu + cB[q] * dfdx<R, LX2>(sT, sx, sy, i, nx);
      const R ty_ = R(3) * TT * vv + cB[q] * dfdy<R, LX2>(sT, sx, sy, j, ny);
      G[q] = R(0);
      G[1 * A1 + q] = ((TT - sT[s2 + 1]) + tx_) * (R(1) / R(9));
      G[3 * A1 + q] = ((TT - sT[s2 - 1]) - tx_) * (R(1) / R(9));
      G[2 * A1 + q] = ((TT - sT[s2 + LX2]) + ty_) * (R(1) / R(9));
      G[4 * A1 + q] = ((TT - sT[s2 - LX2]) - ty_) * (R(1) / R(9));
      G[5 * A1 + q] = ((TT - sT[s2 + LX2 + 1]) + tx_ + ty_) * (R(1) / R(36));
      G[6 * A1 + q] = ((TT - sT[s2 + LX2 - 1]) - tx_ + ty_) * (R(1) / R(36));
      G[7 * A1 + q] = ((TT - sT[s2 - LX2 - 1]) - tx_ - ty_) * (R(1) / R(36));
      G[8 * A1 + q] = ((TT - sT[s2 - LX2 + 1]) + tx_ - ty_) * (R(1) / R(36));
    }
  };

  // Output of tile node (ox, oy) into o[0..3].
  auto node = [&](int ox, int oy, R* o) {
    const int i = x0 + ox, j = y0 + oy;
    o[0] = o[1] = o[2] = o[3] = R(0);
    if (i >= nx || j >= ny) return;
    const int q = (oy + 1) * LX1 + (ox + 1);
    const int s2 = (oy + 2) * LX2 + (ox + 2);
    int nxo, nyo;
    const int cls = node_class(g, i, j, nxo, nyo);
    const R drx = sdr[s2];
    // f_k arriving at x comes from x - c_k
    R fk[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) fk[k] = F[k * A1 + q - cxk(k) - cyk(k) * LX1];
    R drn, un, vn, Tn = R(0);
    if (cls == C_INTERIOR) {
      drn = drx + (((fk[0] + fk[1]) + (fk[2] + fk[3])) + ((fk[4] + fk[5]) + (fk[6] + fk[7])) + fk[8]);
      const R inv = sinv[oy * TXR + ox];
      un = (fk[1] - fk[3] + fk[5] - fk[6] - fk[7] + fk[8]) * inv;
      vn = (fk[2] - fk[4] + fk[5] + fk[6] - fk[7] - fk[8]) * inv;
      if (TH) {
        R gs = R(0);
#pragma unroll
        for (int k = 1; k < 9; ++k) gs += G[k * A1 + q - cxk(k) - cyk(k) * LX1];
        Tn = sT[s2] + gs;
      }
    } else {
      R s0 = R(0), sp = R(0), g0 = R(0), gp = R(0);
#pragma unroll
      for (int k = 0; k < 9; ++k) {
        const int cx = cxk(k), cy = cyk(k);
        const int si = i - cx, sj = j - cy;
        if (si < 0 || si >= nx || sj < 0 || sj >= ny) continue;
        const int cn = cx * nxo + cy * nyo;
        if (cn == 0) s0 += fk[k];
        else if (cn > 0) sp += fk[k];
        if (TH) {
          const R gk = G[k * A1 + q - cx - cy * LX1];
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
          Tn = sT[(jn - y0 + 2) * LX2 + (ox + 2)];
        } else {
          Tn = (sT[s2] + g0 + R(2) * gp + flux_value(g, c, e, i)) / (R(1) + un * R(nxo) + vn * R(nyo));
        }
      }
    }
    o[0] = drn;
    o[1] = un;
    o[2] = vn;
    o[3] = Tn;
    if (bad_velocity(un, vn)) raise_status(a.status, 4);
  };

  auto inner_pos = [&](int t, int& ox, int& oy) {
    oy = 2 + t / (TXR - 4);
    ox = 2 + t - (oy - 2) * (TXR - 4);
  };
  auto outer_pos = [&](int t, int& ox, int& oy) {  // the band of width 2 around the inner block
    if (t < 2 * TXR) {
      oy = t / TXR;                   // rows 0, 1
      ox = t - oy * TXR;
    } else if (t < 4 * TXR) {
      const int u = t - 2 * TXR;
      oy = TYR - 2 + u / TXR;         // rows TYR-2, TYR-1
      ox = u - (u / TXR) * TXR;
    } else {
      const int u = t - 4 * TXR, r = u / 4, cidx = u - r * 4;
      oy = 2 + r;                      // rows 2 .. TYR-3, columns 0, 1, TXR-2, TXR-1
      ox = cidx < 2 ? cidx : TXR - 4 + cidx;
    }
  };

  R oi[PI][4], oo[PO][4];
  for (int s = 0; s < a.n_steps; ++s) {
    // (1) inner push values and inner outputs: own data only
    for (int t = threadIdx.x; t < (TXR - 2) * (TYR - 2); t += NT) {
      const int ly = 2 + t / (TXR - 2), lx = 2 + t - (ly - 2) * (TXR - 2);
      coef(lx, ly);
    }
    __syncthreads();
#pragma unroll
    for (int p = 0; p < PI; ++p) {
      const int t = threadIdx.x + p * NT;
      if (t < NOI) {
        int ox, oy;
        inner_pos(t, ox, oy);
        node(ox, oy, oi[p]);
      }
    }
    // (2) halo of this level from the neighbours
    if (s > 0) {
      if (!res_wait(a.flags, tx, ty, a.ntx, nty, s, a.status, &s_abort)) return;
      const int pb = (a.cur + s) & 1;
      res_load_ring<R, TXR, TYR, NT, TH ? 4 : 3>(sf, a.buf[pb], nf, x0, y0, nx, ny);
      __syncthreads();
    }
    // (3) outer push values and the tile band
    for (int t = threadIdx.x; t < 4 * (LX1 + TYR - 2); t += NT) {
      int lx, ly;
      band_coef_pos<TXR, TYR>(t, lx, ly);
      coef(lx, ly);
    }
    __syncthreads();
#pragma unroll
    for (int p = 0; p < PO; ++p) {
      const int t = threadIdx.x + p * NT;
      if (t < NOO) {
        int ox, oy;
        outer_pos(t, ox, oy);
        node(ox, oy, oo[p]);
      }
    }
    __syncthreads();  // every read of this level is done
    // (4) the band (what the neighbours read) to shared and global memory, publish;
    // then the interior to shared memory (to global memory after the last step)
    const int nb = (a.cur + s + 1) & 1;
    const bool last = s == a.n_steps - 1;
    auto put = [&](int ox, int oy, const R* o, bool global) {
      const int i = x0 + ox, j = y0 + oy;
      if (i >= nx || j >= ny) return;
      const int s2 = (oy + 2) * LX2 + (ox + 2);
      const size_t off = (size_t)j * nx + i;
      for (int f = 0; f < nf; ++f) {
        sf[f][s2] = o[f];
        if (global) __stcg(a.buf[nb][f] + off, o[f]);
      }
    };
#pragma unroll
    for (int p = 0; p < PO; ++p) {
      const int t = threadIdx.x + p * NT;
      if (t < NOO) {
        int ox, oy;
        outer_pos(t, ox, oy);
        put(ox, oy, oo[p], true);
      }
    }
    res_publish(a.flags, tile, s + 1);
#pragma unroll
    for (int p = 0; p < PI; ++p) {
      const int t = threadIdx.x + p * NT;
      if (t < NOI) {
        int ox, oy;
        inner_pos(t, ox, oy);
        put(ox, oy, oi[p], last);
      }
    }
    __syncthreads();
  }
}

template <int TXR, int TYR>
constexpr int adj_res_smem_elems() {
  return 8 * (TXR + 4) * (TYR + 4) + 9 * (TXR + 2) * (TYR + 2) + 3 * TXR * TYR;
}

// ---------------------------------------------------------------------------------
// Steady ALKS march, resident form (non-thermal).  Buffers hold the six adjoint
// moments; the state (u, v) is frozen.
// ---------------------------------------------------------------------------------
template <typename R, int TXR, int TYR, int NT>
__global__ void __launch_bounds__(NT, 1) adj_resident_kernel(ResArgs<R> a, Geom g, Coef<R> c) {
  constexpr int LX2 = TXR + 4, LY2 = TYR + 4, LX1 = TXR + 2, LY1 = TYR + 2;
  constexpr int A2 = LX2 * LY2, A1 = LX1 * LY1, NO = TXR * TYR;
  constexpr int NOI = (TXR - 4) * (TYR - 4), NOO = NO - NOI;
  constexpr int PI = (NOI + NT - 1) / NT, PO = (NOO + NT - 1) / NT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R* sm = reinterpret_cast<R*>(smem_raw);
  R* sa[6];
  for (int f = 0; f < 6; ++f) sa[f] = sm + f * A2;
  R* su = sm + 6 * A2;
  R* sv = su + A2;
  R* Pq = sv + A2;            // push values P + c_k . V towards x - c_k, 9 x A1
  R* sju = Pq + 9 * A1;       // objective source dJ_O/du, dJ_O/dv on the tile
  R* sjv = sju + NO;
  R* sinv = sjv + NO;
  __shared__ int s_abort;

  if (a.status && *reinterpret_cast<const volatile int*>(a.status) == 6) return;  // earlier timeout
  const int nx = g.nx, ny = g.ny;
  const int tile = blockIdx.x, tx = tile % a.ntx, ty = tile / a.ntx;
  const int nty = gridDim.x / a.ntx;
  const int x0 = tx * TXR, y0 = ty * TYR;
  if (threadIdx.x == 0) s_abort = 0;
  for (int f = 0; f < 6; ++f) res_load<R, TXR, TYR, NT>(sa[f], a.buf[a.cur][f], x0, y0, nx, ny, false);
  res_load<R, TXR, TYR, NT>(su, a.u, x0, y0, nx, ny, false);
  res_load<R, TXR, TYR, NT>(sv, a.v, x0, y0, nx, ny, false);
  __syncthreads();
  // Strain of the frozen state on interior nodes (staged in the push array), then
  // the objective source and 1/(1 + alpha) of every tile node.
  R* cSxx = Pq;
  R* cSxy = Pq + A1;
  R* cSyy = Pq + 2 * A1;
  for (int q = threadIdx.x; q < A1; q += NT) {
    const int ly = q / LX1, lx = q - ly * LX1;
    const int i = x0 - 1 + lx, j = y0 - 1 + ly;
    R Sxx = R(0), Sxy = R(0), Syy = R(0);
    if (i > 0 && j > 0 && i < nx - 1 && j < ny - 1) {
      const int s2 = (ly + 1) * LX2 + lx + 1;
      Sxx = R(2) * ((su[s2 + 1] - su[s2 - 1]) * R(0.5));
      Syy = R(2) * ((sv[s2 + LX2] - sv[s2 - LX2]) * R(0.5));
      Sxy = (su[s2 + LX2] - su[s2 - LX2]) * R(0.5) + (sv[s2 + 1] - sv[s2 - 1]) * R(0.5);
    }
    cSxx[q] = Sxx;
    cSxy[q] = Sxy;
    cSyy[q] = Syy;
  }
  __syncthreads();
  for (int q = threadIdx.x; q < NO; q += NT) {
    const int oy = q / TXR, ox = q - oy * TXR, i = x0 + ox, j = y0 + oy;
    R ju = R(0), jv = R(0), inv = R(0);
    if (i < nx && j < ny) {
      const int q1 = (oy + 1) * LX1 + ox + 1, s2 = (oy + 2) * LX2 + ox + 2;
      const R al = alpha_of(c, __ldg(a.gamma + (size_t)j * nx + i));
      ju = c.nu * (cSxx[q1 - 1] - cSxx[q1 + 1] + cSxy[q1 - LX1] - cSxy[q1 + LX1]) + R(2) * al * su[s2];
      jv = c.nu * (cSyy[q1 - LX1] - cSyy[q1 + LX1] + cSxy[q1 - 1] - cSxy[q1 + 1]) + R(2) * al * sv[s2];
      inv = R(1) / (R(1) + al);
    }
    sju[q] = ju;
    sjv[q] = jv;
    sinv[q] = inv;
  }
  __syncthreads();

  // Push values of halo-1 node (lx, ly): f~_k(x) = P(y) + c_k . V(y) for x = y - c_k.
  auto coef = [&](int lx, int ly) {
    const int q = ly * LX1 + lx;
    const int i = x0 - 1 + lx, j = y0 - 1 + ly;
    if (i < 0 || i >= nx || j < 0 || j >= ny) {
#pragma unroll
      for (int k = 0; k < 9; ++k) Pq[k * A1 + q] = R(0);
      return;
    }
    const int sx = lx + 1, sy = ly + 1, s2 = sy * LX2 + sx;
    const R rt = sa[0][s2], ux = sa[1][s2], uy = sa[2][s2];
    const R sxx = sa[3][s2], sxy = sa[4][s2], syy = sa[5][s2];
    const R uu = su[s2], vv = sv[s2];
    const R Dx = R(2) * (dfdx<R, LX2>(sa[3], sx, sy, i, nx) + dfdy<R, LX2>(sa[4], sx, sy, j, ny));
    const R Dy = R(2) * (dfdx<R, LX2>(sa[4], sx, sy, i, nx) + dfdy<R, LX2>(sa[5], sx, sy, j, ny));
    const R P = rt;
    const R Vx = R(3) * (ux + R(3) * (sxx * uu + sxy * vv) - rt * uu) - c.A * Dx;
    const R Vy = R(3) * (uy + R(3) * (sxy * uu + syy * vv) - rt * vv) - c.A * Dy;
#pragma unroll
    for (int k = 0; k < 9; ++k) Pq[k * A1 + q] = P + R(cxk(k)) * Vx + R(cyk(k)) * Vy;
  };

  auto node = [&](int ox, int oy, R* o) {
    const int i = x0 + ox, j = y0 + oy;
#pragma unroll
    for (int f = 0; f < 6; ++f) o[f] = R(0);
    if (i >= nx || j >= ny) return;
    const int q = (oy + 1) * LX1 + (ox + 1);
    const bool interior = i > 0 && j > 0 && i < nx - 1 && j < ny - 1;
    R ft[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) ft[k] = Pq[k * A1 + q + cxk(k) + cyk(k) * LX1];
    if (interior) {
      const R w0 = R(4) / R(9), w1 = R(1) / R(9), w5 = R(1) / R(36);
      const R ax = ft[1] + ft[3], ay = ft[2] + ft[4], dg = ft[5] + ft[6] + ft[7] + ft[8];
      o[0] = w0 * ft[0] + w1 * (ax + ay) + w5 * dg;
      const R m1 = w1 * (ft[1] - ft[3]) + w5 * (ft[5] - ft[6] - ft[7] + ft[8]);
      const R m2 = w1 * (ft[2] - ft[4]) + w5 * (ft[5] + ft[6] - ft[7] - ft[8]);
      o[3] = w1 * ax + w5 * dg;
      o[4] = w5 * (ft[5] - ft[6] + ft[7] - ft[8]);
      o[5] = w1 * ay + w5 * dg;
      const int qt = oy * TXR + ox;
      const R inv = sinv[qt];
      o[1] = (m1 - sju[qt] * (R(1) / R(3))) * inv;
      o[2] = (m2 - sjv[qt] * (R(1) / R(3))) * inv;
    } else {
#pragma unroll
      for (int k = 0; k < 9; ++k) {
        const int gi = i + cxk(k), gj = j + cyk(k);
        if (gi < 0 || gi >= nx || gj < 0 || gj >= ny) ft[k] = R(0);
      }
      const int ec = edge_class(g, i, j);
      const R* M = a.emap + ec * 60;
      const R jb = edge_objective_term(g, c, ec, j);  // the static pressure drop
#pragma unroll
      for (int r = 0; r < 6; ++r) {
        R acc = R(0);
#pragma unroll
        for (int k = 0; k < 9; ++k) acc += M[r * 10 + k] * ft[k];
        if (jb != R(0)) acc += jb * a.emap[540 + ec * 6 + r];
        o[r] = acc;
      }
    }
    if (!(o[1] * o[1] + o[2] * o[2] < R(1e30))) raise_status(a.status, 4);
  };

  auto inner_pos = [&](int t, int& ox, int& oy) {
    oy = 2 + t / (TXR - 4);
    ox = 2 + t - (oy - 2) * (TXR - 4);
  };
  auto outer_pos = [&](int t, int& ox, int& oy) {
    if (t < 2 * TXR) {
      oy = t / TXR;
      ox = t - oy * TXR;
    } else if (t < 4 * TXR) {
      const int u = t - 2 * TXR;
      oy = TYR - 2 + u / TXR;
      ox = u - (u / TXR) * TXR;
    } else {
      const int u = t - 4 * TXR, r = u / 4, cidx = u - r * 4;
      oy = 2 + r;
      ox = cidx < 2 ? cidx : TXR - 4 + cidx;
    }
  };

  R oi[PI][6], oo[PO][6];
  for (int s = 0; s < a.n_steps; ++s) {
    for (int t = threadIdx.x; t < (TXR - 2) * (TYR - 2); t += NT) {
      const int ly = 2 + t / (TXR - 2), lx = 2 + t - (ly - 2) * (TXR - 2);
      coef(lx, ly);
    }
    __syncthreads();
#pragma unroll
    for (int p = 0; p < PI; ++p) {
      const int t = threadIdx.x + p * NT;
      if (t < NOI) {
        int ox, oy;
        inner_pos(t, ox, oy);
        node(ox, oy, oi[p]);
      }
    }
    if (s > 0) {
      if (!res_wait(a.flags, tx, ty, a.ntx, nty, s, a.status, &s_abort)) return;
      const int pb = (a.cur + s) & 1;
      res_load_ring<R, TXR, TYR, NT, 6>(sa, a.buf[pb], 6, x0, y0, nx, ny);
      __syncthreads();
    }
    for (int t = threadIdx.x; t < 4 * (LX1 + TYR - 2); t += NT) {
      int lx, ly;
      band_coef_pos<TXR, TYR>(t, lx, ly);
      coef(lx, ly);
    }
    __syncthreads();
#pragma unroll
    for (int p = 0; p < PO; ++p) {
      const int t = threadIdx.x + p * NT;
      if (t < NOO) {
        int ox, oy;
        outer_pos(t, ox, oy);
        node(ox, oy, oo[p]);
      }
    }
    __syncthreads();
    const int nb = (a.cur + s + 1) & 1;
    const bool last = s == a.n_steps - 1;
    auto put = [&](int ox, int oy, const R* o, bool global) {
      const int i = x0 + ox, j = y0 + oy;
      if (i >= nx || j >= ny) return;
      const int s2 = (oy + 2) * LX2 + (ox + 2);
      const size_t off = (size_t)j * nx + i;
#pragma unroll
      for (int f = 0; f < 6; ++f) {
        sa[f][s2] = o[f];
        if (global) __stcg(a.buf[nb][f] + off, o[f]);
      }
    };
#pragma unroll
    for (int p = 0; p < PO; ++p) {
      const int t = threadIdx.x + p * NT;
      if (t < NOO) {
        int ox, oy;
        outer_pos(t, ox, oy);
        put(ox, oy, oo[p], true);
      }
    }
    res_publish(a.flags, tile, s + 1);
#pragma unroll
    for (int p = 0; p < PI; ++p) {
      const int t = threadIdx.x + p * NT;
      if (t < NOI) {
        int ox, oy;
        inner_pos(t, ox, oy);
        put(ox, oy, oi[p], last);
      }
    }
    __syncthreads();
  }
}

}  // namespace lks
