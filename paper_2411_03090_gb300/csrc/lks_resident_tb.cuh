// lks_resident_tb.cuh -- resident steady marches that advance KS time steps per
// exchange of tile bands (temporal blocking).
//
// Same scheme and per-node arithmetic as the resident marches of lks_resident.cuh,
// but each CTA stages its tile with a halo of H = 2 KS nodes.  One LKS or ALKS step
// needs the previous level within two nodes of an output (the push values are
// evaluated one node out, their gradients one node further), so after one exchange
// the CTA advances KS steps: sub-step m computes the outputs within
// 2 (KS - 1 - m) nodes of the tile from the values the previous sub-step left in
// shared memory.  Only the last sub-step's band (the H outer rows and columns of the
// tile, which the neighbours read) goes to global memory, followed by one flag
// release per exchange.  The neighbour handshake (global store, release, acquire
// poll, ring load: several L2 round trips) is paid once every KS steps, at the price
// of the redundant halo work of the earlier sub-steps.
//
// Exchange x (x = 1, 2, ...) writes its band to buffer (cur + x) & 1; the host
// records (cur + number of exchanges) & 1 as the buffer of the final level.  A CTA
// overwrites a buffer two exchanges after it was written, and only after every
// neighbour has published the exchange in between, i.e. finished reading it.
#pragma once
#include "lks_resident.cuh"

namespace lks {

template <int TXR, int TYR, int KS>
struct TbGeo {
  static constexpr int H = 2 * KS;   // halo of the staged fields
  static constexpr int HC = H - 1;   // halo of the push values of the first sub-step
  static constexpr int HO = H - 2;   // halo of the outputs of the first sub-step
  static constexpr int LXH = TXR + 2 * H, LYH = TYR + 2 * H, AH = LXH * LYH;
  static constexpr int LXC = TXR + 2 * HC, LYC = TYR + 2 * HC, AC = LXC * LYC;
  static constexpr int LXO = TXR + 2 * HO, LYO = TYR + 2 * HO, AO = LXO * LYO;
  static constexpr int NRING = 2 * H * (LXH + TYR);  // halo positions outside the tile
  static_assert(TXR >= 2 * H && TYR >= 2 * H, "the band of width H must fit the tile twice");
};

template <bool TH, int TXR, int TYR, int KS>
constexpr int fwd_tb_smem_elems() {
  using G = TbGeo<TXR, TYR, KS>;
  return (TH ? 4 : 3) * G::AH + (TH ? 19 : 9) * G::AC + G::AO;
}
template <int TXR, int TYR, int KS>
constexpr int adj_tb_smem_elems() {
  using G = TbGeo<TXR, TYR, KS>;
  return 8 * G::AH + 9 * G::AC + 3 * G::AO;
}

// Halo ring (positions of the halo-H region outside the tile) of nf fields from a
// global buffer; every load is issued before the first shared-memory store.
template <typename R, int TXR, int TYR, int KS, int NT, int NF>
__device__ __forceinline__ void tb_load_ring(R* const* s, R* const* gsrc, int x0, int y0, int nx, int ny) {
  using G = TbGeo<TXR, TYR, KS>;
  constexpr int H = G::H, LXH = G::LXH, NROW = 2 * H * LXH, NR = G::NRING;
  constexpr int PER = (NR + NT - 1) / NT;
  R v[PER][NF];
  int pos[PER];
#pragma unroll
  for (int p = 0; p < PER; ++p) {
    const int q = threadIdx.x + p * NT;
    pos[p] = -1;
    if (q >= NR) continue;
    int lx, ly;
    if (q < NROW) {  // H rows below and H rows above the tile, full width
      const int r = q / LXH;
      lx = q - r * LXH;
      ly = r < H ? r : TYR + r;
    } else {         // H columns left and right of the tile
      const int t = q - NROW, cc = t / TYR;
      ly = H + (t - cc * TYR);
      lx = cc < H ? cc : TXR + cc;
    }
    const int i = x0 - H + lx, j = y0 - H + ly;
    pos[p] = ly * LXH + lx;
    const bool in = i >= 0 && i < nx && j >= 0 && j < ny;
    const size_t off = in ? (size_t)j * nx + i : 0;
#pragma unroll
    for (int f = 0; f < NF; ++f) v[p][f] = in ? __ldcg(gsrc[f] + off) : R(0);
  }
#pragma unroll
  for (int p = 0; p < PER; ++p) {
    if (pos[p] < 0) continue;
#pragma unroll
    for (int f = 0; f < NF; ++f) s[f][pos[p]] = v[p][f];
  }
}

// Is tile position (ox, oy) in the band of width H that the neighbours read?
template <int TXR, int TYR, int H>
__device__ __forceinline__ bool tb_in_band(int ox, int oy) {
  return ox < H || oy < H || ox >= TXR - H || oy >= TYR - H;
}

// ---------------------------------------------------------------------------------
// Steady LKS march (state drho, u, v[, T]), KS steps per exchange.
// ---------------------------------------------------------------------------------
template <typename R, bool TH, int TXR, int TYR, int NT, int KS>
__global__ void __launch_bounds__(NT, 1) fwd_resident_tb_kernel(ResArgs<R> a, Geom g, Coef<R> c) {
  using GT = TbGeo<TXR, TYR, KS>;
  constexpr int H = GT::H, HC = GT::HC, HO = GT::HO;
  constexpr int LXH = GT::LXH, LXC = GT::LXC, LXO = GT::LXO;
  constexpr int AH = GT::AH, AC = GT::AC, AO = GT::AO;
  constexpr int NF = TH ? 4 : 3;
  constexpr int PE = (AO + NT - 1) / NT;  // outputs per thread in the widest sub-step
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R* sm = reinterpret_cast<R*>(smem_raw);
  R* sf[NF];
#pragma unroll
  for (int f = 0; f < NF; ++f) sf[f] = sm + f * AH;
  R* const sdr = sf[0];
  R* const su = sf[1];
  R* const sv = sf[2];
  R* const sT = sf[TH ? 3 : 0];      // thermal only
  R* F = sm + NF * AH;               // push values f_k^eq, 9 x AC
  R* Gp = F + 9 * AC;                // thermal push values g_k^eq, 9 x AC
  R* cB = Gp + (TH ? 9 * AC : 0);    // thermal: B on the push region
  R* sinv = cB + (TH ? AC : 0);      // 1 / (1 + alpha) on the output region
  __shared__ int s_abort;

  if (a.status && *reinterpret_cast<const volatile int*>(a.status) == 6) return;  // earlier timeout
  const int nx = g.nx, ny = g.ny;
  const int tile = blockIdx.x, tx = tile % a.ntx, ty = tile / a.ntx;
  const int nty = gridDim.x / a.ntx;
  const int x0 = tx * TXR, y0 = ty * TYR;
  auto in_lat = [&](int i, int j) { return i >= 0 && i < nx && j >= 0 && j < ny; };
  auto sidx = [&](int i, int j) { return (j - y0 + H) * LXH + (i - x0 + H); };
  auto cidx = [&](int i, int j) { return (j - y0 + HC) * LXC + (i - x0 + HC); };
  auto oidx = [&](int i, int j) { return (j - y0 + HO) * LXO + (i - x0 + HO); };
  if (threadIdx.x == 0) s_abort = 0;
  for (int q = threadIdx.x; q < AH; q += NT) {
    const int ly = q / LXH, lx = q - ly * LXH, i = x0 - H + lx, j = y0 - H + ly;
    const bool in = in_lat(i, j);
    const size_t off = in ? (size_t)j * nx + i : 0;
#pragma unroll
    for (int f = 0; f < NF; ++f) sf[f][q] = in ? __ldcg(a.buf[a.cur][f] + off) : R(0);
  }
  for (int q = threadIdx.x; q < AO; q += NT) {
    const int ly = q / LXO, lx = q - ly * LXO, i = x0 - HO + lx, j = y0 - HO + ly;
    sinv[q] = in_lat(i, j) ? R(1) / (R(1) + alpha_of(c, __ldg(a.gamma + (size_t)j * nx + i))) : R(0);
  }
  if (TH)
    for (int q = threadIdx.x; q < AC; q += NT) {
      const int ly = q / LXC, lx = q - ly * LXC, i = x0 - HC + lx, j = y0 - HC + ly;
      cB[q] = in_lat(i, j) ? B_of(c, __ldg(a.gamma + (size_t)j * nx + i)) : R(0);
    }
  __syncthreads();

  // Push values of node (i, j): f_k^eq towards x + c_k as an increment on the
  // destination's density (and temperature).
  auto coef = [&](int i, int j) {
    const int q = cidx(i, j);
    if (!in_lat(i, j)) {
#pragma unroll
      for (int k = 0; k < 9; ++k) {
        F[k * AC + q] = R(0);
        if (TH) Gp[k * AC + q] = R(0);
      }
      return;
    }
    const int sx = i - x0 + H, sy = j - y0 + H, s2 = sy * LXH + sx;
    const R uu = su[s2], vv = sv[s2];
    R dudx = dfdx<R, LXH>(su, sx, sy, i, nx);
    const R dudy = dfdy<R, LXH>(su, sx, sy, j, ny);
    const R dvdx = dfdx<R, LXH>(sv, sx, sy, i, nx);
    R dvdy = dfdy<R, LXH>(sv, sx, sy, j, ny);
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
    F[1 * AC + q] = ((dr - sdr[s2 + 1]) + e0 + bx + qxx) * (R(1) / R(9));
    F[3 * AC + q] = ((dr - sdr[s2 - 1]) + e0 - bx + qxx) * (R(1) / R(9));
    F[2 * AC + q] = ((dr - sdr[s2 + LXH]) + e0 + by + qyy) * (R(1) / R(9));
    F[4 * AC + q] = ((dr - sdr[s2 - LXH]) + e0 - by + qyy) * (R(1) / R(9));
    const R d0 = e0 + qxx + qyy;
    F[5 * AC + q] = (((dr - sdr[s2 + LXH + 1]) + d0) + bx + by + qxy) * (R(1) / R(36));
    F[6 * AC + q] = (((dr - sdr[s2 + LXH - 1]) + d0) - bx + by - qxy) * (R(1) / R(36));
    F[7 * AC + q] = (((dr - sdr[s2 - LXH - 1]) + d0) - bx - by + qxy) * (R(1) / R(36));
    F[8 * AC + q] = (((dr - sdr[s2 - LXH + 1]) + d0) + bx - by - qxy) * (R(1) / R(36));
    if (TH) {
      const R TT = sT[s2];
      const R tx_ = R(3) * TT * uu + cB[q] * dfdx<R, LXH>(sT, sx, sy, i, nx);
      const R ty_ = R(3) * TT * vv + cB[q] * dfdy<R, LXH>(sT, sx, sy, j, ny);
      Gp[q] = R(0);
      Gp[1 * AC + q] = ((TT - sT[s2 + 1]) + tx_) * (R(1) / R(9));
      Gp[3 * AC + q] = ((TT - sT[s2 - 1]) - tx_) * (R(1) / R(9));
      Gp[2 * AC + q] = ((TT - sT[s2 + LXH]) + ty_) * (R(1) / R(9));
      Gp[4 * AC + q] = ((TT - sT[s2 - LXH]) - ty_) * (R(1) / R(9));
      Gp[5 * AC + q] = ((TT - sT[s2 + LXH + 1]) + tx_ + ty_) * (R(1) / R(36));
      Gp[6 * AC + q] = ((TT - sT[s2 + LXH - 1]) - tx_ + ty_) * (R(1) / R(36));
      Gp[7 * AC + q] = ((TT - sT[s2 - LXH - 1]) - tx_ - ty_) * (R(1) / R(36));
      Gp[8 * AC + q] = ((TT - sT[s2 - LXH + 1]) + tx_ - ty_) * (R(1) / R(36));
    }
  };

  // New level at node (i, j) (inside the lattice) into o[0..NF).
  auto node = [&](int i, int j, R* o) {
    const int q = cidx(i, j), s2 = sidx(i, j);
    int nxo, nyo;
    const int cls = node_class(g, i, j, nxo, nyo);
    const R drx = sdr[s2];
    R fk[9];  // f_k arriving at x comes from x - c_k
#pragma unroll
    for (int k = 0; k < 9; ++k) fk[k] = F[k * AC + q - cxk(k) - cyk(k) * LXC];
    R drn, un, vn, Tn = R(0);
    if (cls == C_INTERIOR) {
      drn = drx + (((fk[0] + fk[1]) + (fk[2] + fk[3])) + ((fk[4] + fk[5]) + (fk[6] + fk[7])) + fk[8]);
      const R inv = sinv[oidx(i, j)];
      un = (fk[1] - fk[3] + fk[5] - fk[6] - fk[7] + fk[8]) * inv;
      vn = (fk[2] - fk[4] + fk[5] + fk[6] - fk[7] - fk[8]) * inv;
      if (TH) {
        R gs = R(0);
#pragma unroll
        for (int k = 1; k < 9; ++k) gs += Gp[k * AC + q - cxk(k) - cyk(k) * LXC];
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
          const R gk = Gp[k * AC + q - cx - cy * LXC];
          if (cn == 0) g0 += gk;
          else if (cn > 0) gp += gk;
        }
      }
      if (cls == C_CORNER) {
        drn = sdr[sidx(i, (j == 0) ? 1 : ny - 2)];
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
          Tn = sT[sidx(i, (j == 0) ? 1 : ny - 2)];
        } else {
          Tn = (sT[s2] + g0 + R(2) * gp + flux_value(g, c, e, i)) / (R(1) + un * R(nxo) + vn * R(nyo));
        }
      }
    }
    o[0] = drn;
    o[1] = un;
    o[2] = vn;
    if (TH) o[3] = Tn;
    if (bad_velocity(un, vn)) raise_status(a.status, 4);
  };

  const int nex = (a.n_steps + KS - 1) / KS;
  R o[PE][NF];
  for (int x = 1; x <= nex; ++x) {
    if (x > 1) {  // the ring of this level from the neighbours
      if (!res_wait(a.flags, tx, ty, a.ntx, nty, x - 1, a.status, &s_abort)) return;
      R* src[NF];
#pragma unroll
      for (int f = 0; f < NF; ++f) src[f] = a.buf[(a.cur + x - 1) & 1][f];
      tb_load_ring<R, TXR, TYR, KS, NT, NF>(sf, src, x0, y0, nx, ny);
      __syncthreads();
    }
    const int ns = min(KS, a.n_steps - (x - 1) * KS);
    const bool last_x = x == nex;
    R* dst[NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) dst[f] = a.buf[(a.cur + x) & 1][f];
    for (int m = 0; m < ns; ++m) {
      const int e = 2 * (ns - 1 - m);  // output halo of this sub-step
      const int wc = TXR + 2 * (e + 1), nc = wc * (TYR + 2 * (e + 1));
      for (int t = threadIdx.x; t < nc; t += NT) {
        const int ly = t / wc, lx = t - ly * wc;
        coef(x0 - (e + 1) + lx, y0 - (e + 1) + ly);
      }
      __syncthreads();
      const int wo = TXR + 2 * e, no = wo * (TYR + 2 * e);
#pragma unroll
      for (int p = 0; p < PE; ++p) {
        const int t = threadIdx.x + p * NT;
        if (t < no) {
          const int ly = t / wo, lx = t - ly * wo, i = x0 - e + lx, j = y0 - e + ly;
          if (in_lat(i, j)) node(i, j, o[p]);
        }
      }
      __syncthreads();  // every read of this level is done
      const bool final_sub = m == ns - 1;
#pragma unroll
      for (int p = 0; p < PE; ++p) {
        const int t = threadIdx.x + p * NT;
        if (t < no) {
          const int ly = t / wo, lx = t - ly * wo, i = x0 - e + lx, j = y0 - e + ly;
          if (!in_lat(i, j)) continue;
          const int s2 = sidx(i, j);
#pragma unroll
          for (int f = 0; f < NF; ++f) sf[f][s2] = o[p][f];
          if (final_sub && (last_x || tb_in_band<TXR, TYR, H>(lx, ly))) {
            const size_t off = (size_t)j * nx + i;
#pragma unroll
            for (int f = 0; f < NF; ++f) __stcg(dst[f] + off, o[p][f]);
          }
        }
      }
      if (final_sub) res_publish(a.flags, tile, x);  // includes the CTA barrier
      else __syncthreads();
    }
  }
}

// ---------------------------------------------------------------------------------
// Steady ALKS march (six adjoint moments; the state u, v is frozen), KS steps per
// exchange.
// ---------------------------------------------------------------------------------
template <typename R, int TXR, int TYR, int NT, int KS>
__global__ void __launch_bounds__(NT, 1) adj_resident_tb_kernel(ResArgs<R> a, Geom g, Coef<R> c) {
  using GT = TbGeo<TXR, TYR, KS>;
  constexpr int H = GT::H, HC = GT::HC, HO = GT::HO;
  constexpr int LXH = GT::LXH, LXC = GT::LXC, LXO = GT::LXO;
  constexpr int AH = GT::AH, AC = GT::AC, AO = GT::AO;
  constexpr int PE = (AO + NT - 1) / NT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R* sm = reinterpret_cast<R*>(smem_raw);
  R* sa[6];
#pragma unroll
  for (int f = 0; f < 6; ++f) sa[f] = sm + f * AH;
  R* su = sm + 6 * AH;
  R* sv = su + AH;
  R* Pq = sv + AH;       // push values P + c_k . V towards x - c_k, 9 x AC
  R* sju = Pq + 9 * AC;  // objective source dJ_O/du, dJ_O/dv on the output region
  R* sjv = sju + AO;
  R* sinv = sjv + AO;
  __shared__ int s_abort;

  if (a.status && *reinterpret_cast<const volatile int*>(a.status) == 6) return;  // earlier timeout
  const int nx = g.nx, ny = g.ny;
  const int tile = blockIdx.x, tx = tile % a.ntx, ty = tile / a.ntx;
  const int nty = gridDim.x / a.ntx;
  const int x0 = tx * TXR, y0 = ty * TYR;
  auto in_lat = [&](int i, int j) { return i >= 0 && i < nx && j >= 0 && j < ny; };
  auto sidx = [&](int i, int j) { return (j - y0 + H) * LXH + (i - x0 + H); };
  auto cidx = [&](int i, int j) { return (j - y0 + HC) * LXC + (i - x0 + HC); };
  auto oidx = [&](int i, int j) { return (j - y0 + HO) * LXO + (i - x0 + HO); };
  if (threadIdx.x == 0) s_abort = 0;
  for (int q = threadIdx.x; q < AH; q += NT) {
    const int ly = q / LXH, lx = q - ly * LXH, i = x0 - H + lx, j = y0 - H + ly;
    const bool in = in_lat(i, j);
    const size_t off = in ? (size_t)j * nx + i : 0;
#pragma unroll
    for (int f = 0; f < 6; ++f) sa[f][q] = in ? __ldcg(a.buf[a.cur][f] + off) : R(0);
    su[q] = in ? __ldg(a.u + off) : R(0);
    sv[q] = in ? __ldg(a.v + off) : R(0);
  }
  __syncthreads();
  // Strain of the frozen state on interior nodes of the push region (staged in the
  // push array), then the objective source and 1/(1 + alpha) on the output region.
  R* cSxx = Pq;
  R* cSxy = Pq + AC;
  R* cSyy = Pq + 2 * AC;
  for (int q = threadIdx.x; q < AC; q += NT) {
    const int ly = q / LXC, lx = q - ly * LXC, i = x0 - HC + lx, j = y0 - HC + ly;
    R Sxx = R(0), Sxy = R(0), Syy = R(0);
    if (i > 0 && j > 0 && i < nx - 1 && j < ny - 1) {
      const int s2 = sidx(i, j);
      Sxx = R(2) * ((su[s2 + 1] - su[s2 - 1]) * R(0.5));
      Syy = R(2) * ((sv[s2 + LXH] - sv[s2 - LXH]) * R(0.5));
      Sxy = (su[s2 + LXH] - su[s2 - LXH]) * R(0.5) + (sv[s2 + 1] - sv[s2 - 1]) * R(0.5);
    }
    cSxx[q] = Sxx;
    cSxy[q] = Sxy;
    cSyy[q] = Syy;
  }
  __syncthreads();
  for (int q = threadIdx.x; q < AO; q += NT) {
    const int ly = q / LXO, lx = q - ly * LXO, i = x0 - HO + lx, j = y0 - HO + ly;
    R ju = R(0), jv = R(0), inv = R(0);
    if (in_lat(i, j)) {
      const int q1 = cidx(i, j), s2 = sidx(i, j);
      const R al = alpha_of(c, __ldg(a.gamma + (size_t)j * nx + i));
      ju = c.nu * (cSxx[q1 - 1] - cSxx[q1 + 1] + cSxy[q1 - LXC] - cSxy[q1 + LXC]) + R(2) * al * su[s2];
      jv = c.nu * (cSyy[q1 - LXC] - cSyy[q1 + LXC] + cSxy[q1 - 1] - cSxy[q1 + 1]) + R(2) * al * sv[s2];
      inv = R(1) / (R(1) + al);
    }
    sju[q] = ju;
    sjv[q] = jv;
    sinv[q] = inv;
  }
  __syncthreads();

  // Push values of node (i, j): f~_k(x) = P(y) + c_k . V(y) for x = y - c_k.
  auto coef = [&](int i, int j) {
    const int q = cidx(i, j);
    if (!in_lat(i, j)) {
#pragma unroll
      for (int k = 0; k < 9; ++k) Pq[k * AC + q] = R(0);
      return;
    }
    const int sx = i - x0 + H, sy = j - y0 + H, s2 = sy * LXH + sx;
    const R rt = sa[0][s2], ux = sa[1][s2], uy = sa[2][s2];
    const R sxx = sa[3][s2], sxy = sa[4][s2], syy = sa[5][s2];
    const R uu = su[s2], vv = sv[s2];
    const R Dx = R(2) * (dfdx<R, LXH>(sa[3], sx, sy, i, nx) + dfdy<R, LXH>(sa[4], sx, sy, j, ny));
    const R Dy = R(2) * (dfdx<R, LXH>(sa[4], sx, sy, i, nx) + dfdy<R, LXH>(sa[5], sx, sy, j, ny));
    const R P = rt;
    const R Vx = R(3) * (ux + R(3) * (sxx * uu + sxy * vv) - rt * uu) - c.A * Dx;
    const R Vy = R(3) * (uy + R(3) * (sxy * uu + syy * vv) - rt * vv) - c.A * Dy;
#pragma unroll
    for (int k = 0; k < 9; ++k) Pq[k * AC + q] = P + R(cxk(k)) * Vx + R(cyk(k)) * Vy;
  };

  // New adjoint moments at node (i, j) (inside the lattice) into o[0..6).
  auto node = [&](int i, int j, R* o) {
    const int q = cidx(i, j);
    const bool interior = i > 0 && j > 0 && i < nx - 1 && j < ny - 1;
    R ft[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) ft[k] = Pq[k * AC + q + cxk(k) + cyk(k) * LXC];
    if (interior) {
      const R w0 = R(4) / R(9), w1 = R(1) / R(9), w5 = R(1) / R(36);
      const R ax = ft[1] + ft[3], ay = ft[2] + ft[4], dg = ft[5] + ft[6] + ft[7] + ft[8];
      o[0] = w0 * ft[0] + w1 * (ax + ay) + w5 * dg;
      const R m1 = w1 * (ft[1] - ft[3]) + w5 * (ft[5] - ft[6] - ft[7] + ft[8]);
      const R m2 = w1 * (ft[2] - ft[4]) + w5 * (ft[5] + ft[6] - ft[7] - ft[8]);
      o[3] = w1 * ax + w5 * dg;
      o[4] = w5 * (ft[5] - ft[6] + ft[7] - ft[8]);
      o[5] = w1 * ay + w5 * dg;
      const int qo = oidx(i, j);
      const R inv = sinv[qo];
      o[1] = (m1 - sju[qo] * (R(1) / R(3))) * inv;
      o[2] = (m2 - sjv[qo] * (R(1) / R(3))) * inv;
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

  const int nex = (a.n_steps + KS - 1) / KS;
  R o[PE][6];
  for (int x = 1; x <= nex; ++x) {
    if (x > 1) {
      if (!res_wait(a.flags, tx, ty, a.ntx, nty, x - 1, a.status, &s_abort)) return;
      R* src[6];
#pragma unroll
      for (int f = 0; f < 6; ++f) src[f] = a.buf[(a.cur + x - 1) & 1][f];
      tb_load_ring<R, TXR, TYR, KS, NT, 6>(sa, src, x0, y0, nx, ny);
      __syncthreads();
    }
    const int ns = min(KS, a.n_steps - (x - 1) * KS);
    const bool last_x = x == nex;
    R* dst[6];
#pragma unroll
    for (int f = 0; f < 6; ++f) dst[f] = a.buf[(a.cur + x) & 1][f];
    for (int m = 0; m < ns; ++m) {
      const int e = 2 * (ns - 1 - m);
      const int wc = TXR + 2 * (e + 1), nc = wc * (TYR + 2 * (e + 1));
      for (int t = threadIdx.x; t < nc; t += NT) {
        const int ly = t / wc, lx = t - ly * wc;
        coef(x0 - (e + 1) + lx, y0 - (e + 1) + ly);
      }
      __syncthreads();
      const int wo = TXR + 2 * e, no = wo * (TYR + 2 * e);
#pragma unroll
      for (int p = 0; p < PE; ++p) {
        const int t = threadIdx.x + p * NT;
        if (t < no) {
          const int ly = t / wo, lx = t - ly * wo, i = x0 - e + lx, j = y0 - e + ly;
          if (in_lat(i, j)) node(i, j, o[p]);
        }
      }
      __syncthreads();
      const bool final_sub = m == ns - 1;
#pragma unroll
      for (int p = 0; p < PE; ++p) {
        const int t = threadIdx.x + p * NT;
        if (t < no) {
          const int ly = t / wo, lx = t - ly * wo, i = x0 - e + lx, j = y0 - e + ly;
          if (!in_lat(i, j)) continue;
          const int s2 = sidx(i, j);
#pragma unroll
          for (int f = 0; f < 6; ++f) sa[f][s2] = o[p][f];
          if (final_sub && (last_x || tb_in_band<TXR, TYR, H>(lx, ly))) {
            const size_t off = (size_t)j * nx + i;
#pragma unroll
            for (int f = 0; f < 6; ++f) __stcg(dst[f] + off, o[p][f]);
          }
        }
      }
      if (final_sub) res_publish(a.flags, tile, x);
      else __syncthreads();
    }
  }
}

}  // namespace lks
