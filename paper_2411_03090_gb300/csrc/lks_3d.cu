// lks_3d.cu -- the three-dimensional (D3Q19) steady duct path: LKS forward march,
// ALKS adjoint iteration with the generalized-inverse face rules, sensitivity.
//
// The paper (arXiv 2411.03090) states LKS and ALKS in two dimensions (Secs.
// 2.4-2.5, App. A); here every equation is written for 19 velocities:
//   forward   f_k^eq = w_k { rho + 3 c.u + 9/2 (c.u)^2 - 3/2 u^2 + A c_a c_b S_ab }
//             (Eq. feq2), streamed from x - c_k, rho = sum f, u = sum c f / (1+alpha)
//   adjoint   f~_k = P(x + c_k) + c_k . V(x + c_k),  P = rho~,
//             V_a = 3 (u~_a + 3 s~_ab u_b - rho~ u_a) - 2A d_b s~_ab  (Eq. afeq);
//             moments rho~, u~ (implicit Brinkman, objective source), s~
//   faces     Zou-He-type density / normal velocity (inlet velocity, outlet
//             pressure, walls); the adjoint's unknown f~ by least squares over the
//             19 rows (Sec. 2.5, Eq. r_definition), folded into 10 x 19 maps.
//
// Kernel structure (2.5-D march).  Each CTA owns a 32 x 8 column of output nodes
// and marches a chunk of z planes.  Staged planes of the input fields sit in a
// ring in shared memory (a two-node halo in x and y).  The forward step keeps the
// pushed populations of the halo-1 ring grouped by c_z: the five links with
// c_z = +1 are consumed two planes later, the nine with c_z = 0 one plane later,
// the five with c_z = -1 at once, so three, two and one plane of them are kept.
// The adjoint keeps P and V of three planes.  Every node's arithmetic is that of
// the per-node formulas above; there is no blocking of the mathematics itself.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <type_traits>
#include <vector>

#include "lks_3d.cuh"
#include "lks_host.cuh"
#include "lks_kernels.cuh"
#include "lks_tma.cuh"

namespace lks3 {

using lks::block_sum;
using lks::NTHREADS;
using lks::raise_status;
using lks::reduce_partials_kernel;

constexpr int TX3 = 32, TY3 = 8, NT3 = TX3 * TY3, ZC3 = 32;
// Threads of the TMA-staged forward and adjoint: enough for the halo-1 coefficient
// region (34 x 10) in one pass; the first NT3 of them gather the 32 x 8 outputs.
constexpr int NTF3 = 352;
constexpr int HX3 = TX3 + 4, HY3 = TY3 + 4, HA3 = HX3 * HY3;  // plane box with a 2-node halo
constexpr int PX3 = TX3 + 2, PY3 = TY3 + 2, PA3 = PX3 * PY3;  // plane box with a 1-node halo

// D3Q19 velocities: rest, six faces, twelve edges.
__host__ __device__ constexpr int c3(int k, int a) {
  constexpr int c[19][3] = {{0, 0, 0},  {1, 0, 0},   {-1, 0, 0}, {0, 1, 0},  {0, -1, 0}, {0, 0, 1},  {0, 0, -1},
                            {1, 1, 0},  {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0}, {1, 0, 1},  {-1, 0, -1}, {1, 0, -1},
                            {-1, 0, 1}, {0, 1, 1},   {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};
  return c[k][a];
}
__host__ __device__ constexpr double w3d(int k) { return k == 0 ? 1.0 / 3.0 : (k < 7 ? 1.0 / 18.0 : 1.0 / 36.0); }
// Link group by c_z (0: c_z = 0, 1: c_z = +1, 2: c_z = -1) and slot in its group.
__host__ __device__ constexpr int grp3(int k) { return c3(k, 2) == 0 ? 0 : (c3(k, 2) > 0 ? 1 : 2); }
__host__ __device__ constexpr int slot3(int k) {
  int s = 0;
  for (int q = 0; q < k; ++q)
    if (grp3(q) == grp3(k)) ++s;
  return s;
}
// First and second nonzero component of link k (-1: none).
__host__ __device__ constexpr int ax3(int k, int which) {
  int n = 0;
  for (int a = 0; a < 3; ++a)
    if (c3(k, a) != 0) {
      if (n == which) return a;
      ++n;
    }
  return -1;
}

// Component A of (x, y, z), chosen at compile time.
template <int A, typename R>
__device__ __forceinline__ R pick3(R x, R y, R z) {
  if constexpr (A == 0) return x;
  else if constexpr (A == 1) return y;
  else return z;
}

// Pushed increment of link K (Eq. feq2 in 3-D, increment form):
// w_K [(drho - drho(x + c_K)) + e0 + c_K.b + c_K c_K : Q] with b = 3u.  Only the
// nonzero components of c_K enter (a product with a zero constant is not folded
// away under IEEE rules).
template <int K, typename R>
__device__ __forceinline__ R push_link3(R dr, R dest, R e0, R bx, R by, R bz, R Qxx, R Qyy, R Qzz, R Qxy, R Qxz,
                                        R Qyz) {
  constexpr int a0 = ax3(K, 0), a1 = ax3(K, 1);
  const R base = (dr - dest) + e0;
  if constexpr (a0 < 0) {
    return R(w3d(K)) * base;
  } else if constexpr (a1 < 0) {
    const R ba = pick3<a0>(bx, by, bz);
    const R cb = c3(K, a0) > 0 ? ba : -ba;
    return R(w3d(K)) * ((base + cb) + pick3<a0>(Qxx, Qyy, Qzz));
  } else {
    const R ba = pick3<a0>(bx, by, bz), bb = pick3<a1>(bx, by, bz);
    const R cb = (c3(K, a0) > 0 ? ba : -ba) + (c3(K, a1) > 0 ? bb : -bb);
    const R qab = pick3<3 - a0 - a1>(Qyz, Qxz, Qxy);  // the entry of the two axes a0, a1
    const R qo = c3(K, a0) * c3(K, a1) > 0 ? qab : -qab;
    return R(w3d(K)) * ((base + cb) + ((pick3<a0>(Qxx, Qyy, Qzz) + pick3<a1>(Qxx, Qyy, Qzz)) + qo));
  }
}

// Compile-time loop over the lattice links: every link index, velocity, weight and
// slot inside fn is a constant expression.
template <int B, int E, typename Fn>
__device__ __forceinline__ void static_for(Fn&& fn) {
  if constexpr (B < E) {
    fn(std::integral_constant<int, B>{});
    static_for<B + 1, E>(fn);
  }
}

__device__ __forceinline__ int mod5(int p) { return (p + 10) % 5; }
__device__ __forceinline__ int mod3(int p) { return (p + 9) % 3; }
__device__ __forceinline__ int mod2(int p) { return (p + 8) & 1; }

template <typename R>
struct Coef3 {
  R A, nu, alpha_bar, q_alpha, drho_out;
  double u_max;
  double kappa_p;  // weight of the static pressure drop in J
};
struct Geom3 {
  int nx, ny, nz;
};

template <typename R>
__device__ __forceinline__ R alpha3(const Coef3<R>& c, R g) {
  return c.alpha_bar * c.q_alpha * (R(1) - g) / (c.q_alpha + g);
}
template <typename R>
__device__ __forceinline__ R dalpha3(const Coef3<R>& c, R g) {
  const R d = c.q_alpha + g;
  return -c.alpha_bar * c.q_alpha * (R(1) + c.q_alpha) / (d * d);
}

// Derivative along an axis from values spaced `stride` apart around f[0]: central
// inside, second-order one-sided on the faces (at = index along the axis).
template <typename R>
__device__ __forceinline__ R dax(const R* f, int stride, int at, int n) {
  if (at == 0) return (R(-3) * f[0] + R(4) * f[stride] - f[2 * stride]) * R(0.5);
  if (at == n - 1) return (R(3) * f[0] - R(4) * f[-stride] + f[-2 * stride]) * R(0.5);
  return (f[stride] - f[-stride]) * R(0.5);
}
// The same along z through a ring of planes: plane(dz) returns the value dz planes away.
template <typename R, typename Pl>
__device__ __forceinline__ R daz(Pl plane, int p, int nz) {
  if (p == 0) return (R(-3) * plane(0) + R(4) * plane(1) - plane(2)) * R(0.5);
  if (p == nz - 1) return (R(3) * plane(0) - R(4) * plane(-1) + plane(-2)) * R(0.5);
  return (plane(1) - plane(-1)) * R(0.5);
}

__device__ __forceinline__ size_t gidx(const Geom3& g, int i, int j, int k) {
  return ((size_t)k * g.ny + j) * g.nx + i;
}

// Loads plane p of nf fields (halo h in x and y) into dst[f][box]; zeros outside.
template <typename R, int NF, int H>
__device__ __forceinline__ void load_plane(R* dst, const R* const* src, const Geom3& g, int x0, int y0, int p) {
  constexpr int BX = TX3 + 2 * H, BA = BX * (TY3 + 2 * H);
  const bool pin = p >= 0 && p < g.nz;
  for (int q = threadIdx.x; q < NF * BA; q += NT3) {
    const int f = q / BA, r = q - f * BA;
    const int ly = r / BX, lx = r - ly * BX;
    const int i = x0 - H + lx, j = y0 - H + ly;
    R v = R(0);
    if (pin && i >= 0 && i < g.nx && j >= 0 && j < g.ny) v = src[f][gidx(g, i, j, p)];
    dst[f * BA + r] = v;
  }
}

// ------------------------------------------------------------------------------------
// Forward
// ------------------------------------------------------------------------------------
template <typename R>
struct Fwd3Args {
  const R* in[4];  // drho, u, v, w
  R* out[4];
  const R* binv;   // 1 / (1 + alpha_gamma)
  int* status;
};

template <typename R>
constexpr size_t fwd3_smem() {
  return sizeof(R) * (size_t)(5 * 4 * HA3 + 3 * 5 * PA3 + 2 * 9 * PA3 + 5 * PA3);
}

template <typename R>
__global__ void __launch_bounds__(NT3) fwd3_kernel(const __grid_constant__ Fwd3Args<R> a, Geom3 g, Coef3<R> c) {
  extern __shared__ unsigned char smem3[];
  R* stg = reinterpret_cast<R*>(smem3);  // [5 planes][4 fields][HA3]
  R* up = stg + 5 * 4 * HA3;             // [3 planes][5 links][PA3]  c_z = +1
  R* mid = up + 3 * 5 * PA3;             // [2 planes][9 links][PA3]  c_z = 0
  R* dn = mid + 2 * 9 * PA3;             // [5 links][PA3]            c_z = -1
  const int x0 = blockIdx.x * TX3, y0 = blockIdx.y * TY3;
  const int z0 = blockIdx.z * ZC3, z1 = min(z0 + ZC3, g.nz);
  const int nx = g.nx, ny = g.ny, nz = g.nz;

  auto load = [&](int p) { load_plane<R, 4, 2>(stg + mod5(p) * 4 * HA3, a.in, g, x0, y0, p); };

  // Pushed populations of plane p on the halo-1 ring, for the link groups asked.
  auto push = [&](int p, auto up_tag, auto mid_tag, auto dn_tag) {
    constexpr bool want_up = decltype(up_tag)::value, want_mid = decltype(mid_tag)::value,
                   want_dn = decltype(dn_tag)::value;
    if (p < 0 || p >= nz) return;
    for (int q = threadIdx.x; q < PA3; q += NT3) {
      const int ly = q / PX3, lx = q - ly * PX3;
      const int i = x0 - 1 + lx, j = y0 - 1 + ly;
      if (i < 0 || i >= nx || j < 0 || j >= ny) continue;
      const int off = (ly + 1) * HX3 + (lx + 1);
      auto fld = [&](int f, int dz) { return stg + (mod5(p + dz) * 4 + f) * HA3 + off; };
      R uu[3], gr[3][3];
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const R* f0 = fld(1 + d, 0);
        uu[d] = f0[0];
        gr[d][0] = dax(f0, 1, i, nx);
        gr[d][1] = dax(f0, HX3, j, ny);
        gr[d][2] = daz<R>([&](int dz) { return fld(1 + d, dz)[0]; }, p, nz);
      }
      const bool on[3] = {i == 0 || i == nx - 1, j == 0 || j == ny - 1, p == 0 || p == nz - 1};
      const int faces = (int)on[0] + (int)on[1] + (int)on[2];
      if (faces == 1) {  // continuity: normal derivative of the normal component
        if (on[0]) gr[0][0] = -(gr[1][1] + gr[2][2]);
        else if (on[1]) gr[1][1] = -(gr[0][0] + gr[2][2]);
        else gr[2][2] = -(gr[0][0] + gr[1][1]);
      } else if (faces >= 2) {
#pragma unroll
        for (int d = 0; d < 3; ++d)
          if (on[d]) gr[d][d] = R(0);
      }
      const R e0 = R(-1.5) * (uu[0] * uu[0] + uu[1] * uu[1] + uu[2] * uu[2]);
      const R bx = R(3) * uu[0], by = R(3) * uu[1], bz = R(3) * uu[2];
      const R Qxx = R(4.5) * uu[0] * uu[0] + c.A * (R(2) * gr[0][0]);
      const R Qyy = R(4.5) * uu[1] * uu[1] + c.A * (R(2) * gr[1][1]);
      const R Qzz = R(4.5) * uu[2] * uu[2] + c.A * (R(2) * gr[2][2]);
      const R Qxy = R(9) * uu[0] * uu[1] + R(2) * c.A * (gr[0][1] + gr[1][0]);
      const R Qxz = R(9) * uu[0] * uu[2] + R(2) * c.A * (gr[0][2] + gr[2][0]);
      const R Qyz = R(9) * uu[1] * uu[2] + R(2) * c.A * (gr[1][2] + gr[2][1]);
      const R dr = fld(0, 0)[0];
      R* const midq = mid + mod2(p) * 9 * PA3 + q;
      R* const upq = up + mod3(p) * 5 * PA3 + q;
      R* const dnq = dn + q;
      static_for<0, 19>([&](auto kk) {
        constexpr int k = decltype(kk)::value;
        constexpr int gk = grp3(k), sl = slot3(k);
        constexpr int cx = c3(k, 0), cy = c3(k, 1), cz = c3(k, 2);
        if constexpr ((gk == 0 && !want_mid) || (gk == 1 && !want_up) || (gk == 2 && !want_dn)) return;
        const R val = push_link3<k>(dr, fld(0, cz)[cy * HX3 + cx], e0, bx, by, bz, Qxx, Qyy, Qzz, Qxy, Qxz, Qyz);
        if constexpr (gk == 0) midq[sl * PA3] = val;
        else if constexpr (gk == 1) upq[sl * PA3] = val;
        else dnq[sl * PA3] = val;
      });
    }
  };

  // New state of output plane z.
  auto gather = [&](int z) {
    const int tx = threadIdx.x % TX3, ty = threadIdx.x / TX3;
    const int i = x0 + tx, j = y0 + ty;
    if (i >= nx || j >= ny) return;
    const int q1 = (ty + 1) * PX3 + (tx + 1);
    R F[19];
    static_for<0, 19>([&](auto kk) {
      constexpr int k = decltype(kk)::value;
      constexpr int cx = c3(k, 0), cy = c3(k, 1), gk = grp3(k), sl = slot3(k);
      const int qs = q1 - cy * PX3 - cx;  // source x - c_k
      if (gk == 0) F[k] = mid[(mod2(z) * 9 + sl) * PA3 + qs];
      else if (gk == 1) F[k] = up[(mod3(z - 1) * 5 + sl) * PA3 + qs];
      else F[k] = dn[sl * PA3 + qs];
    });
    const int off = (ty + 2) * HX3 + (tx + 2);
    const R drx = stg[(mod5(z) * 4 + 0) * HA3 + off];
    const int n0 = i == 0 ? -1 : (i == nx - 1 ? 1 : 0);
    const int n1 = j == 0 ? -1 : (j == ny - 1 ? 1 : 0);
    const int n2 = z == 0 ? -1 : (z == nz - 1 ? 1 : 0);
    const int faces = abs(n0) + abs(n1) + abs(n2);
    R drn, uo[3] = {R(0), R(0), R(0)};
    if (faces == 0) {
      R s = R(0), mx = R(0), my = R(0), mz = R(0);
      static_for<0, 19>([&](auto kk) {
        constexpr int k = decltype(kk)::value;
        s += F[k];
        if constexpr (c3(k, 0) != 0) mx += R(c3(k, 0)) * F[k];
        if constexpr (c3(k, 1) != 0) my += R(c3(k, 1)) * F[k];
        if constexpr (c3(k, 2) != 0) mz += R(c3(k, 2)) * F[k];
      });
      drn = drx + s;
      const R inv = a.binv[gidx(g, i, j, z)];
      uo[0] = mx * inv;
      uo[1] = my * inv;
      uo[2] = mz * inv;
    } else if (faces >= 2) {  // wall node on two or three faces
      const int jn = (j == 0) ? 1 : (j == ny - 1 ? -1 : 0);
      const int kn = (z == 0) ? 1 : (z == nz - 1 ? -1 : 0);
      drn = stg[(mod5(z + kn) * 4 + 0) * HA3 + off + jn * HX3];
    } else {
      R s0 = R(0), sp = R(0);
      static_for<0, 19>([&](auto kk) {
        constexpr int k = decltype(kk)::value;
        constexpr int cx = c3(k, 0), cy = c3(k, 1), cz = c3(k, 2);
        const int si = i - cx, sj = j - cy, sk = z - cz;
        if (si < 0 || si >= nx || sj < 0 || sj >= ny || sk < 0 || sk >= nz) return;
        const int cn = cx * n0 + cy * n1 + cz * n2;
        if (cn == 0) s0 += F[k];
        else if (cn > 0) sp += F[k];
      });
      if (n0 == 1) {  // outlet: prescribed pressure, tangential velocity zero
        drn = c.drho_out;
        uo[0] = (s0 + R(2) * sp) + (drx - c.drho_out);
      } else {
        if (n0 == -1) {
          const double y = (double)j / (double)(ny - 1), zz = (double)z / (double)(nz - 1);
          uo[0] = (R)(c.u_max * 16.0 * y * (1.0 - y) * zz * (1.0 - zz));
        }
        drn = drx + (s0 + R(2) * sp - (uo[0] * R(n0) + uo[1] * R(n1) + uo[2] * R(n2)));
      }
    }
    const size_t o = gidx(g, i, j, z);
    a.out[0][o] = drn;
    a.out[1][o] = uo[0];
    a.out[2][o] = uo[1];
    a.out[3][o] = uo[2];
    const R m = uo[0] * uo[0] + uo[1] * uo[1] + uo[2] * uo[2];
    if (!(m <= R(0.25))) raise_status(a.status, 4);
  };

  for (int p = z0 - 2; p <= z0 + 2; ++p) load(p);
  __syncthreads();
  using yes = std::true_type;
  using no = std::false_type;
  push(z0 - 1, yes{}, no{}, no{});
  push(z0, yes{}, yes{}, no{});
  __syncthreads();
  for (int z = z0; z < z1; ++z) {
    load(z + 3);
    __syncthreads();
    push(z + 1, yes{}, yes{}, yes{});
    __syncthreads();
    gather(z);
    __syncthreads();
  }
}

// ------------------------------------------------------------------------------------
// Adjoint
// ------------------------------------------------------------------------------------
template <typename R>
struct Adj3Args {
  const R* m1[kNA3];  // adjoint at level t+1: rho~, u~x, u~y, u~z, s~xx, s~xy, s~xz, s~yy, s~yz, s~zz
  R* m0[kNA3];        // adjoint at level t
  const R* u[3];      // state (frozen)
  const R* binv;
  const R* src[3];    // objective source -(1/3) dJ_O/du
  const R* emap;      // kClasses3 x 10 x 19
  int* status;
  const R* zs[3];     // staged with a plane ring: s~xz, s~yz, s~zz
  const R* ps[3];     // staged for one plane: s~xx, s~xy, s~yy
  const R* ns[7];     // staged for one plane on the halo-1 ring: rho~, u~ (3), u (3)
};

template <typename R>
constexpr size_t adj3_smem() {
  return sizeof(R) * (size_t)(5 * 3 * HA3 + 3 * HA3 + 7 * PA3 + 3 * 4 * PA3);
}

template <typename R>
__global__ void __launch_bounds__(NT3) adj3_kernel(const __grid_constant__ Adj3Args<R> a, Geom3 g, Coef3<R> c) {
  extern __shared__ unsigned char smem3[];
  R* szr = reinterpret_cast<R*>(smem3);  // [5 planes][s~xz, s~yz, s~zz][HA3]
  R* spl = szr + 5 * 3 * HA3;            // [s~xx, s~xy, s~yy][HA3] of plane p
  R* nd = spl + 3 * HA3;                 // [rho~, u~x, u~y, u~z, u, v, w][PA3] of plane p
  R* PV = nd + 7 * PA3;                  // [3 planes][P, Vx, Vy, Vz][PA3]
  const int x0 = blockIdx.x * TX3, y0 = blockIdx.y * TY3;
  const int z0 = blockIdx.z * ZC3, z1 = min(z0 + ZC3, g.nz);
  const int nx = g.nx, ny = g.ny, nz = g.nz;
  auto load_ring = [&](int p) { load_plane<R, 3, 2>(szr + mod5(p) * 3 * HA3, a.zs, g, x0, y0, p); };
  auto load_pl = [&](int p) {
    load_plane<R, 3, 2>(spl, a.ps, g, x0, y0, p);
    load_plane<R, 7, 1>(nd, a.ns, g, x0, y0, p);
  };
  // P and V of plane p on the halo-1 ring (Eq. afeq); zero off the lattice.
  auto coefs = [&](int p) {
    R* out = PV + mod3(p) * 4 * PA3;
    for (int q = threadIdx.x; q < PA3; q += NT3) {
      const int ly = q / PX3, lx = q - ly * PX3;
      const int i = x0 - 1 + lx, j = y0 - 1 + ly;
      if (p < 0 || p >= nz || i < 0 || i >= nx || j < 0 || j >= ny) {
        out[q] = out[PA3 + q] = out[2 * PA3 + q] = out[3 * PA3 + q] = R(0);
        continue;
      }
      const int off = (ly + 1) * HX3 + (lx + 1);
      auto ring = [&](int f, int dz) { return szr[(mod5(p + dz) * 3 + f) * HA3 + off]; };
      const R* sxx = spl + off;
      const R* sxy = spl + HA3 + off;
      const R* syy = spl + 2 * HA3 + off;
      const R* sxz = szr + (mod5(p) * 3 + 0) * HA3 + off;
      const R* syz = szr + (mod5(p) * 3 + 1) * HA3 + off;
      const R Dx = R(2) * (dax(sxx, 1, i, nx) + dax(sxy, HX3, j, ny) + daz<R>([&](int dz) { return ring(0, dz); }, p, nz));
      const R Dy = R(2) * (dax(sxy, 1, i, nx) + dax(syy, HX3, j, ny) + daz<R>([&](int dz) { return ring(1, dz); }, p, nz));
      const R Dz = R(2) * (dax(sxz, 1, i, nx) + dax(syz, HX3, j, ny) + daz<R>([&](int dz) { return ring(2, dz); }, p, nz));
      const R rt = nd[q], ux = nd[PA3 + q], uy = nd[2 * PA3 + q], uz = nd[3 * PA3 + q];
      const R u0 = nd[4 * PA3 + q], u1 = nd[5 * PA3 + q], u2 = nd[6 * PA3 + q];
      const R vxx = sxx[0], vxy = sxy[0], vyy = syy[0], vxz = sxz[0], vyz = syz[0], vzz = ring(2, 0);
      out[q] = rt;
      out[PA3 + q] = R(3) * (ux + R(3) * (vxx * u0 + vxy * u1 + vxz * u2) - rt * u0) - c.A * Dx;
      out[2 * PA3 + q] = R(3) * (uy + R(3) * (vxy * u0 + vyy * u1 + vyz * u2) - rt * u1) - c.A * Dy;
      out[3 * PA3 + q] = R(3) * (uz + R(3) * (vxz * u0 + vyz * u1 + vzz * u2) - rt * u2) - c.A * Dz;
    }
  };
  // Adjoint moments of output plane z.
  auto gather = [&](int z) {
    const int tx = threadIdx.x % TX3, ty = threadIdx.x / TX3;
    const int i = x0 + tx, j = y0 + ty;
    if (i >= nx || j >= ny) return;
    const int q1 = (ty + 1) * PX3 + (tx + 1);
    const int n0 = i == 0 ? -1 : (i == nx - 1 ? 1 : 0);
    const int n1 = j == 0 ? -1 : (j == ny - 1 ? 1 : 0);
    const int n2 = z == 0 ? -1 : (z == nz - 1 ? 1 : 0);
    const bool edge = (n0 | n1 | n2) != 0;
    R f[19];
    static_for<0, 19>([&](auto kk) {
      constexpr int k = decltype(kk)::value;
      constexpr int cx = c3(k, 0), cy = c3(k, 1), cz = c3(k, 2);
      const R* pv = PV + mod3(z + cz) * 4 * PA3 + q1 + cy * PX3 + cx;
      R v = pv[0];
      if constexpr (cx != 0) v += R(cx) * pv[PA3];
      if constexpr (cy != 0) v += R(cy) * pv[2 * PA3];
      if constexpr (cz != 0) v += R(cz) * pv[3 * PA3];
      f[k] = v;
      if (edge) {
        const int gi = i + cx, gj = j + cy, gk = z + cz;
        if (gi < 0 || gi >= nx || gj < 0 || gj >= ny || gk < 0 || gk >= nz) f[k] = R(0);
      }
    });
    R m[kNA3];
    const size_t o = gidx(g, i, j, z);
    if (!edge) {
#pragma unroll
      for (int r = 0; r < kNA3; ++r) m[r] = R(0);
      static_for<0, 19>([&](auto kk) {
        constexpr int k = decltype(kk)::value;
        constexpr int cx = c3(k, 0), cy = c3(k, 1), cz = c3(k, 2);
        const R wf = R(w3d(k)) * f[k];
        m[0] += wf;
        if constexpr (cx != 0) m[1] += R(cx) * wf;
        if constexpr (cy != 0) m[2] += R(cy) * wf;
        if constexpr (cz != 0) m[3] += R(cz) * wf;
        if constexpr (cx != 0) m[4] += wf;
        if constexpr (cx * cy != 0) m[5] += R(cx * cy) * wf;
        if constexpr (cx * cz != 0) m[6] += R(cx * cz) * wf;
        if constexpr (cy != 0) m[7] += wf;
        if constexpr (cy * cz != 0) m[8] += R(cy * cz) * wf;
        if constexpr (cz != 0) m[9] += wf;
      });
      const R inv = a.binv[o];
      m[1] = (m[1] + a.src[0][o]) * inv;
      m[2] = (m[2] + a.src[1][o]) * inv;
      m[3] = (m[3] + a.src[2][o]) * inv;
    } else {
      const int cls = (n0 + 1) * 9 + (n1 + 1) * 3 + (n2 + 1);
      const R* M = a.emap + cls * (kNA3 * 19);
      const R* M0 = a.emap + kClasses3 * kNA3 * 19 + cls * kNA3;  // boundary objective term
#pragma unroll
      for (int r = 0; r < kNA3; ++r) {
        R s = R(0);
        static_for<0, 19>([&](auto kk) {
          constexpr int k = decltype(kk)::value;
          s += M[r * 19 + k] * f[k];
        });
        m[r] = s + M0[r];
      }
    }
#pragma unroll
    for (int r = 0; r < kNA3; ++r) a.m0[r][o] = m[r];
    if (!(m[1] * m[1] + m[2] * m[2] + m[3] * m[3] < R(1e30))) raise_status(a.status, 4);
  };

  for (int p = z0 - 2; p <= z0 + 2; ++p) load_ring(p);
  load_pl(z0 - 1);
  __syncthreads();
  coefs(z0 - 1);
  __syncthreads();
  load_pl(z0);
  __syncthreads();
  coefs(z0);
  __syncthreads();
  for (int z = z0; z < z1; ++z) {
    load_ring(z + 3);
    load_pl(z + 1);
    __syncthreads();
    coefs(z + 1);
    __syncthreads();
    gather(z);
    __syncthreads();
  }
}

// ------------------------------------------------------------------------------------
// TMA-staged forms (FP32, nx % 4 == 0)
// ------------------------------------------------------------------------------------
// The same marches with every staged plane brought in by 3-D tensor copies
// (cp.async.bulk.tensor.3d) into ring slots guarded by mbarriers with transaction
// counts: the copy of a plane a few planes ahead overlaps the compute of the
// current one, out-of-lattice parts of a box arrive as zeros, and no thread
// computes a load address.  A box is 40 x 12 nodes starting at (x0 - 4, y0 - 2):
// the two-node halo, with x rounded down to a multiple of four floats (16 bytes).
// Columns whose two-node halo lies inside the lattice in x and y take a path
// without face tests except on the z faces.  Every mbarrier wait is bounded; on a
// timeout the kernel records LKS_ERR_TIMEOUT, drains its own copies and returns.
constexpr int BW3 = TX3 + 8, BH3 = TY3 + 4, BOX3 = BW3 * BH3;
constexpr int NSL3 = 6;  // plane ring slots
constexpr int NFF3 = 5;  // forward: drho, u, v, w, 1/(1+alpha)

struct Maps3F {
  CUtensorMap m[NFF3];
};
struct Maps3A {
  CUtensorMap zr[3];   // ring: s~xz, s~yz, s~zz
  CUtensorMap pl[10];  // plane of PV: s~xx, s~xy, s~yy, rho~, u~x, u~y, u~z, u, v, w
  CUtensorMap out[4];  // output plane (boxes 32 x 8): 1/(1+alpha), src x, y, z
};

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(
          lks::smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(lks::smem_u32(bar))
      : "memory");
}

__host__ __device__ constexpr size_t fwd3t_smem() {
  return sizeof(float) * (size_t)(NSL3 * NFF3 * BOX3 + 3 * 5 * PA3 + 2 * 9 * PA3 + 5 * PA3) + 8 * NSL3 + 128;
}
__host__ __device__ constexpr size_t adj3t_smem() {
  return sizeof(float) * (size_t)(NSL3 * 3 * BOX3 + 2 * 10 * BOX3 + 2 * 4 * NT3 + 3 * 4 * PA3) + 8 * (NSL3 + 4) + 128;
}

struct Fwd3TArgs {
  float* out[4];
  const float* binv;  // 1/(1+alpha) per node (read by the warp-column forward)
  int* status;
  int zc;             // z planes per CTA of the warp-column forward
};

__global__ void __launch_bounds__(NTF3, 2) fwd3t_kernel(const __grid_constant__ Maps3F maps, const __grid_constant__ Fwd3TArgs a,
                                                    Geom3 g, Coef3<float> c) {
  using R = float;
  extern __shared__ unsigned char smem_raw3[];
  R* ring = reinterpret_cast<R*>(lks::smem_base128(smem_raw3));  // [NSL3][NFF3][BOX3]
  R* up = ring + NSL3 * NFF3 * BOX3;                               // [3][5][PA3]
  R* mid = up + 3 * 5 * PA3;                                       // [2][9][PA3]
  R* dn = mid + 2 * 9 * PA3;                                       // [5][PA3]
  uint64_t* bar = reinterpret_cast<uint64_t*>(dn + 5 * PA3);       // [NSL3]
  if (lks::timed_out_before(a.status)) return;
  if (!lks::tma_layout_ok(ring, bar, a.status)) return;
  const int x0 = blockIdx.x * TX3, y0 = blockIdx.y * TY3;
  const int z0 = blockIdx.z * ZC3, z1 = min(z0 + ZC3, g.nz);
  const int nx = g.nx, ny = g.ny, nz = g.nz;
  const int pbase = z0 - 2, plast = z1 + 2;
  const bool xyi = x0 >= 2 && y0 >= 2 && x0 + TX3 + 2 <= nx && y0 + TY3 + 2 <= ny;
  auto slot = [&](int p) { return (p - pbase) % NSL3; };
  auto issue = [&](int p) {
    const int sl = slot(p);
    lks::mbar_expect_tx(&bar[sl], NFF3 * BOX3 * 4);
    for (int f = 0; f < NFF3; ++f) tma_load_3d(ring + (sl * NFF3 + f) * BOX3, &maps.m[f], x0 - 4, y0 - 2, p, &bar[sl]);
  };
  int waited = pbase - 1, issued = pbase - 1;
  auto drain_and_fail = [&]() {
    raise_status(a.status, 6);
    if (threadIdx.x == 0)
      for (int p = waited + 1; p <= issued; ++p) lks::mbar_wait(&bar[slot(p)], ((p - pbase) / NSL3) & 1);
  };
  auto wait = [&](int p) {
    const bool ok = lks::mbar_wait(&bar[slot(p)], ((p - pbase) / NSL3) & 1);
    if (ok) waited = p;
    return ok;
  };
  if (threadIdx.x == 0) {
    for (int sl = 0; sl < NSL3; ++sl) lks::mbar_init(&bar[sl], 1);
    lks::fence_mbar_init();
    lks::fence_proxy_async();
  }
  __syncthreads();
  for (int p = pbase; p < pbase + NSL3 && p <= plast; ++p) {
    if (threadIdx.x == 0) issue(p);
    issued = p;
  }
  auto plane = [&](int f, int p) -> const R* { return ring + (slot(p) * NFF3 + f) * BOX3; };

  auto push = [&](int p, auto up_tag, auto mid_tag, auto dn_tag, auto fast_tag) {
    constexpr bool FAST = decltype(fast_tag)::value;
    constexpr bool want_up = decltype(up_tag)::value, want_mid = decltype(mid_tag)::value,
                   want_dn = decltype(dn_tag)::value;
    if (p < 0 || p >= nz) return;
    const bool zf = p == 0 || p == nz - 1;
    for (int q = threadIdx.x; q < PA3; q += NTF3) {
      const int ly = q / PX3, lx = q - ly * PX3;
      const int i = x0 - 1 + lx, j = y0 - 1 + ly;
      if (!FAST && (i < 0 || i >= nx || j < 0 || j >= ny)) continue;
      const int boff = (ly + 1) * BW3 + (lx + 3);
      R uu[3], gr[3][3];
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const R* f0 = plane(1 + d, p) + boff;
        uu[d] = f0[0];
        if (FAST) {
          gr[d][0] = (f0[1] - f0[-1]) * R(0.5);
          gr[d][1] = (f0[BW3] - f0[-BW3]) * R(0.5);
        } else {
          gr[d][0] = dax(f0, 1, i, nx);
          gr[d][1] = dax(f0, BW3, j, ny);
        }
        gr[d][2] = zf ? daz<R>([&](int dz) { return plane(1 + d, p + dz)[boff]; }, p, nz)
                      : (plane(1 + d, p + 1)[boff] - plane(1 + d, p - 1)[boff]) * R(0.5);
      }
      const bool on[3] = {!FAST && (i == 0 || i == nx - 1), !FAST && (j == 0 || j == ny - 1), zf};
      const int faces = (int)on[0] + (int)on[1] + (int)on[2];
      if (faces == 1) {
        if (on[0]) gr[0][0] = -(gr[1][1] + gr[2][2]);
        else if (on[1]) gr[1][1] = -(gr[0][0] + gr[2][2]);
        else gr[2][2] = -(gr[0][0] + gr[1][1]);
      } else if (faces >= 2) {
#pragma unroll
        for (int d = 0; d < 3; ++d)
          if (on[d]) gr[d][d] = R(0);
      }
      const R e0 = R(-1.5) * (uu[0] * uu[0] + uu[1] * uu[1] + uu[2] * uu[2]);
      const R bx = R(3) * uu[0], by = R(3) * uu[1], bz = R(3) * uu[2];
      const R Qxx = R(4.5) * uu[0] * uu[0] + c.A * (R(2) * gr[0][0]);
      const R Qyy = R(4.5) * uu[1] * uu[1] + c.A * (R(2) * gr[1][1]);
      const R Qzz = R(4.5) * uu[2] * uu[2] + c.A * (R(2) * gr[2][2]);
      const R Qxy = R(9) * uu[0] * uu[1] + R(2) * c.A * (gr[0][1] + gr[1][0]);
      const R Qxz = R(9) * uu[0] * uu[2] + R(2) * c.A * (gr[0][2] + gr[2][0]);
      const R Qyz = R(9) * uu[1] * uu[2] + R(2) * c.A * (gr[1][2] + gr[2][1]);
      const R* d0 = plane(0, p) + boff;
      const R* dm = plane(0, p - 1) + boff;
      const R* dp = plane(0, p + 1) + boff;
      const R dr = d0[0];
      R* const midq = mid + mod2(p) * 9 * PA3 + q;
      R* const upq = up + mod3(p) * 5 * PA3 + q;
      R* const dnq = dn + q;
      static_for<0, 19>([&](auto kk) {
        constexpr int k = decltype(kk)::value;
        constexpr int gk = grp3(k), sl = slot3(k);
        constexpr int cx = c3(k, 0), cy = c3(k, 1), cz = c3(k, 2);
        if constexpr ((gk == 0 && !want_mid) || (gk == 1 && !want_up) || (gk == 2 && !want_dn)) return;
        const R val = push_link3<k>(dr, (cz == 0 ? d0 : (cz > 0 ? dp : dm))[cy * BW3 + cx], e0, bx, by, bz, Qxx, Qyy,
                                    Qzz, Qxy, Qxz, Qyz);
        if constexpr (gk == 0) midq[sl * PA3] = val;
        else if constexpr (gk == 1) upq[sl * PA3] = val;
        else dnq[sl * PA3] = val;
      });
    }
  };

  auto gather = [&](int z, auto fast_tag) {
    constexpr bool FAST = decltype(fast_tag)::value;
    if (threadIdx.x >= NT3) return;
    const int tx = threadIdx.x % TX3, ty = threadIdx.x / TX3;
    const int i = x0 + tx, j = y0 + ty;
    if (!FAST && (i >= nx || j >= ny)) return;
    const int q1 = (ty + 1) * PX3 + (tx + 1);
    R F[19];
    static_for<0, 19>([&](auto kk) {
      constexpr int k = decltype(kk)::value;
      constexpr int cx = c3(k, 0), cy = c3(k, 1), gk = grp3(k), sl = slot3(k);
      const int qs = q1 - cy * PX3 - cx;
      if (gk == 0) F[k] = mid[(mod2(z) * 9 + sl) * PA3 + qs];
      else if (gk == 1) F[k] = up[(mod3(z - 1) * 5 + sl) * PA3 + qs];
      else F[k] = dn[sl * PA3 + qs];
    });
    const int boff = (ty + 2) * BW3 + (tx + 4);
    const R drx = plane(0, z)[boff];
    const int n0 = FAST ? 0 : (i == 0 ? -1 : (i == nx - 1 ? 1 : 0));
    const int n1 = FAST ? 0 : (j == 0 ? -1 : (j == ny - 1 ? 1 : 0));
    const int n2 = z == 0 ? -1 : (z == nz - 1 ? 1 : 0);
    const int faces = abs(n0) + abs(n1) + abs(n2);
    R drn, uo[3] = {R(0), R(0), R(0)};
    if (faces == 0) {
      R sm = R(0), mx = R(0), my = R(0), mz = R(0);
      static_for<0, 19>([&](auto kk) {
        constexpr int k = decltype(kk)::value;
        sm += F[k];
        if constexpr (c3(k, 0) != 0) mx += R(c3(k, 0)) * F[k];
        if constexpr (c3(k, 1) != 0) my += R(c3(k, 1)) * F[k];
        if constexpr (c3(k, 2) != 0) mz += R(c3(k, 2)) * F[k];
      });
      drn = drx + sm;
      const R inv = plane(4, z)[boff];
      uo[0] = mx * inv;
      uo[1] = my * inv;
      uo[2] = mz * inv;
    } else if (faces >= 2) {
      const int jn = (j == 0) ? 1 : (j == ny - 1 ? -1 : 0);
      const int kn = (z == 0) ? 1 : (z == nz - 1 ? -1 : 0);
      drn = plane(0, z + kn)[boff + jn * BW3];
    } else {
      R s0 = R(0), sp = R(0);
      static_for<0, 19>([&](auto kk) {
        constexpr int k = decltype(kk)::value;
        constexpr int cx = c3(k, 0), cy = c3(k, 1), cz = c3(k, 2);
        const int si = i - cx, sj = j - cy, sk = z - cz;
        if (si < 0 || si >= nx || sj < 0 || sj >= ny || sk < 0 || sk >= nz) return;
        const int cn = cx * n0 + cy * n1 + cz * n2;
        if (cn == 0) s0 += F[k];
        else if (cn > 0) sp += F[k];
      });
      if (n0 == 1) {
        drn = c.drho_out;
        uo[0] = (s0 + R(2) * sp) + (drx - c.drho_out);
      } else {
        if (n0 == -1) {
          const double y = (double)j / (double)(ny - 1), zz = (double)z / (double)(nz - 1);
          uo[0] = (R)(c.u_max * 16.0 * y * (1.0 - y) * zz * (1.0 - zz));
        }
        drn = drx + (s0 + R(2) * sp - (uo[0] * R(n0) + uo[1] * R(n1) + uo[2] * R(n2)));
      }
    }
    const size_t o = gidx(g, i, j, z);
    a.out[0][o] = drn;
    a.out[1][o] = uo[0];
    a.out[2][o] = uo[1];
    a.out[3][o] = uo[2];
    const R m = uo[0] * uo[0] + uo[1] * uo[1] + uo[2] * uo[2];
    if (!(m <= R(0.25))) raise_status(a.status, 4);
  };

  auto run = [&](auto fast_tag) {
    for (int p = pbase; p <= pbase + 4; ++p)
      if (!wait(p)) return false;
    using yes = std::true_type;
    using no = std::false_type;
    push(z0 - 1, yes{}, no{}, no{}, fast_tag);
    push(z0, yes{}, yes{}, no{}, fast_tag);
    __syncthreads();
    for (int z = z0; z < z1; ++z) {
      if (z + 4 <= plast) {  // the slot of plane z - 2 is free
        if (threadIdx.x == 0) issue(z + 4);
        issued = z + 4;
      }
      if (!wait(z + 3)) return false;
      push(z + 1, yes{}, yes{}, yes{}, fast_tag);
      __syncthreads();
      gather(z, fast_tag);
      __syncthreads();
    }
    return true;
  };
  const bool ok = xyi ? run(std::true_type{}) : run(std::false_type{});
  if (!ok) drain_and_fail();
}

// Index of the link with velocity (x, y, z).
__host__ __device__ constexpr int link3(int x, int y, int z) {
  int k = 0;
  while (k < 19 && !(c3(k, 0) == x && c3(k, 1) == y && c3(k, 2) == z)) ++k;
  return k;
}

// The ten ALKS moments (rho~, u~x, u~y, u~z, s~xx, s~xy, s~xz, s~yy, s~yz, s~zz) of
// the 19 gathered values F at an interior node, sum_k w_k F_k {1, c_k, c_k c_k}
// (Sec. 2.5), summed by link class: the pair of axis links of each axis, and the
// four diagonal links of each pair of axes, which enter the momentum of both axes,
// the two diagonal second moments and the off-diagonal one.
__device__ __forceinline__ void adj_moments3(const float (&F)[19], float (&m)[kNA3]) {
  constexpr float w0 = (float)w3d(link3(0, 0, 0)), w1 = (float)w3d(link3(1, 0, 0)), w2 = (float)w3d(link3(1, 1, 0));
  constexpr int sa[3][3] = {{4, 5, 6}, {5, 7, 8}, {6, 8, 9}};  // moment index of s~_ab
  float sum_ax[3], dif_ax[3];
  static_for<0, 3>([&](auto aa) {
    constexpr int a = decltype(aa)::value;
    constexpr int kp = link3(a == 0, a == 1, a == 2), km = link3(-(a == 0), -(a == 1), -(a == 2));
    sum_ax[a] = F[kp] + F[km];
    dif_ax[a] = F[kp] - F[km];
  });
  float mom[3] = {w1 * dif_ax[0], w1 * dif_ax[1], w1 * dif_ax[2]};
  float dia[3] = {w1 * sum_ax[0], w1 * sum_ax[1], w1 * sum_ax[2]};
  float s4all = 0.f;
  static_for<0, 3>([&](auto pp) {
    constexpr int p = decltype(pp)::value;
    constexpr int a = p == 2 ? 1 : 0, b = p == 0 ? 1 : 2;  // axis pairs (x,y), (x,z), (y,z)
    constexpr int ea[3] = {a == 0, a == 1, a == 2}, eb[3] = {b == 0, b == 1, b == 2};
    constexpr int kpp = link3(ea[0] + eb[0], ea[1] + eb[1], ea[2] + eb[2]);
    constexpr int kmm = link3(-ea[0] - eb[0], -ea[1] - eb[1], -ea[2] - eb[2]);
    constexpr int kpm = link3(ea[0] - eb[0], ea[1] - eb[1], ea[2] - eb[2]);
    constexpr int kmp = link3(eb[0] - ea[0], eb[1] - ea[1], eb[2] - ea[2]);
    const float P = F[kpp] + F[kmm], Q = F[kpm] + F[kmp];
    const float Rr = F[kpp] - F[kmm], S = F[kpm] - F[kmp];
    const float s4 = P + Q;
    s4all += s4;
    m[sa[a][b]] = w2 * (P - Q);
    mom[a] += w2 * (Rr + S);
    mom[b] += w2 * (Rr - S);
    dia[a] += w2 * s4;
    dia[b] += w2 * s4;
  });
  m[0] = w0 * F[0] + (w1 * (sum_ax[0] + sum_ax[1] + sum_ax[2]) + w2 * s4all);
  m[1] = mom[0];
  m[2] = mom[1];
  m[3] = mom[2];
  m[4] = dia[0];
  m[7] = dia[1];
  m[9] = dia[2];
}

// ---------------------------------------------------------------------------------
// Warp-column D3Q19 tiles (FP32)
// ---------------------------------------------------------------------------------
// The column kernels (the paired forward fwd3p_kernel and the adjoint adj3c_kernel)
// share one tiling: 28 x 8 output tiles, a halo row above and below, and a chunk of
// z planes marched by each CTA.  The staged fields of each plane arrive by 3-D tensor
// copies into a ring of plane slots (box 36 x (NYC3 + 4) from (x0 - 4, y0 - 2)).  The
// pushed values of a source plane are routed at once: links with c_y = 0 stay in
// the warp (c_x by shuffle, c_z through a register ring of destination planes), the
// others go to the neighbouring rows through a shared exchange buffer indexed by
// destination plane mod NXS3.  One barrier per plane separates the exchange writes
// from the gather of plane z - 1, which is complete then.  A slot of the exchange
// buffer is rewritten two steps after it is read, with that barrier in between.
constexpr int CX3 = 28, NYC3 = 8, NWC3 = NYC3 + 2, NTC3 = 32 * NWC3;
constexpr int CBW3 = CX3 + 8, CBH3 = NYC3 + 4, CBOX3 = CBW3 * CBH3;
constexpr int CFS3 = (CBOX3 * 4 + 127) / 128 * 128 / 4;  // field stride in a ring slot (128-byte multiple)
constexpr int NFC3 = 4;                                   // forward ring fields: drho, u, v, w
constexpr int NSLC3 = 8;                                  // adjoint ring slots (planes z - 2 .. z + 5)
constexpr int NXS3 = 4;                                   // exchange slots (destination planes mod 4)
constexpr int XW3 = CX3;                                  // exchange row: the output columns x0 .. x0 + 27
constexpr int NXL3 = 10;                                  // links with c_y != 0

// Slot of link k among the ten links with c_y != 0, and among the nine with c_y = 0.
__host__ __device__ constexpr int yslot3(int k) {
  int s = 0;
  for (int q = 0; q < k; ++q)
    if (c3(q, 1) != 0) ++s;
  return s;
}
__host__ __device__ constexpr int oslot3(int k) {
  int s = 0;
  for (int q = 0; q < k; ++q)
    if (c3(q, 1) == 0) ++s;
  return s;
}

// Link q (0..4, in link order) of face ff (axis a = ff / 2, outward sign s = +1 for
// odd ff, -1 for even): among the links with c_a = s (unknown at that face) or with
// c_a = -s (the opposite links).
__host__ __device__ constexpr int face_link3(int ff, int q, bool unknown) {
  const int a = ff / 2, want = ((ff & 1) ? 1 : -1) * (unknown ? 1 : -1);
  int n = 0;
  for (int k = 0; k < 19; ++k)
    if (c3(k, a) == want) {
      if (n == q) return k;
      ++n;
    }
  return -1;
}

// Sums of the pushed increments at a node on exactly one face, normal along axis A
// with sign n (the face rules of the gather): s0 over links with c_A = 0, sp over
// links pointing out of the lattice (c_A n > 0).  Off the normal's axis every
// source is inside, so no link needs a bounds test; the sums run in link order.
template <int A>
__device__ __forceinline__ void face_sums3(const float (&F)[19], int n, float& s0, float& sp) {
  float z = 0.f, p = 0.f, m = 0.f;
  static_for<0, 19>([&](auto kk) {
    constexpr int k = decltype(kk)::value;
    if constexpr (c3(k, A) == 0) z += F[k];
    else if constexpr (c3(k, A) > 0) p += F[k];
    else m += F[k];
  });
  s0 = z;
  sp = n > 0 ? p : m;
}

struct Adj3TArgs {
  float* m0[kNA3];
  const float* emap;
  int* status;
};

__global__ void __launch_bounds__(NTF3, 2) adj3t_kernel(const __grid_constant__ Maps3A maps, const __grid_constant__ Adj3TArgs a,
                                                    Geom3 g, Coef3<float> c) {
  using R = float;
  extern __shared__ unsigned char smem_raw3[];
  R* ra = reinterpret_cast<R*>(lks::smem_base128(smem_raw3));  // [NSL3][3][BOX3]
  R* rb = ra + NSL3 * 3 * BOX3;                                  // [2][10][BOX3]
  R* rc = rb + 2 * 10 * BOX3;                                    // [2][4][NT3]
  R* PV = rc + 2 * 4 * NT3;                                      // [3][4][PA3]
  uint64_t* bar = reinterpret_cast<uint64_t*>(PV + 3 * 4 * PA3);  // A: NSL3, B: 2, C: 2
  uint64_t* barB = bar + NSL3;
  uint64_t* barC = barB + 2;
  if (lks::timed_out_before(a.status)) return;
  if (!lks::tma_layout_ok(ra, bar, a.status)) return;
  const int x0 = blockIdx.x * TX3, y0 = blockIdx.y * TY3;
  const int z0 = blockIdx.z * ZC3, z1 = min(z0 + ZC3, g.nz);
  const int nx = g.nx, ny = g.ny, nz = g.nz;
  const int pa0 = z0 - 2, pa_last = z1 + 2;  // ring A planes
  const int pb0 = z0 - 1, pb_last = z1;      // PV planes
  const bool xyi = x0 >= 2 && y0 >= 2 && x0 + TX3 + 2 <= nx && y0 + TY3 + 2 <= ny;
  auto slotA = [&](int p) { return (p - pa0) % NSL3; };
  auto parA = [&](int p) { return (uint32_t)(((p - pa0) / NSL3) & 1); };
  auto bufB = [&](int p) { return (p - pb0) & 1; };
  auto parB = [&](int p) { return (uint32_t)(((p - pb0) >> 1) & 1); };
  auto bufC = [&](int p) { return (p - z0) & 1; };
  auto parC = [&](int p) { return (uint32_t)(((p - z0) >> 1) & 1); };
  auto issueA = [&](int p) {
    lks::mbar_expect_tx(&bar[slotA(p)], 3 * BOX3 * 4);
    for (int f = 0; f < 3; ++f)
      tma_load_3d(ra + (slotA(p) * 3 + f) * BOX3, &maps.zr[f], x0 - 4, y0 - 2, p, &bar[slotA(p)]);
  };
  auto issueB = [&](int p) {
    lks::mbar_expect_tx(&barB[bufB(p)], 10 * BOX3 * 4);
    for (int f = 0; f < 10; ++f)
      tma_load_3d(rb + (bufB(p) * 10 + f) * BOX3, &maps.pl[f], x0 - 4, y0 - 2, p, &barB[bufB(p)]);
  };
  auto issueC = [&](int p) {
    lks::mbar_expect_tx(&barC[bufC(p)], 4 * NT3 * 4);
    for (int f = 0; f < 4; ++f) tma_load_3d(rc + (bufC(p) * 4 + f) * NT3, &maps.out[f], x0, y0, p, &barC[bufC(p)]);
  };
  // Copies in flight, for the drain on a timeout: [lo, hi] per group.
  int a_lo = pa0, a_hi = pa0 - 1, b_lo = pb0, b_hi = pb0 - 1, c_lo = z0, c_hi = z0 - 1;
  auto drain_and_fail = [&]() {
    raise_status(a.status, 6);
    if (threadIdx.x == 0) {
      for (int p = a_lo; p <= a_hi; ++p) lks::mbar_wait(&bar[slotA(p)], parA(p));
      for (int p = b_lo; p <= b_hi; ++p) lks::mbar_wait(&barB[bufB(p)], parB(p));
      for (int p = c_lo; p <= c_hi; ++p) lks::mbar_wait(&barC[bufC(p)], parC(p));
    }
  };
  auto waitA = [&](int p) { const bool ok = lks::mbar_wait(&bar[slotA(p)], parA(p)); if (ok) a_lo = p + 1; return ok; };
  auto waitB = [&](int p) { const bool ok = lks::mbar_wait(&barB[bufB(p)], parB(p)); if (ok) b_lo = p + 1; return ok; };
  auto waitC = [&](int p) { const bool ok = lks::mbar_wait(&barC[bufC(p)], parC(p)); if (ok) c_lo = p + 1; return ok; };
  if (threadIdx.x == 0) {
    for (int q = 0; q < NSL3 + 4; ++q) lks::mbar_init(&bar[q], 1);
    lks::fence_mbar_init();
    lks::fence_proxy_async();
  }
  __syncthreads();
  for (int p = pa0; p < pa0 + NSL3 && p <= pa_last; ++p) {
    if (threadIdx.x == 0) issueA(p);
    a_hi = p;
  }
  for (int p = pb0; p <= pb0 + 1 && p <= pb_last; ++p) {
    if (threadIdx.x == 0) issueB(p);
    b_hi = p;
  }
  if (threadIdx.x == 0) issueC(z0);
  c_hi = z0;

  auto ringv = [&](int f, int p) -> const R* { return ra + (slotA(p) * 3 + f) * BOX3; };
  auto coefs = [&](int p, auto fast_tag) {
    constexpr bool FAST = decltype(fast_tag)::value;
    R* out = PV + mod3(p) * 4 * PA3;
    const R* B = rb + bufB(p) * 10 * BOX3;
    const bool zf = p == 0 || p == nz - 1;
    for (int q = threadIdx.x; q < PA3; q += NTF3) {
      const int ly = q / PX3, lx = q - ly * PX3;
      const int i = x0 - 1 + lx, j = y0 - 1 + ly;
      if (p < 0 || p >= nz || (!FAST && (i < 0 || i >= nx || j < 0 || j >= ny))) {
        out[q] = out[PA3 + q] = out[2 * PA3 + q] = out[3 * PA3 + q] = R(0);
        continue;
      }
      const int boff = (ly + 1) * BW3 + (lx + 3);
      const R* sxx = B + boff;
      const R* sxy = B + BOX3 + boff;
      const R* syy = B + 2 * BOX3 + boff;
      const R* sxz = ringv(0, p) + boff;
      const R* syz = ringv(1, p) + boff;
      auto dzr = [&](int f) {
        return zf ? daz<R>([&](int dz) { return ringv(f, p + dz)[boff]; }, p, nz)
                  : (ringv(f, p + 1)[boff] - ringv(f, p - 1)[boff]) * R(0.5);
      };
      R Dx, Dy, Dz;
      if (FAST) {
        Dx = R(2) * ((sxx[1] - sxx[-1]) * R(0.5) + (sxy[BW3] - sxy[-BW3]) * R(0.5) + dzr(0));
        Dy = R(2) * ((sxy[1] - sxy[-1]) * R(0.5) + (syy[BW3] - syy[-BW3]) * R(0.5) + dzr(1));
        Dz = R(2) * ((sxz[1] - sxz[-1]) * R(0.5) + (syz[BW3] - syz[-BW3]) * R(0.5) + dzr(2));
      } else {
        Dx = R(2) * (dax(sxx, 1, i, nx) + dax(sxy, BW3, j, ny) + dzr(0));
        Dy = R(2) * (dax(sxy, 1, i, nx) + dax(syy, BW3, j, ny) + dzr(1));
        Dz = R(2) * (dax(sxz, 1, i, nx) + dax(syz, BW3, j, ny) + dzr(2));
      }
      const R rt = B[3 * BOX3 + boff], ux = B[4 * BOX3 + boff], uy = B[5 * BOX3 + boff], uz = B[6 * BOX3 + boff];
      const R u0 = B[7 * BOX3 + boff], u1 = B[8 * BOX3 + boff], u2 = B[9 * BOX3 + boff];
      const R vxx = sxx[0], vxy = sxy[0], vyy = syy[0], vxz = sxz[0], vyz = syz[0], vzz = ringv(2, p)[boff];
      out[q] = rt;
      out[PA3 + q] = R(3) * (ux + R(3) * (vxx * u0 + vxy * u1 + vxz * u2) - rt * u0) - c.A * Dx;
      out[2 * PA3 + q] = R(3) * (uy + R(3) * (vxy * u0 + vyy * u1 + vyz * u2) - rt * u1) - c.A * Dy;
      out[3 * PA3 + q] = R(3) * (uz + R(3) * (vxz * u0 + vyz * u1 + vzz * u2) - rt * u2) - c.A * Dz;
    }
  };
  auto gather = [&](int z, auto fast_tag) {
    constexpr bool FAST = decltype(fast_tag)::value;
    if (threadIdx.x >= NT3) return;
    const int tx = threadIdx.x % TX3, ty = threadIdx.x / TX3;
    const int i = x0 + tx, j = y0 + ty;
    if (!FAST && (i >= nx || j >= ny)) return;
    const int q1 = (ty + 1) * PX3 + (tx + 1);
    const int n0 = FAST ? 0 : (i == 0 ? -1 : (i == nx - 1 ? 1 : 0));
    const int n1 = FAST ? 0 : (j == 0 ? -1 : (j == ny - 1 ? 1 : 0));
    const int n2 = z == 0 ? -1 : (z == nz - 1 ? 1 : 0);
    const bool edge = (n0 | n1 | n2) != 0;
    R f[19];
    static_for<0, 19>([&](auto kk) {
      constexpr int k = decltype(kk)::value;
      constexpr int cx = c3(k, 0), cy = c3(k, 1), cz = c3(k, 2);
      const R* pv = PV + mod3(z + cz) * 4 * PA3 + q1 + cy * PX3 + cx;
      R v = pv[0];
      if constexpr (cx != 0) v += R(cx) * pv[PA3];
      if constexpr (cy != 0) v += R(cy) * pv[2 * PA3];
      if constexpr (cz != 0) v += R(cz) * pv[3 * PA3];
      f[k] = v;
      if (edge) {
        const int gi = i + cx, gj = j + cy, gk = z + cz;
        if (gi < 0 || gi >= nx || gj < 0 || gj >= ny || gk < 0 || gk >= nz) f[k] = R(0);
      }
    });
    R m[kNA3];
    if (!edge) {
#pragma unroll
      for (int r = 0; r < kNA3; ++r) m[r] = R(0);
      static_for<0, 19>([&](auto kk) {
        constexpr int k = decltype(kk)::value;
        constexpr int cx = c3(k, 0), cy = c3(k, 1), cz = c3(k, 2);
        const R wf = R(w3d(k)) * f[k];
        m[0] += wf;
        if constexpr (cx != 0) m[1] += R(cx) * wf;
        if constexpr (cy != 0) m[2] += R(cy) * wf;
        if constexpr (cz != 0) m[3] += R(cz) * wf;
        if constexpr (cx != 0) m[4] += wf;
        if constexpr (cx * cy != 0) m[5] += R(cx * cy) * wf;
        if constexpr (cx * cz != 0) m[6] += R(cx * cz) * wf;
        if constexpr (cy != 0) m[7] += wf;
        if constexpr (cy * cz != 0) m[8] += R(cy * cz) * wf;
        if constexpr (cz != 0) m[9] += wf;
      });
      const R* C = rc + bufC(z) * 4 * NT3 + ty * TX3 + tx;
      const R inv = C[0];
      m[1] = (m[1] + C[NT3]) * inv;
      m[2] = (m[2] + C[2 * NT3]) * inv;
      m[3] = (m[3] + C[3 * NT3]) * inv;
    } else {
      const int cls = (n0 + 1) * 9 + (n1 + 1) * 3 + (n2 + 1);
      const R* M = a.emap + cls * (kNA3 * 19);
      const R* M0 = a.emap + kClasses3 * kNA3 * 19 + cls * kNA3;  // boundary objective term
#pragma unroll
      for (int r = 0; r < kNA3; ++r) {
        R sacc = R(0);
        static_for<0, 19>([&](auto kk) {
          constexpr int k = decltype(kk)::value;
          sacc += M[r * 19 + k] * f[k];
        });
        m[r] = sacc + M0[r];
      }
    }
    const size_t o = gidx(g, i, j, z);
#pragma unroll
    for (int r = 0; r < kNA3; ++r) a.m0[r][o] = m[r];
    if (!(m[1] * m[1] + m[2] * m[2] + m[3] * m[3] < R(1e30))) raise_status(a.status, 4);
  };

  auto run = [&](auto fast_tag) {
    for (int p = pa0; p <= pa0 + 4; ++p)
      if (!waitA(p)) return false;
    if (!waitB(pb0)) return false;
    coefs(pb0, fast_tag);
    __syncthreads();
    if (pb0 + 2 <= pb_last) {  // the buffer of plane z0 - 1 is free
      if (threadIdx.x == 0) issueB(pb0 + 2);
      b_hi = pb0 + 2;
    }
    if (!waitB(z0)) return false;
    coefs(z0, fast_tag);
    __syncthreads();
    for (int z = z0; z < z1; ++z) {
      if (z + 4 <= pa_last) {
        if (threadIdx.x == 0) issueA(z + 4);
        a_hi = z + 4;
      }
      if (z + 2 <= pb_last && z + 2 > b_hi) {
        if (threadIdx.x == 0) issueB(z + 2);
        b_hi = z + 2;
      }
      if (z + 1 < z1) {
        if (threadIdx.x == 0) issueC(z + 1);
        c_hi = z + 1;
      }
      if (!waitA(z + 3) || !waitB(z + 1) || !waitC(z)) return false;
      coefs(z + 1, fast_tag);
      __syncthreads();
      gather(z, fast_tag);
      __syncthreads();
    }
    return true;
  };
  const bool ok = xyi ? run(std::true_type{}) : run(std::false_type{});
  if (!ok) drain_and_fail();
}

// ---------------------------------------------------------------------------------
// Warp-column D3Q19 steady adjoint (FP32)
// ---------------------------------------------------------------------------------
// The tiles, lanes, warps and z chunks of the warp-column forward.  The ALKS step of
// a node gathers, over its 19 links, P + c_k . V taken at the neighbour x + c_k
// (Sec. 2.5).  Here every node forms its own P, V and the 19 values P + c_k . V, and
// routes value k to x - c_k: links with c_y = 0 by shuffles along x and a register
// ring of destination planes along z, the ten others through the shared exchange
// (indexed by destination plane mod NXS3).  Only the fields with y stencils (s~xy,
// s~yy, s~yz) are staged by tensor copies; a lane loads the other fields of its own
// node (coalesced along x) a plane before it uses them.  Sources outside the lattice
// route zeros, so every exchange entry an output reads is rewritten each step.
constexpr int NAY3 = 3;  // staged fields: s~xy, s~yy, s~yz

__host__ __device__ constexpr size_t adj3c_smem() {
  return sizeof(float) * ((size_t)NSLC3 * NAY3 * CFS3 + (size_t)NXS3 * NYC3 * NXL3 * XW3 + 6 * kFillLen3) + 8 * NSLC3 +
         128;
}

struct Adj3CArgs {
  const float* own[10];  // previous level rho~, u~x, u~y, u~z, s~xx, s~xz, s~zz; frozen u, v, w
  const float* cf[4];    // 1/(1+alpha), src x, src y, src z
  float* m0[kNA3];       // adjoint at the new level
  const float* emap;
  int* status;
  int zc;  // z planes per CTA
};

// d/dx at node `at` of n from values at offsets 0, +-1, +-2 (one-sided on a face),
// the same formulas as dax.
__device__ __forceinline__ float dax_v(float f0, float fp1, float fp2, float fm1, float fm2, int at, int n) {
  if (at == 0) return (-3.f * f0 + 4.f * fp1 - fp2) * 0.5f;
  if (at == n - 1) return (3.f * f0 - 4.f * fm1 + fm2) * 0.5f;
  return (fp1 - fm1) * 0.5f;
}

__global__ void __launch_bounds__(NTC3, 2) adj3c_kernel(const __grid_constant__ Maps3F maps,
                                                        const __grid_constant__ Adj3CArgs a, Geom3 g,
                                                        Coef3<float> c) {
  using R = float;
  extern __shared__ unsigned char smem_raw3[];
  R* ring = reinterpret_cast<R*>(lks::smem_base128(smem_raw3));  // [NSLC3][NAY3][CFS3]
  R* ex = ring + NSLC3 * NAY3 * CFS3;                              // [NXS3][NYC3][NXL3][XW3]
  R* fill = ex + NXS3 * NYC3 * NXL3 * XW3;                         // [6][kFillLen3]: single-face fills
  uint64_t* bar = reinterpret_cast<uint64_t*>(fill + 6 * kFillLen3);
  if (lks::timed_out_before(a.status)) return;
  if (!lks::tma_layout_ok(ring, bar, a.status)) return;
  const int nx = g.nx, ny = g.ny, nz = g.nz;
  const int x0 = blockIdx.x * CX3, y0 = blockIdx.y * NYC3;
  const int z0 = blockIdx.z * a.zc, z1 = min(z0 + a.zc, nz);
  const int pbase = z0 - 3, plast = z1 + 2;  // planes staged: z0 - 3 .. z1 + 2
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int i = x0 - 2 + lane, j = y0 - 1 + warp;
  const int bx = lane + 2, by = warp + 1;  // the node's column and row in the staged box
  const bool out_node = lane >= 2 && lane < 2 + CX3 && i < nx && warp >= 1 && warp <= NYC3 && j < ny;
  const bool in_xy = i >= 0 && i < nx && j >= 0 && j < ny;
  // lanes 0 .. 31 and warps 0 .. NYC3 + 1 inside the lattice, lanes 1 .. 30 and all
  // warps off the x and y faces
  const bool tile_fast = x0 >= 2 && x0 + CX3 <= nx - 2 && y0 >= 2 && y0 + NYC3 <= ny - 2;
  static_assert((NSLC3 & (NSLC3 - 1)) == 0, "ring slots index by mask");
  auto slot = [&](int p) { return (p - pbase) & (NSLC3 - 1); };
  auto issue = [&](int p) {
    const int sl = slot(p);
    lks::mbar_expect_tx(&bar[sl], NAY3 * CBOX3 * 4);
    for (int f = 0; f < NAY3; ++f)
      tma_load_3d(ring + (sl * NAY3 + f) * CFS3, &maps.m[f], x0 - 4, y0 - 2, p, &bar[sl]);
  };
  int waited = pbase - 1, issued = pbase - 1;
  auto wait = [&](int p) {
    const bool ok = lks::mbar_wait(&bar[slot(p)], ((p - pbase) / NSLC3) & 1);
    if (ok) waited = p;
    return ok;
  };
  auto drain_and_fail = [&]() {
    raise_status(a.status, 6);
    if (threadIdx.x == 0)
      for (int p = waited + 1; p <= issued; ++p) lks::mbar_wait(&bar[slot(p)], ((p - pbase) / NSLC3) & 1);
  };
  if (threadIdx.x == 0) {
    for (int sl = 0; sl < NSLC3; ++sl) lks::mbar_init(&bar[sl], 1);
    lks::fence_mbar_init();
    lks::fence_proxy_async();
  }
  for (int q = threadIdx.x; q < 6 * kFillLen3; q += NTC3) fill[q] = a.emap[kClasses3 * kNA3 * 20 + q];
  __syncthreads();
  for (int p = pbase; p < pbase + NSLC3 && p <= plast; ++p) {
    if (threadIdx.x == 0) issue(p);
    issued = p;
  }
  for (int p = pbase; p <= pbase + 4 && p <= plast; ++p)
    if (!wait(p)) {
      drain_and_fail();
      return;
    }
  int zs = 2;  // ring slot of the plane z being formed; plane z + k sits in slot zs + k
  auto slk = [&](int k) { return (zs + k) & (NSLC3 - 1); };
  // staged field f (0 s~xy, 1 s~yy, 2 s~yz) of plane z + k at row dy, column dx from the node
  auto at = [&](int f, int k, int dy, int dx) {
    return ring[(slk(k) * NAY3 + f) * CFS3 + (by + dy) * CBW3 + bx + dx];
  };
  auto xslot = [&](int p, int row) { return ex + ((p & (NXS3 - 1)) * NYC3 + row) * NXL3 * XW3; };
  // a field of the node at plane p; zero outside the lattice
  auto ld = [&](const float* f, int p) { return (in_xy && p >= 0 && p < nz) ? __ldg(f + gidx(g, i, j, p)) : R(0); };
  constexpr int kOwn[8] = {0, 1, 2, 3, 4, 7, 8, 9};  // rho~, u~x, u~y, u~z, s~xx, u, v, w
  R cr[8], nr[8];  // those fields of the node at planes z and z + 1
#pragma unroll
  for (int q = 0; q < 8; ++q) cr[q] = ld(a.own[kOwn[q]], z0 - 1);
  // s~xz and s~zz of the node at planes z - 1, z, z + 1
  R xz_m = ld(a.own[5], z0 - 2), xz_c = ld(a.own[5], z0 - 1), xz_p = ld(a.own[5], z0);
  R zz_m = ld(a.own[6], z0 - 2), zz_c = ld(a.own[6], z0 - 1), zz_p = ld(a.own[6], z0);
  R Am[9], Ac[9], Ap[9];  // links with c_y = 0 arriving at planes z - 1, z, z + 1 (slot oslot3(k))
#pragma unroll
  for (int q = 0; q < 9; ++q) Am[q] = Ac[q] = Ap[q] = R(0);

  // One plane: P, V and the routed values of plane z, then the gather of plane z - 1.
  // FAST: no node of the tile at planes z and z - 1 lies on a face (all are inside).
  auto plane_step = [&](int z, auto fast_tag) {
    constexpr bool FAST = decltype(fast_tag)::value;
    const bool src = FAST || (in_xy && z >= 0 && z < nz);
#pragma unroll
    for (int q = 0; q < 8; ++q) nr[q] = ld(a.own[kOwn[q]], z + 1);
    const R xz_n = ld(a.own[5], z + 2), zz_n = ld(a.own[6], z + 2);
    const int zd = z - 1;
    const bool gat = out_node && zd >= z0 && zd < z1;
    R C[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) C[q] = gat ? ld(a.cf[q], zd) : R(0);

    // ---- P and V of node (i, j, z) ----
    const R rt = cr[0], ux = cr[1], uy = cr[2], uz = cr[3], vxx = cr[4], u0 = cr[5], u1 = cr[6], u2 = cr[7];
    const R vxy = at(0, 0, 0, 0), vyy = at(1, 0, 0, 0), vyz = at(2, 0, 0, 0), vxz = xz_c, vzz = zz_c;
    const R xx_r = __shfl_down_sync(0xffffffffu, vxx, 1), xx_l = __shfl_up_sync(0xffffffffu, vxx, 1);
    const R xz_r = __shfl_down_sync(0xffffffffu, vxz, 1), xz_l = __shfl_up_sync(0xffffffffu, vxz, 1);
    R d_xx_x = (xx_r - xx_l) * R(0.5);
    R d_xy_x = (at(0, 0, 0, 1) - at(0, 0, 0, -1)) * R(0.5);
    R d_xz_x = (xz_r - xz_l) * R(0.5);
    R d_xy_y = (at(0, 0, 1, 0) - at(0, 0, -1, 0)) * R(0.5);
    R d_yy_y = (at(1, 0, 1, 0) - at(1, 0, -1, 0)) * R(0.5);
    R d_yz_y = (at(2, 0, 1, 0) - at(2, 0, -1, 0)) * R(0.5);
    R d_xz_z = (xz_p - xz_m) * R(0.5);
    R d_yz_z = (at(2, 1, 0, 0) - at(2, -1, 0, 0)) * R(0.5);
    R d_zz_z = (zz_p - zz_m) * R(0.5);
    if constexpr (!FAST) {
      // one-sided differences on the faces (x: two lanes away, by shuffles of the whole warp)
      const R xx_r2 = __shfl_down_sync(0xffffffffu, vxx, 2), xx_l2 = __shfl_up_sync(0xffffffffu, vxx, 2);
      const R xz_r2 = __shfl_down_sync(0xffffffffu, vxz, 2), xz_l2 = __shfl_up_sync(0xffffffffu, vxz, 2);
      if (src && (i == 0 || i == nx - 1)) {
        d_xx_x = dax_v(vxx, xx_r, xx_r2, xx_l, xx_l2, i, nx);
        d_xz_x = dax_v(vxz, xz_r, xz_r2, xz_l, xz_l2, i, nx);
        d_xy_x = dax(&ring[(slk(0) * NAY3 + 0) * CFS3 + by * CBW3 + bx], 1, i, nx);
      }
      if (src && (j == 0 || j == ny - 1)) {
        d_xy_y = dax(&ring[(slk(0) * NAY3 + 0) * CFS3 + by * CBW3 + bx], CBW3, j, ny);
        d_yy_y = dax(&ring[(slk(0) * NAY3 + 1) * CFS3 + by * CBW3 + bx], CBW3, j, ny);
        d_yz_y = dax(&ring[(slk(0) * NAY3 + 2) * CFS3 + by * CBW3 + bx], CBW3, j, ny);
      }
      if (src && (z == 0 || z == nz - 1)) {
        d_xz_z = daz<R>([&](int dz) { return dz == 0 ? xz_c : dz == 1 ? xz_p : dz == -1 ? xz_m : ld(a.own[5], z + dz); },
                        z, nz);
        d_yz_z = daz<R>([&](int dz) { return at(2, dz, 0, 0); }, z, nz);
        d_zz_z = daz<R>([&](int dz) { return dz == 0 ? zz_c : dz == 1 ? zz_p : dz == -1 ? zz_m : ld(a.own[6], z + dz); },
                        z, nz);
      }
    }
    const R Dx = R(2) * (d_xx_x + d_xy_y + d_xz_z);
    const R Dy = R(2) * (d_xy_x + d_yy_y + d_yz_z);
    const R Dz = R(2) * (d_xz_x + d_yz_y + d_zz_z);
    R P = rt;
    R Vx = R(3) * (ux + R(3) * (vxx * u0 + vxy * u1 + vxz * u2) - rt * u0) - c.A * Dx;
    R Vy = R(3) * (uy + R(3) * (vxy * u0 + vyy * u1 + vyz * u2) - rt * u1) - c.A * Dy;
    R Vz = R(3) * (uz + R(3) * (vxz * u0 + vyz * u1 + vzz * u2) - rt * u2) - c.A * Dz;
    if constexpr (!FAST) {
      if (!src) P = Vx = Vy = Vz = R(0);
    }

    // ---- P + c_k . V of node (i, j, z), routed to (i, j, z) - c_k ----
    R* const xr_m = xslot(z - 1, 0) + lane - 2;  // exchange rows of the destination planes
    R* const xr_c = xslot(z, 0) + lane - 2;
    R* const xr_p = xslot(z + 1, 0) + lane - 2;
    // destination row warp - 1 - c_y and lane lane - c_x are an output row and column
    const bool r_dn = warp >= 2, r_up = warp < NYC3;
    const bool xl_r = lane >= 3 && lane <= CX3 + 2, xl_c = lane >= 2 && lane <= CX3 + 1, xl_l = lane >= 1 && lane <= CX3;
    static_for<0, 19>([&](auto kk) {
      constexpr int k = decltype(kk)::value;
      constexpr int cx = c3(k, 0), cy = c3(k, 1), cz = c3(k, 2);
      R v = P;
      if constexpr (cx != 0) v += R(cx) * Vx;
      if constexpr (cy != 0) v += R(cy) * Vy;
      if constexpr (cz != 0) v += R(cz) * Vz;
      if constexpr (cy != 0) {
        R* const xr = (cz > 0 ? xr_m : (cz == 0 ? xr_c : xr_p)) + ((cy > 0 ? -2 : 0) * NXL3 + yslot3(k)) * XW3 - cx;
        if ((cy > 0 ? r_dn : r_up) && (cx > 0 ? xl_r : (cx == 0 ? xl_c : xl_l))) xr[warp * NXL3 * XW3] = v;
      } else {
        R w;
        if constexpr (cx > 0) w = __shfl_down_sync(0xffffffffu, v, 1);  // from the lane on the right
        else if constexpr (cx < 0) w = __shfl_up_sync(0xffffffffu, v, 1);
        else w = v;
        if constexpr (cz > 0) Am[oslot3(k)] = w;
        else if constexpr (cz == 0) Ac[oslot3(k)] = w;
        else Ap[oslot3(k)] = w;
      }
    });
    __syncthreads();  // plane z's exchange writes are in; plane z - 1 is complete
    if (z + NSLC3 - 3 <= plast && z + NSLC3 - 3 > issued) {  // the slot of plane z - 3 is free
      if (threadIdx.x == 0) issue(z + NSLC3 - 3);
      issued = z + NSLC3 - 3;
    }
    // ---- gather of node (i, j, z - 1) ----
    R F[19];
    int nf = 0, cls = 0;  // faces the node lies on; its edge class
    if (gat) {
      const R* xr = xslot(zd, warp - 1) + lane - 2;
      static_for<0, 19>([&](auto kk) {
        constexpr int k = decltype(kk)::value;
        if constexpr (c3(k, 1) != 0) F[k] = xr[yslot3(k) * XW3];
        else F[k] = Am[oslot3(k)];
      });
      if constexpr (!FAST) {
        const int n0 = i == 0 ? -1 : (i == nx - 1 ? 1 : 0);
        const int n1 = j == 0 ? -1 : (j == ny - 1 ? 1 : 0);
        const int n2 = zd == 0 ? -1 : (zd == nz - 1 ? 1 : 0);
        nf = abs(n0) + abs(n1) + abs(n2);
        cls = (n0 + 1) * 9 + (n1 + 1) * 3 + (n2 + 1);
        if (nf == 1) {
          // One face: its five unknown links (c . n > 0) from the five opposite ones
          // (c . n < 0), the least-squares fill of the face rule, plus the boundary
          // objective term; the other links' columns of the rule are zero.
          const int ff = n0 != 0 ? (n0 > 0) : (n1 != 0 ? 2 + (n1 > 0) : 4 + (n2 > 0));
          static_for<0, 6>([&](auto fc) {
            constexpr int f = decltype(fc)::value;
            if (ff == f) {
              const R* X = fill + f * kFillLen3;
              R O[5];
              static_for<0, 5>([&](auto pp) {
                constexpr int p = decltype(pp)::value;
                O[p] = F[face_link3(f, p, false)];
              });
              static_for<0, 5>([&](auto qq) {
                constexpr int q = decltype(qq)::value;
                R v = X[25 + q];
#pragma unroll
                for (int p = 0; p < 5; ++p) v += X[q * 5 + p] * O[p];
                F[face_link3(f, q, true)] = v;
              });
            }
          });
        }
      }
      if (nf <= 1) {
        R m[kNA3];
        adj_moments3(F, m);
        if (nf == 0) {
          m[1] = (m[1] + C[1]) * C[0];
          m[2] = (m[2] + C[2]) * C[0];
          m[3] = (m[3] + C[3]) * C[0];
        }
        const size_t o = gidx(g, i, j, zd);
#pragma unroll
        for (int r = 0; r < kNA3; ++r) a.m0[r][o] = m[r];
        if (!(m[1] * m[1] + m[2] * m[2] + m[3] * m[3] < R(1e30))) raise_status(a.status, 4);
      }
    }
    if constexpr (!FAST) {
      // Box-edge and corner nodes apply their class's moment map (10 x 19, plus the
      // boundary objective term).  Where few lanes of the warp are such nodes, the
      // whole warp computes each one's ten moments, one row per lane, and lanes 0..9
      // store them, instead of that lane alone running the 190 products while the
      // others wait.
      unsigned fm = __ballot_sync(0xffffffffu, gat && nf >= 2);
      if (__popc(fm) > 2) {
        if (gat && nf >= 2) {
          const R* M = a.emap + cls * (kNA3 * 19);
          const R* M0 = a.emap + kClasses3 * kNA3 * 19 + cls * kNA3;  // boundary objective term
          const size_t o = gidx(g, i, j, zd);
          R u2 = R(0);
#pragma unroll
          for (int r = 0; r < kNA3; ++r) {
            R sacc = R(0);
            static_for<0, 19>([&](auto kk) {
              constexpr int k = decltype(kk)::value;
              sacc += M[r * 19 + k] * F[k];
            });
            sacc += M0[r];
            a.m0[r][o] = sacc;
            if (r >= 1 && r <= 3) u2 += sacc * sacc;
          }
          if (!(u2 < R(1e30))) raise_status(a.status, 4);
        }
      } else {
        const int row = lane < kNA3 ? lane : kNA3 - 1;
        while (fm) {
          const int srcl = __ffs(fm) - 1;
          fm &= fm - 1;
          const int cs = __shfl_sync(0xffffffffu, cls, srcl);
          const R* M = a.emap + (cs * kNA3 + row) * 19;
          R sacc = R(0);
          static_for<0, 19>([&](auto kk) {
            constexpr int k = decltype(kk)::value;
            sacc += M[k] * __shfl_sync(0xffffffffu, F[k], srcl);
          });
          sacc += a.emap[kClasses3 * kNA3 * 19 + cs * kNA3 + row];
          if (lane < kNA3) {
            a.m0[lane][gidx(g, x0 - 2 + srcl, j, zd)] = sacc;
            if (lane >= 1 && lane <= 3 && !(sacc * sacc < R(1e30))) raise_status(a.status, 4);
          }
        }
      }
    }
    // ---- rotate ----
#pragma unroll
    for (int q = 0; q < 9; ++q) {
      Am[q] = Ac[q];
      Ac[q] = Ap[q];
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) cr[q] = nr[q];
    xz_m = xz_c, xz_c = xz_p, xz_p = xz_n;
    zz_m = zz_c, zz_c = zz_p, zz_p = zz_n;
    zs = (zs + 1) & (NSLC3 - 1);
  };

  for (int z = z0 - 1; z <= z1; ++z) {
    if (z + 2 <= plast && z + 2 > waited && !wait(z + 2)) {
      drain_and_fail();
      return;
    }
    if (tile_fast && z >= 2 && z <= nz - 2) plane_step(z, std::true_type{});
    else plane_step(z, std::false_type{});
  }
}

// ---------------------------------------------------------------------------------
// Paired-column D3Q19 forward (FP32)
// ---------------------------------------------------------------------------------
// The tiles (CX3 x NYC3 outputs), z chunks, staged boxes and exchange protocol of
// the warp-column adjoint, with two nodes per lane and two rows per warp:
//   - a lane owns an even column and the odd one after it (pair q of a half-warp owns
//     columns x0 - 2 + 2q and x0 - 1 + 2q; pairs 1..14 write, 28 columns);
//   - warp w owns rows y0 - 1 + 2w (lanes 0..15, the upper row) and y0 + 2w (lanes
//     16..31); rows y0 .. y0 + NYC3 - 1 are outputs, the first warp's upper row and
//     the last warp's lower row are halo.
// Both nodes of a lane run as packed FP32 pairs (one f32x2 instruction for the two),
// a node pair is loaded and stored as one 8-byte vector, and the per-lane work of the
// plane loop (addresses, tests, rings) is shared by two nodes.  A routed value stays
// in the lane between the pair's columns, moves by one shuffle between the lanes of
// a row and by shuffles across the half-warps between the warp's two rows; only the
// five links that leave the warp (one sign of c_y per row) pass through the shared
// exchange.
// Tiles of the paired forward: CX3 x NYP3 outputs (taller than the adjoint's NYC3,
// so that the two halo rows are a smaller share), boxes CBW3 x PBH3.
constexpr int NYP3 = 12, NWP3 = NYP3 / 2 + 1, NTP3 = 32 * NWP3;
constexpr int PBH3 = NYP3 + 4, PBOX3 = CBW3 * PBH3;
constexpr int PFS3 = (PBOX3 * 4 + 127) / 128 * 128 / 4;  // field stride in a ring slot (128-byte multiple)
// Plane ring of the paired forward: planes z - 2 .. z + 5 (eight slots).
constexpr int NSLP3 = 8;
static_assert((NSLP3 & (NSLP3 - 1)) == 0, "ring slots index by mask");
static_assert(2 * NWP3 == NYP3 + 2, "two rows per warp, one halo row above and below the tile");
static_assert(CX3 % 2 == 0 && XW3 % 2 == 0 && PFS3 % 2 == 0 && CBW3 % 2 == 0, "node pairs are 8-byte aligned");
constexpr unsigned kFull3 = 0xffffffffu;
// Links with c_y != 0 in classes by (c_x, c_z), two links (c_y = +1, -1) each:
// 0: (0, 0), 1: (1, 0), 2: (-1, 0), 3: (0, 1), 4: (0, -1).
constexpr int NCB3 = 5;
__host__ __device__ constexpr int cbx3(int b) { return b == 1 ? 1 : (b == 2 ? -1 : 0); }
__host__ __device__ constexpr int cbz3(int b) { return b == 3 ? 1 : (b == 4 ? -1 : 0); }
__host__ __device__ constexpr int cls_of3(int cx, int cz) { return cz == 0 ? (cx == 0 ? 0 : (cx > 0 ? 1 : 2)) : (cz > 0 ? 3 : 4); }
// Register slots of the values a node keeps for one destination plane (the links that
// stay in the warp), grouped by c_z of the link:
//   c_z = 0:  links (0,0,0), (1,0,0), (-1,0,0), classes 0, 1, 2 from the other row
//   c_z = +1: links (0,0,1), (1,0,1), (-1,0,1), class 3
//   c_z = -1: links (0,0,-1), (1,0,-1), (-1,0,-1), class 4
constexpr int NRS3 = 14;
__host__ __device__ constexpr int rs3(int cx, int cz) { return (cz == 0 ? 0 : (cz > 0 ? 6 : 10)) + (cx == 0 ? 0 : (cx > 0 ? 1 : 2)); }
__host__ __device__ constexpr int rsb3(int b) { return b <= 2 ? 3 + b : (b == 3 ? 9 : 13); }

using F2 = float2;
__device__ __forceinline__ F2 p2(float a) { return make_float2(a, a); }
__device__ __forceinline__ F2 add2(F2 a, F2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ F2 sub2(F2 a, F2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ F2 mul2(F2 a, F2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ F2 fma2(F2 a, F2 b, F2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ F2 zero2() { return make_float2(0.f, 0.f); }
template <int C>
__device__ __forceinline__ float& cmp2(F2& v) {
  if constexpr (C == 0) return v.x;
  else return v.y;
}
template <int C>
__device__ __forceinline__ float cmp2(const F2& v) {
  if constexpr (C == 0) return v.x;
  else return v.y;
}
__device__ __forceinline__ F2 ld2s(const float* p) { return *reinterpret_cast<const F2*>(p); }
__device__ __forceinline__ void st2s(float* p, F2 v) { *reinterpret_cast<F2*>(p) = v; }

// At each column c of the pair, v taken at column c + CX of the same row.
template <int CX>
__device__ __forceinline__ F2 recv_x3(F2 v) {
  if constexpr (CX > 0) return make_float2(v.y, __shfl_down_sync(kFull3, v.x, 1));
  else if constexpr (CX < 0) return make_float2(__shfl_up_sync(kFull3, v.y, 1), v.x);
  else return v;
}
// At each column c of the pair, v taken at column c + CX of the warp's other row
// (oth: the lane of the same pair in that row).
template <int CX>
__device__ __forceinline__ F2 recv_xo3(F2 v, int oth) {
  if constexpr (CX > 0) return make_float2(__shfl_sync(kFull3, v.y, oth), __shfl_sync(kFull3, v.x, oth + 1));
  else if constexpr (CX < 0) return make_float2(__shfl_sync(kFull3, v.y, oth - 1), __shfl_sync(kFull3, v.x, oth));
  else return make_float2(__shfl_sync(kFull3, v.x, oth), __shfl_sync(kFull3, v.y, oth));
}

// Class sums of the values a node pair gathered (interior rule), the groupings of
// adj_moments3: the links with c_y = 0 by slot, and per y class b the
// sum S_b = F(c_y = +1) + F(c_y = -1) and difference D_b = F(c_y = +1) - F(c_y = -1).
struct ClassSums3 {
  F2 F000, ax, dx, az, dz, e1, e2, f1, f2;
};
__device__ __forceinline__ ClassSums3 class_sums3(const F2 (&A)[NRS3]) {
  ClassSums3 s;
  const F2 Fp00 = A[rs3(1, 0)], Fm00 = A[rs3(-1, 0)], F00p = A[rs3(0, 1)], F00m = A[rs3(0, -1)];
  const F2 Fp0p = A[rs3(1, 1)], Fm0p = A[rs3(-1, 1)], Fp0m = A[rs3(1, -1)], Fm0m = A[rs3(-1, -1)];
  s.F000 = A[rs3(0, 0)];
  s.ax = add2(Fp00, Fm00);
  s.dx = sub2(Fp00, Fm00);
  s.az = add2(F00p, F00m);
  s.dz = sub2(F00p, F00m);
  s.e1 = add2(Fp0p, Fm0m);  // xz diagonals with c_x c_z = +1
  s.e2 = add2(Fp0m, Fm0p);  // and with c_x c_z = -1
  s.f1 = sub2(Fp0p, Fm0m);
  s.f2 = sub2(Fp0m, Fm0p);
  return s;
}
// The 19 gathered values of component C of the pair in link order (the face rules);
// Fp[b] / Fm[b] are class b's links with c_y = +1 / -1.
template <int C>
__device__ __forceinline__ void gathered19(const F2 (&A)[NRS3], const F2 (&Fp)[NCB3], const F2 (&Fm)[NCB3],
                                           float (&F)[19]) {
  static_for<0, 19>([&](auto kk) {
    constexpr int k = decltype(kk)::value;
    constexpr int cx = c3(k, 0), cy = c3(k, 1), cz = c3(k, 2);
    if constexpr (cy == 0) F[k] = cmp2<C>(A[rs3(cx, cz)]);
    else if constexpr (cy > 0) F[k] = cmp2<C>(Fp[cls_of3(cx, cz)]);
    else F[k] = cmp2<C>(Fm[cls_of3(cx, cz)]);
  });
}

// Paired-column forward.  Every node pair computes its 19 pushed values
// P_k = w_k [base + c_k.b + c_k c_k : Q] (Eq. feq2 with base = drho + e0, b = 3u and
// Q the coefficients of c_a c_b, each off-diagonal entry counted once), by link
// pair: opposite links share w (base + Q) and differ by the sign of w c_k.b, the four
// diagonal links of an axis pair share w (base + Q_aa + Q_bb) and split by the sign
// of Q_ab.  Summed over the links a destination receives, these give rho and u*
// directly.  Value k is routed to x + c_k: the links with c_y = 0
// inside the row, one sign of c_y to the warp's other row by shuffles (the upper row
// sends c_y = +1, the lower row c_y = -1), the other sign through the exchange.
// drho, u, v, w of each plane arrive by tensor copies into the ring; 1/(1+alpha) of
// an output pair is one 8-byte load, a plane ahead.
__host__ __device__ constexpr size_t fwd3p_smem() {
  return sizeof(float) * ((size_t)NSLP3 * NFC3 * PFS3 + (size_t)NXS3 * NYP3 * NCB3 * XW3) + 8 * NSLP3 + 128;
}

__global__ void __launch_bounds__(NTP3, 2) fwd3p_kernel(const __grid_constant__ Maps3F maps,
                                                        const __grid_constant__ Fwd3TArgs a, Geom3 g,
                                                        Coef3<float> c) {
  using R = float;
  extern __shared__ unsigned char smem_raw3[];
  R* ring = reinterpret_cast<R*>(lks::smem_base128(smem_raw3));  // [NSLP3][NFC3][PFS3]
  R* ex = ring + NSLP3 * NFC3 * PFS3;                              // [NXS3][NYP3][NCB3][XW3]
  uint64_t* bar = reinterpret_cast<uint64_t*>(ex + NXS3 * NYP3 * NCB3 * XW3);
  if (lks::timed_out_before(a.status)) return;
  if (!lks::tma_layout_ok(ring, bar, a.status)) return;
  const int nx = g.nx, ny = g.ny, nz = g.nz;
  const int x0 = blockIdx.x * CX3, y0 = blockIdx.y * NYP3;
  const int z0 = blockIdx.z * a.zc, z1 = min(z0 + a.zc, nz);
  const int pbase = z0 - 3, plast = z1 + 2;  // planes staged: z0 - 3 .. z1 + 2
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int h = lane >> 4, q = lane & 15, t = 2 * warp + h;
  const int i0 = x0 - 2 + 2 * q, j = y0 - 1 + t;
  const int bx = 2 + 2 * q, by = 1 + t;
  const int xl = 2 * q - 2;
  const int oth = lane ^ 16;
  const bool in_xy = i0 >= 0 && i0 < nx && j >= 0 && j < ny;
  const bool out_node = q >= 1 && q <= 14 && i0 < nx && t >= 1 && t <= NYP3 && j < ny;
  const bool tile_fast = x0 >= 2 && x0 + CX3 <= nx - 2 && y0 >= 2 && y0 + NYP3 <= ny - 2;
  // every lane's row, and every row whose push it reads, is off the y faces
  const bool tile_yfast = y0 >= 2 && y0 + NYP3 <= ny - 2;
  // sent inside the warp: the class value with c_y = +1 (upper row) / -1 (lower row)
  const F2 sy2 = p2(h ? -1.f : 1.f);
  auto slot = [&](int p) { return (p - pbase) & (NSLP3 - 1); };
  auto issue = [&](int p) {
    const int sl = slot(p);
    lks::mbar_expect_tx(&bar[sl], NFC3 * PBOX3 * 4);
    for (int f = 0; f < NFC3; ++f)
      tma_load_3d(ring + (sl * NFC3 + f) * PFS3, &maps.m[f], x0 - 4, y0 - 2, p, &bar[sl]);
  };
  int waited = pbase - 1, issued = pbase - 1;
  auto wait = [&](int p) {
    const bool ok = lks::mbar_wait(&bar[slot(p)], ((p - pbase) / NSLP3) & 1);
    if (ok) waited = p;
    return ok;
  };
  auto drain_and_fail = [&]() {
    raise_status(a.status, 6);
    if (threadIdx.x == 0)
      for (int p = waited + 1; p <= issued; ++p) lks::mbar_wait(&bar[slot(p)], ((p - pbase) / NSLP3) & 1);
  };
  if (threadIdx.x == 0) {
    for (int sl = 0; sl < NSLP3; ++sl) lks::mbar_init(&bar[sl], 1);
    lks::fence_mbar_init();
    lks::fence_proxy_async();
  }
  __syncthreads();
  for (int p = pbase; p < pbase + NSLP3 && p <= plast; ++p) {
    if (threadIdx.x == 0) issue(p);
    issued = p;
  }
  for (int p = pbase; p <= pbase + 4 && p <= plast; ++p)
    if (!wait(p)) {
      drain_and_fail();
      return;
    }
  int zs = 2;  // ring slot of the plane z being pushed; plane z + k sits in slot zs + k
  auto slk = [&](int k) { return (zs + k) & (NSLP3 - 1); };
  // field f (0 drho, 1 u, 2 v, 3 w) of plane z + k at row offset dy, the pair's even column
  auto fp = [&](int f, int k, int dy) { return ring + (slk(k) * NFC3 + f) * PFS3 + (by + dy) * CBW3 + bx; };
  auto at2 = [&](int f, int k, int dy) { return ld2s(fp(f, k, dy)); };
  auto xrow = [&](int p, int od) { return ex + ((p & (NXS3 - 1)) * NYP3 + od) * (NCB3 * XW3); };
  // 1/(1+alpha) of the output pair at plane p (loaded one plane before the gather reads it)
  auto binv_at = [&](int p) {
    return (out_node && p >= 0 && p < nz) ? __ldg(reinterpret_cast<const float2*>(a.binv + gidx(g, i0, j, p)))
                                          : zero2();
  };
  F2 inv_n = binv_at(z0 - 1);
  // the pair's u, v, w at planes z - 1 (m), z (c), z + 1 (p), and drho at z and z + 1
  F2 Am[NRS3], Ac[NRS3], Ap[NRS3];  // values for the destination planes z - 1, z, z + 1
#pragma unroll
  for (int s = 0; s < NRS3; ++s) Am[s] = Ac[s] = Ap[s] = zero2();

  // One plane: push of plane z, then gather of plane z - 1.  MODE 0 (fast): no node
  // of the tile at planes z and z - 1 lies on a face (all are inside); MODE 1: only
  // the x faces can occur (rows and planes are off the y and z faces); MODE 2: any.
  auto plane_step = [&](int z, auto mode_tag) {
    constexpr int MODE = decltype(mode_tag)::value;
    constexpr bool FAST = MODE == 0, XO = MODE == 1;
    const bool src = FAST || (XO ? (i0 >= 0 && i0 < nx) : (in_xy && z >= 0 && z < nz));
    // the pair's drho, u, v, w at plane z (staged; planes z - 1 and z + 1 are read
    // where the z differences need them)
    const F2 dc = at2(0, 0, 0), uc = at2(1, 0, 0), vc = at2(2, 0, 0), wc = at2(3, 0, 0);
    // velocity gradient, g[d][a] = f(x + e_a) - f(x - e_a) of u_d (twice d u_d / d x_a)
    F2 gr[3][3];
    {
      const F2 uvw[3] = {uc, vc, wc};
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const float l = __shfl_up_sync(kFull3, uvw[d].y, 1), r = __shfl_down_sync(kFull3, uvw[d].x, 1);
        gr[d][0].x = uvw[d].y - l;
        gr[d][0].y = r - uvw[d].x;
        gr[d][1] = sub2(at2(1 + d, 0, 1), at2(1 + d, 0, -1));
        gr[d][2] = sub2(at2(1 + d, 1, 0), at2(1 + d, -1, 0));
      }
    }
    if constexpr (!FAST) {
      // faces: one-sided differences, then continuity (one face: the normal derivative
      // of the normal velocity; two or more: zero normal derivatives)
      static_for<0, 2>([&](auto cc) {
        constexpr int CC = decltype(cc)::value;
        const int i = i0 + CC;
        const bool on[3] = {i == 0 || i == nx - 1, !XO && (j == 0 || j == ny - 1), !XO && (z == 0 || z == nz - 1)};
        if (src && (on[0] || on[1] || on[2])) {
#pragma unroll
          for (int d = 0; d < 3; ++d) {
            const R* f0 = fp(1 + d, 0, 0) + CC;
            if (on[0]) {
              const int s = i == 0 ? 1 : -1;
              cmp2<CC>(gr[d][0]) = (float)s * ((4.f * f0[s] - 3.f * f0[0]) - f0[2 * s]);
            }
            if (on[1]) {
              const int s = j == 0 ? 1 : -1;
              cmp2<CC>(gr[d][1]) = (float)s * ((4.f * f0[s * CBW3] - 3.f * f0[0]) - f0[2 * s * CBW3]);
            }
            if (on[2]) {
              const int s = z == 0 ? 1 : -1;
              cmp2<CC>(gr[d][2]) = (float)s * ((4.f * fp(1 + d, s, 0)[CC] - 3.f * f0[0]) - fp(1 + d, 2 * s, 0)[CC]);
            }
          }
          const int faces = (int)on[0] + (int)on[1] + (int)on[2];
          if (faces == 1) {
            if (on[0]) cmp2<CC>(gr[0][0]) = -(cmp2<CC>(gr[1][1]) + cmp2<CC>(gr[2][2]));
            else if (on[1]) cmp2<CC>(gr[1][1]) = -(cmp2<CC>(gr[0][0]) + cmp2<CC>(gr[2][2]));
            else cmp2<CC>(gr[2][2]) = -(cmp2<CC>(gr[0][0]) + cmp2<CC>(gr[1][1]));
          } else {
#pragma unroll
            for (int d = 0; d < 3; ++d)
              if (on[d]) cmp2<CC>(gr[d][d]) = 0.f;
          }
        }
      });
    }
    // Eq. feq2: base = drho + e0 with e0 = -3/2 |u|^2, b = 3u,
    // Q_aa = 9/2 u_a^2 + A (2 d_a u_a), Q_ab = 9 u_a u_b + 2A (d_b u_a + d_a u_b)
    const F2 A2 = p2(c.A);
    const F2 uu = mul2(uc, uc), vv = mul2(vc, vc), ww = mul2(wc, wc);
    F2 bs = fma2(p2(-1.5f), add2(add2(uu, vv), ww), dc);
    F2 Qxx = fma2(p2(4.5f), uu, mul2(A2, gr[0][0]));
    F2 Qyy = fma2(p2(4.5f), vv, mul2(A2, gr[1][1]));
    F2 Qzz = fma2(p2(4.5f), ww, mul2(A2, gr[2][2]));
    F2 Qxy = fma2(p2(9.f), mul2(uc, vc), mul2(A2, add2(gr[0][1], gr[1][0])));
    F2 Qxz = fma2(p2(9.f), mul2(uc, wc), mul2(A2, add2(gr[0][2], gr[2][0])));
    F2 Qyz = fma2(p2(9.f), mul2(vc, wc), mul2(A2, add2(gr[1][2], gr[2][1])));
    F2 bxv = uc, byv = vc, bzv = wc;  // b / 3
    if constexpr (!FAST) {
      if (!src) bs = Qxx = Qyy = Qzz = Qxy = Qxz = Qyz = bxv = byv = bzv = zero2();
    }
    // pushed values by link pair: w1 b = u / 6, w2 b = w1 b / 2
    const F2 w0 = p2((float)w3d(0)), w1 = p2((float)w3d(1)), w2 = p2((float)w3d(7));
    const F2 w1b = mul2(w1, bs), w2b = mul2(w2, bs);
    const F2 b1x = mul2(p2(3.f * (float)w3d(1)), bxv), b1y = mul2(p2(3.f * (float)w3d(1)), byv),
             b1z = mul2(p2(3.f * (float)w3d(1)), bzv);
    const F2 b2x = mul2(p2(0.5f), b1x), b2y = mul2(p2(0.5f), b1y), b2z = mul2(p2(0.5f), b1z);
    const F2 tX = fma2(w1, Qxx, w1b), tY = fma2(w1, Qyy, w1b), tZ = fma2(w1, Qzz, w1b);
    const F2 dXZ = fma2(w2, add2(Qxx, Qzz), w2b), qXZ = mul2(w2, Qxz);
    const F2 dXY = fma2(w2, add2(Qxx, Qyy), w2b), qXY = mul2(w2, Qxy);
    const F2 dYZ = fma2(w2, add2(Qyy, Qzz), w2b), qYZ = mul2(w2, Qyz);
    // links with c_y = 0 (value at x goes to x + c): c_z = 0 to plane z, +1 to z + 1, -1 to z - 1
    {
      const F2 sp = add2(dXZ, qXZ), sm = sub2(dXZ, qXZ), c1 = add2(b2x, b2z), c2 = sub2(b2x, b2z);
      Ac[rs3(0, 0)] = mul2(w0, bs);
      Ac[rs3(1, 0)] = recv_x3<-1>(add2(tX, b1x));
      Ac[rs3(-1, 0)] = recv_x3<1>(sub2(tX, b1x));
      Ap[rs3(0, 1)] = add2(tZ, b1z);
      Am[rs3(0, -1)] = sub2(tZ, b1z);
      Ap[rs3(1, 1)] = recv_x3<-1>(add2(sp, c1));   // (1, 0, 1)
      Am[rs3(-1, -1)] = recv_x3<1>(sub2(sp, c1));  // (-1, 0, -1)
      Am[rs3(1, -1)] = recv_x3<-1>(add2(sm, c2));  // (1, 0, -1)
      Ap[rs3(-1, 1)] = recv_x3<1>(sub2(sm, c2));   // (-1, 0, 1)
    }
    // y classes: P(c_x, +-1, c_z) = G_b +- H_b; one sign to the other row, the other
    // through the exchange
    const F2 G[NCB3] = {tY, add2(dXY, b2x), sub2(dXY, b2x), add2(dYZ, b2z), sub2(dYZ, b2z)};
    const F2 sb1y = mul2(sy2, b1y), sb2y = mul2(sy2, b2y), sqxy = mul2(sy2, qXY), sqyz = mul2(sy2, qYZ);
    const F2 sH[NCB3] = {sb1y, add2(sb2y, sqxy), sub2(sb2y, sqxy), add2(sb2y, sqyz), sub2(sb2y, sqyz)};
    const int td = h ? t + 1 : t - 1;  // destination row (in the tile) of the exchanged links
    const bool xw = td >= 1 && td <= NYP3;
    static_for<0, NCB3>([&](auto bb) {
      constexpr int b = decltype(bb)::value, cx = cbx3(b), cz = cbz3(b);
      const F2 r = recv_xo3<-cx>(add2(G[b], sH[b]), oth);
      if constexpr (cz == 0) Ac[rsb3(b)] = r;
      else if constexpr (cz > 0) Ap[rsb3(b)] = r;
      else Am[rsb3(b)] = r;
      const F2 v = sub2(G[b], sH[b]);
      R* const row = xrow(z + cz, td - 1) + b * XW3;
      if (xw) {
        if constexpr (cx == 0) {
          if (q >= 1 && q <= 14) st2s(row + xl, v);
        } else {
          const int d0 = xl + cx;  // destination column of the even column
          if (d0 >= 0 && d0 < XW3) row[d0] = v.x;
          if (d0 + 1 >= 0 && d0 + 1 < XW3) row[d0 + 1] = v.y;
        }
      }
    });
    const F2 inv_c = inv_n;  // 1/(1+alpha) of the pair at plane z - 1
    inv_n = binv_at(z);
    __syncthreads();  // plane z's exchange writes are in; plane z - 1 is complete
    if (z + NSLP3 - 3 <= plast && z + NSLP3 - 3 > issued) {  // the slot of plane z - 3 is free
      if (threadIdx.x == 0) issue(z + NSLP3 - 3);
      issued = z + NSLP3 - 3;
    }
    // ---- gather of the pair at plane z - 1 ----
    const int zd = z - 1;
    if (out_node && zd >= z0 && zd < z1) {
      const R* xr = xrow(zd, t - 1) + xl;
      F2 E[NCB3], S[NCB3], D[NCB3];
      static_for<0, NCB3>([&](auto bb) {
        constexpr int b = decltype(bb)::value;
        E[b] = ld2s(xr + b * XW3);
        S[b] = add2(Am[rsb3(b)], E[b]);
        D[b] = sub2(E[b], Am[rsb3(b)]);  // the upper row's F(+1) - F(-1); the lower row's negative
      });
      const ClassSums3 s = class_sums3(Am);
      F2 drn = add2(add2(add2(s.F000, add2(s.ax, s.az)), add2(s.e1, s.e2)),
                    add2(add2(S[0], add2(S[1], S[2])), add2(S[3], S[4])));
      const F2 ysg = p2(h ? -1.f : 1.f);
      F2 uo0 = mul2(add2(add2(s.dx, add2(s.f1, s.f2)), sub2(S[1], S[2])), inv_c);
      F2 uo1 = mul2(mul2(ysg, add2(add2(D[0], add2(D[1], D[2])), add2(D[3], D[4]))), inv_c);
      F2 uo2 = mul2(add2(add2(s.dz, sub2(s.f1, s.f2)), sub2(S[3], S[4])), inv_c);
      if constexpr (!FAST) {
        F2 Fp[NCB3], Fm[NCB3];
#pragma unroll
        for (int b = 0; b < NCB3; ++b) {
          Fp[b] = h ? Am[rsb3(b)] : E[b];
          Fm[b] = h ? E[b] : Am[rsb3(b)];
        }
        static_for<0, 2>([&](auto cc) {
          constexpr int CC = decltype(cc)::value;
          const int i = i0 + CC;
          const int n0 = i == 0 ? -1 : (i == nx - 1 ? 1 : 0);
          const int n1 = XO ? 0 : (j == 0 ? -1 : (j == ny - 1 ? 1 : 0));
          const int n2 = XO ? 0 : (zd == 0 ? -1 : (zd == nz - 1 ? 1 : 0));
          const int faces = abs(n0) + abs(n1) + abs(n2);
          if (faces >= 2) {
            // wall edge or corner: density from the node one step inward along the
            // side-wall normals, no velocity
            const int jn = (j == 0) ? 1 : (j == ny - 1 ? -1 : 0);
            const int kn = (zd == 0) ? 1 : (zd == nz - 1 ? -1 : 0);
            cmp2<CC>(drn) = fp(0, kn - 1, jn)[CC];
            cmp2<CC>(uo0) = cmp2<CC>(uo1) = cmp2<CC>(uo2) = 0.f;
          } else if (faces == 1) {
            float F[19];
            gathered19<CC>(Am, Fp, Fm, F);
            R s0, sp;
            if (n0 != 0) face_sums3<0>(F, n0, s0, sp);
            else if (n1 != 0) face_sums3<1>(F, n1, s0, sp);
            else face_sums3<2>(F, n2, s0, sp);
            R u0 = 0.f;
            R dr;
            // the known populations' weights in s0 + 2 sp sum to one, so the pushed
            // values give rho directly
            if (n0 == 1) {
              dr = c.drho_out;
              u0 = (s0 + R(2) * sp) - c.drho_out;
            } else {
              if (n0 == -1) {  // inlet profile in FP32
                const float y = (float)j / (float)(ny - 1), zz = (float)zd / (float)(nz - 1);
                u0 = ((float)c.u_max * 16.f) * (y * (1.f - y)) * (zz * (1.f - zz));
              }
              dr = (s0 + R(2) * sp) - u0 * R(n0);
            }
            cmp2<CC>(drn) = dr;
            cmp2<CC>(uo0) = u0;
            cmp2<CC>(uo1) = cmp2<CC>(uo2) = 0.f;
          }
        });
      }
      const size_t o = gidx(g, i0, j, zd);
      st2s(a.out[0] + o, drn);
      st2s(a.out[1] + o, uo0);
      st2s(a.out[2] + o, uo1);
      st2s(a.out[3] + o, uo2);
      const F2 m = fma2(uo0, uo0, fma2(uo1, uo1, mul2(uo2, uo2)));
      if (!(m.x <= R(0.25)) || !(m.y <= R(0.25))) raise_status(a.status, 4);
    }
    // ---- rotate: the destination sets and the pair's planes ----
#pragma unroll
    for (int s = 0; s < NRS3; ++s) {
      Am[s] = Ac[s];
      Ac[s] = Ap[s];
    }
    zs = (zs + 1) & (NSLP3 - 1);
  };

  for (int z = z0 - 1; z <= z1; ++z) {
    if (z + 2 <= plast && z + 2 > waited && !wait(z + 2)) {
      drain_and_fail();
      return;
    }
    const bool zin = z >= 2 && z <= nz - 2;
    if (tile_fast && zin) plane_step(z, std::integral_constant<int, 0>{});
    else if (tile_yfast && zin) plane_step(z, std::integral_constant<int, 1>{});
    else plane_step(z, std::integral_constant<int, 2>{});
  }
}

// ------------------------------------------------------------------------------------
// Pointwise kernels: material, objective source, objective, sensitivity
// ------------------------------------------------------------------------------------
template <typename R>
__device__ __forceinline__ bool interior3(const Geom3& g, int i, int j, int k) {
  return i > 0 && j > 0 && k > 0 && i < g.nx - 1 && j < g.ny - 1 && k < g.nz - 1;
}
// S_ab = du_a/dx_b + du_b/dx_a at an interior node (central differences).
template <typename R>
__device__ __forceinline__ R strain3(const R* const* u, const Geom3& g, int i, int j, int k, int a, int b) {
  const size_t o = gidx(g, i, j, k);
  const size_t st[3] = {1, (size_t)g.nx, (size_t)g.nx * g.ny};
  return (u[a][o + st[b]] - u[a][o - st[b]]) * R(0.5) + (u[b][o + st[a]] - u[b][o - st[a]]) * R(0.5);
}

// binv = 1/(1+alpha) and src_a = -(1/3) dJ_O/du_a of the frozen state:
//   dJ_O/du_a = nu sum_d [S_ad(x - e_d) - S_ad(x + e_d)] (interior neighbours)
//               + 2 alpha u_a (interior x).
template <typename R>
__global__ void src3_kernel(const R* __restrict__ gamma, const R* u0, const R* u1, const R* u2, Geom3 g, Coef3<R> c,
                            R* __restrict__ binv, R* __restrict__ s0, R* __restrict__ s1, R* __restrict__ s2) {
  const R* u[3] = {u0, u1, u2};
  R* s[3] = {s0, s1, s2};
  const size_t N = (size_t)g.nx * g.ny * g.nz;
  for (size_t o = (size_t)blockIdx.x * blockDim.x + threadIdx.x; o < N; o += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(o % g.nx), j = (int)((o / g.nx) % g.ny), k = (int)(o / ((size_t)g.nx * g.ny));
    const R al = alpha3(c, gamma[o]);
    binv[o] = R(1) / (R(1) + al);
    const bool in = interior3<R>(g, i, j, k);
    for (int aa = 0; aa < 3; ++aa) {
      R acc = R(0);
      for (int d = 0; d < 3; ++d) {
        const int di = d == 0, dj = d == 1, dk = d == 2;
        if (interior3<R>(g, i - di, j - dj, k - dk)) acc += strain3(u, g, i - di, j - dj, k - dk, aa, d);
        if (interior3<R>(g, i + di, j + dj, k + dk)) acc -= strain3(u, g, i + di, j + dj, k + dk, aa, d);
      }
      acc *= c.nu;
      if (in) acc += R(2) * al * u[aa][o];
      s[aa][o] = -acc / R(3);
    }
  }
}

template <typename R>
__global__ void __launch_bounds__(NTHREADS) objective3_kernel(const R* __restrict__ gamma, const R* drho, const R* u0,
                                                              const R* u1, const R* u2, Geom3 g, Coef3<R> c,
                                                              double* partial) {
  __shared__ double red[NTHREADS / 32];
  const R* u[3] = {u0, u1, u2};
  const size_t N = (size_t)g.nx * g.ny * g.nz;
  double acc = 0.0;
  for (size_t o = (size_t)blockIdx.x * NTHREADS + threadIdx.x; o < N; o += (size_t)gridDim.x * NTHREADS) {
    const int i = (int)(o % g.nx), j = (int)((o / g.nx) % g.ny), k = (int)(o / ((size_t)g.nx * g.ny));
    if (!interior3<R>(g, i, j, k)) {
      // static pressure drop (Eq. objective_pipebend, p = rho / 3, dGamma = 1) over
      // the inlet and outlet nodes on one face only; the unit densities cancel
      if (c.kappa_p != 0.0 && (i == 0 || i == g.nx - 1) && j > 0 && j < g.ny - 1 && k > 0 && k < g.nz - 1)
        acc += (i == 0 ? c.kappa_p : -c.kappa_p) * (double)drho[o] / 3.0;
      continue;
    }
    R SS = R(0), uu = R(0);
    for (int aa = 0; aa < 3; ++aa) {
      uu += u[aa][o] * u[aa][o];
      for (int b = 0; b < 3; ++b) {
        const R s = strain3(u, g, i, j, k, aa, b);
        SS += s * s;
      }
    }
    acc += (double)(R(0.5) * c.nu * SS + alpha3(c, gamma[o]) * uu);
  }
  const double s = block_sum(acc, red);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

// dJ/dgamma of the steady state: alpha' |u|^2 + 3 alpha' u.u~ at interior nodes.
template <typename R>
__global__ void sens3_kernel(const R* __restrict__ gamma, const R* u0, const R* u1, const R* u2, const R* a1,
                             const R* a2, const R* a3, Geom3 g, Coef3<R> c, R* __restrict__ out) {
  const size_t N = (size_t)g.nx * g.ny * g.nz;
  for (size_t o = (size_t)blockIdx.x * blockDim.x + threadIdx.x; o < N; o += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(o % g.nx), j = (int)((o / g.nx) % g.ny), k = (int)(o / ((size_t)g.nx * g.ny));
    R s = R(0);
    if (interior3<R>(g, i, j, k)) {
      const R da = dalpha3(c, gamma[o]);
      const R x = u0[o], y = u1[o], z = u2[o];
      s = da * (x * x + y * y + z * z) + R(3) * da * (x * a1[o] + y * a2[o] + z * a3[o]);
    }
    out[o] = s;
  }
}

// ------------------------------------------------------------------------------------
// Host side
// ------------------------------------------------------------------------------------
namespace {

size_t up256(size_t x) { return (x + 255) / 256 * 256; }

template <typename R>
Coef3<R> coef3(const lks_problem_desc& d) {
  Coef3<R> c;
  c.A = (R)((1.0 / 6.0 - d.nu) * 4.5);
  c.nu = (R)d.nu;
  c.alpha_bar = (R)d.alpha_bar;
  c.q_alpha = (R)d.q_alpha;
  c.drho_out = (R)(d.rho_out - 1.0);
  c.u_max = d.u_max;
  c.kappa_p = d.kappa_p;
  return c;
}
Geom3 geom3(const lks_problem_desc& d) { return Geom3{d.nx, d.ny, d.nz}; }

lks_status fail3(const Ctx3& c, lks_status s, const std::string& m) {
  if (c.err) *c.err = m;
  return s;
}
#define CK3(c, call)                                                                      \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess)                                                                \
      return fail3(c, LKS_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

template <typename R>
R* fld3(const Ctx3& c, size_t off, int k = 0) {
  return reinterpret_cast<R*>(c.ws + off) + (size_t)k * c.L->N;
}
template <typename R>
R* st3(const Ctx3& c, int which, int f) {
  return fld3<R>(c, which == 0 ? c.L->stA : c.L->stB, f);
}
template <typename R>
R* ad3(const Ctx3& c, int which, int f) {
  return fld3<R>(c, which == 0 ? c.L->adA : c.L->adB, f);
}
int ew_grid(size_t n) { return lks_host::elementwise_blocks(n); }
// z planes per CTA of the warp-column forward.  A CTA pushes its chunk and one halo
// plane on each side; the CTAs run in rounds of `resident` (every SM's resident
// CTAs), so the march takes about rounds x (zc + 2) plane steps.  The smallest such
// cost over zc in 8 .. 64 avoids a nearly empty last round.
int col_chunk3(const lks_problem_desc& d, int resident, int tile_rows) {
  const long long txy = (long long)((d.nx + CX3 - 1) / CX3) * ((d.ny + tile_rows - 1) / tile_rows);
  int best = ZC3;
  long long best_cost = -1;
  for (int zc = 8; zc <= 64; ++zc) {
    const long long ctas = txy * ((d.nz + zc - 1) / zc);
    const long long cost = (ctas + resident - 1) / resident * (zc + 2);
    if (best_cost < 0 || cost < best_cost) best_cost = cost, best = zc;
  }
  return best;
}

dim3 march_grid(const lks_problem_desc& d) {
  return dim3((d.nx + TX3 - 1) / TX3, (d.ny + TY3 - 1) / TY3, (d.nz + ZC3 - 1) / ZC3);
}

// TMA-staged kernels: FP32 and rows whose byte pitch is a multiple of 16.
bool tma3_ok(const lks_problem_desc& d) {
  return d.real_type == LKS_REAL_F32 && d.nx % 4 == 0 && lks_host::encode_fn() != nullptr;
}
// Tensor map of one nx x ny x nz float field for boxes bw x bh x 1.
lks_status map3(const Ctx3& c, const void* ptr, int bw, int bh, CUtensorMap* m) {
  const auto& d = *c.d;
  const cuuint64_t dims[3] = {(cuuint64_t)d.nx, (cuuint64_t)d.ny, (cuuint64_t)d.nz};
  const cuuint64_t strides[2] = {(cuuint64_t)d.nx * 4, (cuuint64_t)d.nx * d.ny * 4};
  const cuuint32_t box[3] = {(cuuint32_t)bw, (cuuint32_t)bh, 1};
  const cuuint32_t es[3] = {1, 1, 1};
  const CUresult r = lks_host::encode_fn()(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void*>(ptr), dims, strides,
                                           box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                           CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? LKS_OK : fail3(c, LKS_ERR_CUDA, "cuTensorMapEncodeTiled (3-D) failed");
}

template <typename R>
lks_status forward3_t(const Ctx3& c, const void* gamma_dev, double* J_dev, int* cur_out, int* path_out) {
  const auto& d = *c.d;
  const auto& L = *c.L;
  const size_t fb = L.N * sizeof(R);
  if (gamma_dev != c.ws + L.gamma)
    CK3(c, cudaMemcpyAsync(c.ws + L.gamma, gamma_dev, fb, cudaMemcpyDeviceToDevice, c.stream));
  CK3(c, cudaMemsetAsync(c.ws + L.stA, 0, fb * 4, c.stream));
  CK3(c, cudaMemsetAsync(c.ws + L.status, 0, sizeof(int), c.stream));
  const Geom3 g = geom3(d);
  const Coef3<R> cf = coef3<R>(d);
  const R* gam = fld3<R>(c, L.gamma);
  // 1/(1+alpha) (the objective source is not needed for the forward march)
  src3_kernel<R><<<ew_grid(L.N), 256, 0, c.stream>>>(gam, st3<R>(c, 0, 1), st3<R>(c, 0, 2), st3<R>(c, 0, 3), g, cf,
                                                     fld3<R>(c, L.binv), fld3<R>(c, L.src, 0), fld3<R>(c, L.src, 1),
                                                     fld3<R>(c, L.src, 2));
  CK3(c, cudaGetLastError());
  ++*c.launches;
  int cur = 0;
  *path_out = LKS_PATH_STEP;
  if constexpr (sizeof(R) == 4) {
    if (tma3_ok(d)) {
      // the warp-column forward unless the per-tile kernels are asked for
      const bool col = d.exec_path != LKS_PATH_STEP;
      const int bw = col ? CBW3 : BW3, bh = col ? PBH3 : BH3;
      Maps3F maps[2];
      Fwd3TArgs ta[2];
      lks_status st;
      for (int b = 0; b < 2; ++b) {
        for (int f = 0; f < 4; ++f)
          if ((st = map3(c, st3<float>(c, b, f), bw, bh, &maps[b].m[f])) != LKS_OK) return st;
        if ((st = map3(c, fld3<float>(c, L.binv), bw, bh, &maps[b].m[4])) != LKS_OK) return st;
        for (int f = 0; f < 4; ++f) ta[b].out[f] = st3<float>(c, 1 - b, f);
        ta[b].binv = fld3<float>(c, L.binv);
        ta[b].status = reinterpret_cast<int*>(c.ws + L.status);
      }
      if (col) {
        CK3(c, cudaFuncSetAttribute(fwd3p_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fwd3p_smem()));
        int dev = 0, sms = 0, per_sm = 0;
        CK3(c, cudaGetDevice(&dev));
        CK3(c, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        CK3(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fwd3p_kernel, NTP3, fwd3p_smem()));
        const int zc = col_chunk3(d, std::max(1, sms * per_sm), NYP3);
        ta[0].zc = ta[1].zc = zc;
        const dim3 grid((d.nx + CX3 - 1) / CX3, (d.ny + NYP3 - 1) / NYP3, (d.nz + zc - 1) / zc);
        for (int s = 0; s < d.n_steps; ++s) {
          fwd3p_kernel<<<grid, NTP3, fwd3p_smem(), c.stream>>>(maps[cur], ta[cur], g, cf);
          CK3(c, cudaGetLastError());
          ++*c.launches;
          cur = 1 - cur;
        }
        *path_out = LKS_PATH_COLUMN;
      } else {
        CK3(c, cudaFuncSetAttribute(fwd3t_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fwd3t_smem()));
        for (int s = 0; s < d.n_steps; ++s) {
          fwd3t_kernel<<<march_grid(d), NTF3, fwd3t_smem(), c.stream>>>(maps[cur], ta[cur], g, cf);
          CK3(c, cudaGetLastError());
          ++*c.launches;
          cur = 1 - cur;
        }
      }
    }
  }
  const size_t smem = fwd3_smem<R>();
  CK3(c, cudaFuncSetAttribute(fwd3_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  for (int s = 0; s < d.n_steps && !(sizeof(R) == 4 && tma3_ok(d)); ++s) {
    Fwd3Args<R> a;
    for (int f = 0; f < 4; ++f) {
      a.in[f] = st3<R>(c, cur, f);
      a.out[f] = st3<R>(c, 1 - cur, f);
    }
    a.binv = fld3<R>(c, L.binv);
    a.status = reinterpret_cast<int*>(c.ws + L.status);
    fwd3_kernel<R><<<march_grid(d), NT3, smem, c.stream>>>(a, g, cf);
    CK3(c, cudaGetLastError());
    ++*c.launches;
    cur = 1 - cur;
  }
  double* part = reinterpret_cast<double*>(c.ws + L.jpart);
  double* jval = reinterpret_cast<double*>(c.ws + L.jval);
  objective3_kernel<R><<<L.jblocks, NTHREADS, 0, c.stream>>>(gam, st3<R>(c, cur, 0), st3<R>(c, cur, 1),
                                                             st3<R>(c, cur, 2), st3<R>(c, cur, 3), g, cf, part);
  reduce_partials_kernel<<<1, NTHREADS, 0, c.stream>>>(part, L.jblocks, nullptr, 0, jval);
  CK3(c, cudaGetLastError());
  *c.launches += 2;
  if (J_dev) CK3(c, cudaMemcpyAsync(J_dev, jval, sizeof(double), cudaMemcpyDeviceToDevice, c.stream));
  *cur_out = cur;
  return LKS_OK;
}

template <typename R>
lks_status adjoint3_t(const Ctx3& c, int cur, int* acur_out, int* path_out) {
  const auto& d = *c.d;
  const auto& L = *c.L;
  const size_t fb = L.N * sizeof(R);
  const Geom3 g = geom3(d);
  const Coef3<R> cf = coef3<R>(d);
  const R* gam = fld3<R>(c, L.gamma);
  src3_kernel<R><<<ew_grid(L.N), 256, 0, c.stream>>>(gam, st3<R>(c, cur, 1), st3<R>(c, cur, 2), st3<R>(c, cur, 3), g,
                                                     cf, fld3<R>(c, L.binv), fld3<R>(c, L.src, 0),
                                                     fld3<R>(c, L.src, 1), fld3<R>(c, L.src, 2));
  CK3(c, cudaGetLastError());
  ++*c.launches;
  CK3(c, cudaMemsetAsync(c.ws + L.adA, 0, fb * kNA3, c.stream));
  int acur = 0;
  *path_out = LKS_PATH_STEP;
  if constexpr (sizeof(R) == 4) {
    if (tma3_ok(d) && d.exec_path != LKS_PATH_STEP) {  // the warp-column adjoint
      Maps3F maps[2];
      Adj3CArgs ca[2];
      lks_status st;
      const int yi[NAY3] = {5, 7, 8}, oi[7] = {0, 1, 2, 3, 4, 6, 9};
      for (int b = 0; b < 2; ++b) {
        for (int f = 0; f < NAY3; ++f)
          if ((st = map3(c, ad3<float>(c, b, yi[f]), CBW3, CBH3, &maps[b].m[f])) != LKS_OK) return st;
        for (int f = 0; f < 7; ++f) ca[b].own[f] = ad3<float>(c, b, oi[f]);
        for (int f = 0; f < 3; ++f) ca[b].own[7 + f] = st3<float>(c, cur, 1 + f);
        ca[b].cf[0] = fld3<float>(c, L.binv);
        for (int f = 0; f < 3; ++f) ca[b].cf[1 + f] = fld3<float>(c, L.src, f);
        for (int q = 0; q < kNA3; ++q) ca[b].m0[q] = ad3<float>(c, 1 - b, q);
        ca[b].emap = reinterpret_cast<const float*>(c.ws + L.emap);
        ca[b].status = reinterpret_cast<int*>(c.ws + L.status);
      }
      CK3(c, cudaFuncSetAttribute(adj3c_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)adj3c_smem()));
      int dev = 0, sms = 0, per_sm = 0;
      CK3(c, cudaGetDevice(&dev));
      CK3(c, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
      CK3(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, adj3c_kernel, NTC3, adj3c_smem()));
      const int zc = col_chunk3(d, std::max(1, sms * per_sm), NYC3);
      ca[0].zc = ca[1].zc = zc;
      const dim3 grid((d.nx + CX3 - 1) / CX3, (d.ny + NYC3 - 1) / NYC3, (d.nz + zc - 1) / zc);
      for (int it = 0; it < d.n_adj; ++it) {
        adj3c_kernel<<<grid, NTC3, adj3c_smem(), c.stream>>>(maps[acur], ca[acur], g, cf);
        CK3(c, cudaGetLastError());
        ++*c.launches;
        acur = 1 - acur;
      }
      *acur_out = acur;
      *path_out = LKS_PATH_COLUMN;
      return LKS_OK;
    }
    if (tma3_ok(d)) {
      Maps3A maps[2];
      Adj3TArgs ta[2];
      lks_status st;
      const int zi[3] = {6, 8, 9}, pi[7] = {4, 5, 7, 0, 1, 2, 3};
      for (int b = 0; b < 2; ++b) {
        for (int f = 0; f < 3; ++f)
          if ((st = map3(c, ad3<float>(c, b, zi[f]), BW3, BH3, &maps[b].zr[f])) != LKS_OK) return st;
        for (int f = 0; f < 7; ++f)
          if ((st = map3(c, ad3<float>(c, b, pi[f]), BW3, BH3, &maps[b].pl[f])) != LKS_OK) return st;
        for (int f = 0; f < 3; ++f)
          if ((st = map3(c, st3<float>(c, cur, 1 + f), BW3, BH3, &maps[b].pl[7 + f])) != LKS_OK) return st;
        if ((st = map3(c, fld3<float>(c, L.binv), TX3, TY3, &maps[b].out[0])) != LKS_OK) return st;
        for (int f = 0; f < 3; ++f)
          if ((st = map3(c, fld3<float>(c, L.src, f), TX3, TY3, &maps[b].out[1 + f])) != LKS_OK) return st;
        for (int q = 0; q < kNA3; ++q) ta[b].m0[q] = ad3<float>(c, 1 - b, q);
        ta[b].emap = reinterpret_cast<const float*>(c.ws + L.emap);
        ta[b].status = reinterpret_cast<int*>(c.ws + L.status);
      }
      CK3(c, cudaFuncSetAttribute(adj3t_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)adj3t_smem()));
      for (int it = 0; it < d.n_adj; ++it) {
        adj3t_kernel<<<march_grid(d), NTF3, adj3t_smem(), c.stream>>>(maps[acur], ta[acur], g, cf);
        CK3(c, cudaGetLastError());
        ++*c.launches;
        acur = 1 - acur;
      }
      *acur_out = acur;
      return LKS_OK;
    }
  }
  const size_t smem = adj3_smem<R>();
  CK3(c, cudaFuncSetAttribute(adj3_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  for (int it = 0; it < d.n_adj; ++it) {
    Adj3Args<R> a;
    for (int q = 0; q < kNA3; ++q) {
      a.m1[q] = ad3<R>(c, acur, q);
      a.m0[q] = ad3<R>(c, 1 - acur, q);
    }
    for (int q = 0; q < 3; ++q) {
      a.u[q] = st3<R>(c, cur, 1 + q);
      a.src[q] = fld3<R>(c, L.src, q);
    }
    a.binv = fld3<R>(c, L.binv);
    a.emap = reinterpret_cast<const R*>(c.ws + L.emap);
    a.status = reinterpret_cast<int*>(c.ws + L.status);
    const int zi[3] = {6, 8, 9}, pi[3] = {4, 5, 7};
    for (int q = 0; q < 3; ++q) {
      a.zs[q] = a.m1[zi[q]];
      a.ps[q] = a.m1[pi[q]];
    }
    for (int q = 0; q < 4; ++q) a.ns[q] = a.m1[q];
    for (int q = 0; q < 3; ++q) a.ns[4 + q] = a.u[q];
    adj3_kernel<R><<<march_grid(d), NT3, smem, c.stream>>>(a, g, cf);
    CK3(c, cudaGetLastError());
    ++*c.launches;
    acur = 1 - acur;
  }
  *acur_out = acur;
  return LKS_OK;
}

template <typename R>
lks_status sensitivity3_t(const Ctx3& c, int cur, int acur, void* out) {
  const auto& L = *c.L;
  sens3_kernel<R><<<ew_grid(L.N), 256, 0, c.stream>>>(
      fld3<R>(c, L.gamma), st3<R>(c, cur, 1), st3<R>(c, cur, 2), st3<R>(c, cur, 3), ad3<R>(c, acur, 1),
      ad3<R>(c, acur, 2), ad3<R>(c, acur, 3), geom3(*c.d), coef3<R>(*c.d), reinterpret_cast<R*>(out));
  CK3(c, cudaGetLastError());
  ++*c.launches;
  return LKS_OK;
}

// Least squares by the normal equations with partial pivoting: m <= 19 rows,
// columns that are identically zero are dropped (their unknowns are zero).
void lsq19(const double* A, int nc, const double* rhs, double* x) {
  int live[24], nl = 0;
  for (int q = 0; q < nc; ++q) {
    double s = 0.0;
    for (int r = 0; r < 19; ++r) s += std::fabs(A[r * nc + q]);
    x[q] = 0.0;
    if (s > 0) live[nl++] = q;
  }
  double G[24][25];
  for (int p = 0; p < nl; ++p) {
    for (int q = 0; q < nl; ++q) {
      double s = 0.0;
      for (int r = 0; r < 19; ++r) s += A[r * nc + live[p]] * A[r * nc + live[q]];
      G[p][q] = s;
    }
    double s = 0.0;
    for (int r = 0; r < 19; ++r) s += A[r * nc + live[p]] * rhs[r];
    G[p][nl] = s;
  }
  for (int col = 0; col < nl; ++col) {
    int pv = col;
    for (int r = col + 1; r < nl; ++r)
      if (std::fabs(G[r][col]) > std::fabs(G[pv][col])) pv = r;
    for (int q = 0; q <= nl; ++q) std::swap(G[col][q], G[pv][q]);
    for (int r = 0; r < nl; ++r) {
      if (r == col) continue;
      const double f = G[r][col] / G[col][col];
      for (int q = col; q <= nl; ++q) G[r][q] -= f * G[col][q];
    }
  }
  for (int p = 0; p < nl; ++p) x[live[p]] = G[p][nl] / G[p][p];
}

}  // namespace

void flow_moment_map3(double A, int cls, double* out, double* unit, double* fill) {
  const int n[3] = {cls / 9 - 1, (cls / 3) % 3 - 1, cls % 3 - 1};
  std::memset(out, 0, sizeof(double) * kNA3 * 19);
  if (unit) std::memset(unit, 0, sizeof(double) * kNA3);
  if (fill) std::memset(fill, 0, sizeof(double) * kFillLen3);
  if (n[0] == 0 && n[1] == 0 && n[2] == 0) return;
  const int faces = std::abs(n[0]) + std::abs(n[1]) + std::abs(n[2]);
  const bool pressure = faces == 1 && n[0] == 1;
  bool unk[19];
  int U[19], nu = 0;
  for (int k = 0; k < 19; ++k) {
    unk[k] = false;
    for (int a = 0; a < 3; ++a) unk[k] = unk[k] || c3(k, a) * n[a] > 0;
    if (unk[k]) U[nu++] = k;
  }
  auto cdot = [](int k, const int* v) { return c3(k, 0) * v[0] + c3(k, 1) * v[1] + c3(k, 2) * v[2]; };
  double M[19][19];
  for (int r = 0; r < 19; ++r)
    for (int q = 0; q < 19; ++q) {
      const int cq[3] = {c3(q, 0), c3(q, 1), c3(q, 2)};
      M[r][q] = (r == q ? (double)cdot(r, n) : 0.0) - 2.0 * A * w3d(q) * cdot(q, n) * cdot(r, cq);
    }
  const int nc = nu + 3;
  std::vector<double> Am(19 * nc);
  const int ax = n[0] != 0 ? 0 : (n[1] != 0 ? 1 : 2);
  for (int r = 0; r < 19; ++r) {
    for (int q = 0; q < nu; ++q) Am[r * nc + q] = M[r][U[q]];
    if (pressure) {
      Am[r * nc + nu] = 1.0;
      Am[r * nc + nu + 1] = c3(r, (ax + 1) % 3);
      Am[r * nc + nu + 2] = c3(r, (ax + 2) % 3);
    } else {
      for (int a = 0; a < 3; ++a) Am[r * nc + nu + a] = c3(r, a);
    }
  }
  double X[19][19] = {};  // X[u][k]: unknown u per unit of the known f~_k
  for (int k = 0; k < 19; ++k) {
    if (unk[k]) continue;
    double rhs[19], x[24];
    for (int r = 0; r < 19; ++r) rhs[r] = -M[r][k];
    lsq19(Am.data(), nc, rhs, x);
    for (int q = 0; q < nu; ++q) X[U[q]][k] = x[q];
  }
  auto mom = [](int r, int k) {
    const double cx = c3(k, 0), cy = c3(k, 1), cz = c3(k, 2);
    const double phi[kNA3] = {1, cx, cy, cz, cx * cx, cx * cy, cx * cz, cy * cy, cy * cz, cz * cz};
    return w3d(k) * phi[r];
  };
  for (int r = 0; r < kNA3; ++r)
    for (int k = 0; k < 19; ++k) {
      if (unk[k]) continue;
      double s = mom(r, k);
      for (int q = 0; q < nu; ++q) s += mom(r, U[q]) * X[U[q]][k];
      out[r * 19 + k] = s;
    }
  double xu[24];  // the unknowns' response to a unit term in every row
  {
    double rhs[19];
    for (int r = 0; r < 19; ++r) rhs[r] = -1.0;
    lsq19(Am.data(), nc, rhs, xu);
  }
  if (unit)  // its moments
    for (int r = 0; r < kNA3; ++r) {
      double s = 0.0;
      for (int q = 0; q < nu; ++q) s += mom(r, U[q]) * xu[q];
      unit[r] = s;
    }
  if (fill && faces == 1) {
    int O[19], no = 0;
    for (int k = 0; k < 19; ++k)
      if (cdot(k, n) < 0) O[no++] = k;
    for (int q = 0; q < nu && q < 5; ++q) {
      for (int p = 0; p < no && p < 5; ++p) fill[q * 5 + p] = X[U[q]][O[p]];
      fill[25 + q] = xu[q];
    }
  }
}

Layout3 make_layout3(const lks_problem_desc& d) {
  Layout3 L;
  L.N = (size_t)d.nx * d.ny * d.nz;
  L.rsize = d.real_type == LKS_REAL_F64 ? 8 : 4;
  L.jblocks = (int)std::min<size_t>((L.N + NTHREADS - 1) / NTHREADS, 1024);
  size_t off = 0;
  auto take = [&](size_t b) {
    const size_t o = off;
    off = up256(off + b);
    return o;
  };
  const size_t fb = L.N * L.rsize;
  L.gamma = take(fb);
  L.stA = take(fb * 4);
  L.stB = take(fb * 4);
  L.adA = take(fb * kNA3);
  L.adB = take(fb * kNA3);
  L.binv = take(fb);
  L.src = take(fb * 3);
  L.jpart = take(sizeof(double) * L.jblocks);
  L.jval = take(sizeof(double));
  L.status = take(sizeof(int));
  // maps, then the boundary objective terms, then the single-face fills
  L.emap = take(L.rsize * (kClasses3 * kNA3 * 20 + 6 * kFillLen3));
  L.total = off;
  return L;
}

lks_status upload_maps3(const Ctx3& c) {
  const double A = (1.0 / 6.0 - c.d->nu) * 4.5;
  // kClasses3 maps of 10 x 19, then per class the moments' response to the boundary
  // objective term of every row: +kappa_p on the inlet face (class of n = (-1, 0, 0)),
  // -kappa_p on the outlet face (n = (1, 0, 0)), absorbed there by lambda~
  std::vector<double> m((size_t)kClasses3 * kNA3 * 20 + 6 * kFillLen3, 0.0);
  double* off = &m[(size_t)kClasses3 * kNA3 * 19];
  double* fills = &m[(size_t)kClasses3 * kNA3 * 20];
  for (int cls = 0; cls < kClasses3; ++cls) {
    double unit[kNA3], fill[kFillLen3];
    flow_moment_map3(A, cls, &m[(size_t)cls * kNA3 * 19], unit, fill);
    const double jb = cls == 4 ? c.d->kappa_p : (cls == 22 ? -c.d->kappa_p : 0.0);
    for (int r = 0; r < kNA3; ++r) off[cls * kNA3 + r] = jb * unit[r];
    const int n[3] = {cls / 9 - 1, (cls / 3) % 3 - 1, cls % 3 - 1};
    if (std::abs(n[0]) + std::abs(n[1]) + std::abs(n[2]) == 1) {
      const int a = n[0] != 0 ? 0 : (n[1] != 0 ? 1 : 2);
      double* f = fills + (2 * a + (n[a] > 0)) * kFillLen3;
      for (int q = 0; q < 25; ++q) f[q] = fill[q];
      for (int q = 0; q < 5; ++q) f[25 + q] = jb * fill[25 + q];
    }
  }
  if (c.L->rsize == 8) {
    CK3(c, cudaMemcpy(c.ws + c.L->emap, m.data(), m.size() * 8, cudaMemcpyHostToDevice));
  } else {
    std::vector<float> f(m.begin(), m.end());
    CK3(c, cudaMemcpy(c.ws + c.L->emap, f.data(), f.size() * 4, cudaMemcpyHostToDevice));
  }
  return LKS_OK;
}

lks_status forward3(const Ctx3& c, const void* gamma_dev, double* J_dev, int* cur, int* path) {
  return c.L->rsize == 8 ? forward3_t<double>(c, gamma_dev, J_dev, cur, path)
                         : forward3_t<float>(c, gamma_dev, J_dev, cur, path);
}
lks_status adjoint3(const Ctx3& c, int cur, int* acur, int* path) {
  return c.L->rsize == 8 ? adjoint3_t<double>(c, cur, acur, path) : adjoint3_t<float>(c, cur, acur, path);
}
lks_status sensitivity3(const Ctx3& c, int cur, int acur, void* out) {
  return c.L->rsize == 8 ? sensitivity3_t<double>(c, cur, acur, out) : sensitivity3_t<float>(c, cur, acur, out);
}

}  // namespace lks3
