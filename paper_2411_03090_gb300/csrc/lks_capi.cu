// lks_capi.cu -- host side of the C ABI declared in include/lks.h: descriptor
// checks, workspace layout, the generalized-inverse edge maps of the adjoint, and
// the stream-ordered orchestration of the LKS / ALKS marches (arXiv 2411.03090,
// Sec. 2.7 Steps 2-5).  Every step of the path runs in the kernels of
// lks_kernels.cuh; this file only sizes, orders and launches them.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <type_traits>
#include <unordered_map>
#include <vector>

#include "../../include/lks.h"
#include "lks_kernels.cuh"
#include "lks_resident.cuh"
#include "lks_resident_tb.cuh"
#include "lks_3d.cuh"
#include "lks_col.cuh"
#include "lks_host.cuh"
#include "lks_tma.cuh"

using namespace lks;
using namespace lks_host;

namespace {

constexpr size_t kAlign = 256;
inline size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

// ------------------------------------------------------------------------------------
// Workspace layout
// ------------------------------------------------------------------------------------
struct Layout {
  size_t gamma = 0, stA = 0, stB = 0, adA = 0, adB = 0, sens = 0, sens64 = 0;
  size_t jfwd = 0, jobj = 0, jval = 0, status = 0, emap = 0, flags = 0, mat = 0, chg = 0;
  size_t traj = 0, snaps = 0, scales = 0, seg = 0, seg2 = 0, lvl_stage = 0, total = 0;
  int lvl16 = 0;  // trajectory / segment levels stored in 16 bits (segment_type BF16 / F16)
  int nF = 3, nA = 6, nT = 2;  // state fields, adjoint fields, trajectory fields
  int fwd_blocks = 0, obj_blocks = 0;
  int n_ckpt = 0, seg_levels = 0;
  size_t N = 0, rsize = 4, snap_elem = 4;
};

// Tile shapes of the TMA-staged per-step kernels.
constexpr int kFwdTX = 32, kFwdTY = 16, kAdjTX = 32, kAdjTY = 16;

int obj_grid(size_t N) { return (int)std::min<size_t>((N + NTHREADS - 1) / NTHREADS, 1024); }

// overlap: a second segment store, so that the recompute of a segment can run while
// the adjoint marches the one after it (checkpointed unsteady problems).
Layout make_layout(const lks_problem_desc* d, bool overlap = true) {
  Layout L;
  L.N = (size_t)d->nx * d->ny;
  L.rsize = d->real_type == LKS_REAL_F64 ? 8 : 4;
  L.nF = d->thermal ? 4 : 3;
  L.nA = d->thermal ? 9 : 6;
  L.nT = d->thermal ? 3 : 2;
  const int gx = (d->nx + TX - 1) / TX, gy = (d->ny + TY - 1) / TY;
  const int col_tiles = ((d->nx + C2_W - 1) / C2_W) * ((d->ny + Col2Geo<C2_R>::H - 1) / Col2Geo<C2_R>::H);
  const int tma_tiles = ((d->nx + kFwdTX - 1) / kFwdTX) * ((d->ny + kFwdTY - 1) / kFwdTY);
  // J partials: one per CTA of the largest forward grid (the persistent TMA grid is
  // at most one CTA per tile)
  L.fwd_blocks = std::max(std::max(gx * gy, col_tiles), tma_tiles);
  L.obj_blocks = obj_grid(L.N);
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off = align_up(off + bytes);
    return o;
  };
  const size_t fb = L.N * L.rsize;
  L.gamma = take(fb);
  L.stA = take(fb * L.nF);
  L.stB = take(fb * L.nF);
  L.adA = take(fb * L.nA);
  L.adB = take(fb * L.nA);
  L.jfwd = take(sizeof(double) * (L.fwd_blocks + 1));  // per-block partials, then the boundary objectives
  L.jobj = take(sizeof(double) * L.obj_blocks);
  L.jval = take(sizeof(double));
  L.status = take(sizeof(int));
  L.chg = take(2 * sizeof(unsigned));  // change of a measured step (tol > 0)
  L.emap = take(L.rsize * lks::kEdgeMapLen);  // 9 classes x 6 x 10, then 9 x 6 boundary objective terms
  L.flags = take(sizeof(int) * (size_t)((d->nx + 31) / 32) * (size_t)((d->ny + 7) / 8));
  L.mat = take(fb * 3);  // 1/(1+alpha), alpha, B (FP32 staged kernels)
  if (!d->steady) {
    L.sens = take(fb);
    L.sens64 = take(sizeof(double) * L.N);
    // 16-bit levels (FP32 lattices): the level store holds 2-byte values, and three
    // FP32 levels stage what a forward step writes and what an adjoint step reads
    L.lvl16 = d->segment_type != LKS_SNAP_F32 && d->real_type == LKS_REAL_F32;
    const size_t lb = L.lvl16 ? L.N * 2 : fb;  // bytes of one field of one stored level
    if (L.lvl16) L.lvl_stage = take(fb * L.nT * 3);
    if (d->checkpoint_every == 0) {
      L.traj = take(lb * L.nT * ((size_t)d->n_steps + 1));
    } else {
      const int K = d->checkpoint_every;
      L.n_ckpt = (d->n_steps + K - 1) / K;
      L.snap_elem = d->snapshot_type == LKS_SNAP_F32 ? 4 : 2;
      L.snaps = take(L.snap_elem * L.N * L.nF * (size_t)L.n_ckpt);
      L.scales = take(sizeof(float) * 2 * L.nF * (size_t)L.n_ckpt);
      L.seg_levels = K + 2;
      L.seg = take(lb * L.nT * (size_t)L.seg_levels);
      if (overlap) L.seg2 = take(lb * L.nT * (size_t)L.seg_levels);
    }
  }
  L.total = off;
  return L;
}

}  // namespace

// ------------------------------------------------------------------------------------
// Handle
// ------------------------------------------------------------------------------------
struct lks_handle {
  lks_problem_desc d;
  Layout L;
  unsigned char* ws = nullptr;
  size_t ws_bytes = 0;
  cudaStream_t stream = nullptr;
  int device = 0;
  int cur = 0;      // which state buffer holds the current state (0 = A)
  int acur = 0;     // which adjoint buffer holds the current adjoint
  int t = 0;        // time level of the current state
  int phase = 0;
  int fwd_path = 0, adj_path = 0;
  int64_t fwd_steps = 0, adj_steps = 0, launches = 0;
  std::vector<double> emap_h;
  std::vector<float> emap_f;
  std::unordered_map<uint64_t, CUtensorMap> tmaps;  // (pointer, box) -> tensor map
  int tma_grid_fwd = 0, tma_grid_adj[2][2] = {{0, 0}, {0, 0}};  // adj: [thermal][same state]
  int sms = 0;        // multiprocessors of the device (queried once)
  int res_steps_fwd = 0, res_steps_adj = 0;  // steps per exchange of the last resident marches
  double fwd_change = 0.0, adj_change = 0.0;  // relative change of the last measured steps
  bool have_adj = false;  // adjoint fields hold an earlier march (or alks_set_adjoint)
  bool is3 = false;  // D3Q19 problem: the lks3 path with layout L3
  lks3::Layout3 L3;
  std::string err;
  // Checkpointed unsteady problems: a second stream, on which the recompute of a
  // segment runs while the adjoint marches the next one, and the events that order
  // the two segment stores between them.
  cudaStream_t aux = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_seg[2] = {nullptr, nullptr}, ev_adj[2] = {nullptr, nullptr};
  ~lks_handle() {
    for (cudaEvent_t e : {ev_fork, ev_seg[0], ev_seg[1], ev_adj[0], ev_adj[1]})
      if (e) cudaEventDestroy(e);
    if (aux) cudaStreamDestroy(aux);
  }
};

namespace {

lks_status fail(lks_handle* h, lks_status s, const std::string& m) {
  if (h) h->err = m;
  return s;
}

#define CKH(h, call)                                                                    \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess)                                                              \
      return fail(h, LKS_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

template <typename R>
R* fld(lks_handle* h, size_t off, int k) {
  return reinterpret_cast<R*>(h->ws + off) + (size_t)k * h->L.N;
}

template <typename R>
R* state_ptr(lks_handle* h, int which, int f) {
  return fld<R>(h, which == 0 ? h->L.stA : h->L.stB, f);
}
template <typename R>
R* adj_ptr(lks_handle* h, int which, int f) {
  return fld<R>(h, which == 0 ? h->L.adA : h->L.adB, f);
}

template <typename R>
lks_status set_smem_attrs() {
  const int fs = (int)(fwd_smem_elems<false>() * sizeof(R)), fst = (int)(fwd_smem_elems<true>() * sizeof(R));
  const int as = (int)(adj_smem_elems<false>() * sizeof(R)), ast = (int)(adj_smem_elems<true>() * sizeof(R));
  cudaError_t e = cudaSuccess;
  e = cudaFuncSetAttribute(fwd_step_kernel<R, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, fs);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(fwd_step_kernel<R, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, fst);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(adj_step_kernel<R, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, as);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(adj_step_kernel<R, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, ast);
  return e == cudaSuccess ? LKS_OK : LKS_ERR_CUDA;
}

// One forward step: state `cur` -> other buffer, new level t_new.
template <bool TH>
lks_status launch_fwd_tma(lks_handle* h, int t_new, double* Jpartial, float* tu, float* tv, float* tT);
bool tma_ok(lks_handle* h);
template <bool TH, bool SAME>
lks_status launch_adj_tma(lks_handle* h, const float* u1, const float* v1, const float* u0, const float* v0,
                          const float* T0, float* sens, int sens_flow, int sens_thermal);

template <typename R>
lks_status launch_fwd(lks_handle* h, int t_new, double* Jpartial, R* tu, R* tv, R* tT) {
  const auto& d = h->d;
  if constexpr (sizeof(R) == 4) {
    if (tma_ok(h))
      return d.thermal ? launch_fwd_tma<true>(h, t_new, Jpartial, tu, tv, tT)
                       : launch_fwd_tma<false>(h, t_new, Jpartial, tu, tv, tT);
  }
  FwdArgs<R> a;
  const int src = h->cur, dst = 1 - h->cur;
  a.drho = state_ptr<R>(h, src, 0);
  a.u = state_ptr<R>(h, src, 1);
  a.v = state_ptr<R>(h, src, 2);
  a.T = d.thermal ? state_ptr<R>(h, src, 3) : nullptr;
  a.drho_n = state_ptr<R>(h, dst, 0);
  a.u_n = state_ptr<R>(h, dst, 1);
  a.v_n = state_ptr<R>(h, dst, 2);
  a.T_n = d.thermal ? state_ptr<R>(h, dst, 3) : nullptr;
  a.gamma = fld<R>(h, h->L.gamma, 0);
  a.u_in = (R)inlet_amp(d, t_new);
  a.J_partial = Jpartial;
  a.status = reinterpret_cast<int*>(h->ws + h->L.status);
  a.traj_u = tu;
  a.traj_v = tv;
  a.traj_T = tT;
  const dim3 grid((d.nx + TX - 1) / TX, (d.ny + TY - 1) / TY);
  const Geom g = make_geom(d);
  const Coef<R> c = make_coef<R>(d);
  if (d.thermal)
    fwd_step_kernel<R, true><<<grid, NTHREADS, fwd_smem_elems<true>() * sizeof(R), h->stream>>>(a, g, c);
  else
    fwd_step_kernel<R, false><<<grid, NTHREADS, fwd_smem_elems<false>() * sizeof(R), h->stream>>>(a, g, c);
  CKH(h, cudaGetLastError());
  h->cur = dst;
  h->t = t_new;
  h->fwd_steps++;
  h->launches++;
  h->fwd_path = LKS_PATH_STEP;
  return LKS_OK;
}

// One adjoint step: adjoint `acur` (level t+1) -> other buffer (level t).
template <typename R>
lks_status launch_adj(lks_handle* h, const R* u1, const R* v1, const R* u0, const R* v0, const R* T0,
                      R* sens, int sens_flow, int sens_thermal) {
  const auto& d = h->d;
  if constexpr (sizeof(R) == 4) {
    if (tma_ok(h)) {
      const bool same = (u0 == u1 && v0 == v1);
      if (d.thermal)
        return same ? launch_adj_tma<true, true>(h, u1, v1, u0, v0, T0, sens, sens_flow, sens_thermal)
                    : launch_adj_tma<true, false>(h, u1, v1, u0, v0, T0, sens, sens_flow, sens_thermal);
      return same ? launch_adj_tma<false, true>(h, u1, v1, u0, v0, T0, sens, sens_flow, sens_thermal)
                  : launch_adj_tma<false, false>(h, u1, v1, u0, v0, T0, sens, sens_flow, sens_thermal);
    }
  }
  AdjArgs<R> a;
  const int src = h->acur, dst = 1 - h->acur;
  for (int f = 0; f < 9; ++f) {
    const int ff = (f < h->L.nA) ? f : 0;
    a.m1[f] = adj_ptr<R>(h, src, ff);
    a.m0[f] = adj_ptr<R>(h, dst, ff);
  }
  a.u1 = u1;
  a.v1 = v1;
  a.u0 = u0;
  a.v0 = v0;
  a.T0 = T0;
  a.gamma = fld<R>(h, h->L.gamma, 0);
  a.emap = reinterpret_cast<const R*>(h->ws + h->L.emap);
  a.sens = sens;
  a.sens_flow = sens_flow;
  a.sens_thermal = sens_thermal;
  a.status = reinterpret_cast<int*>(h->ws + h->L.status);
  const dim3 grid((d.nx + TX - 1) / TX, (d.ny + TY - 1) / TY);
  const Geom g = make_geom(d);
  const Coef<R> c = make_coef<R>(d);
  if (d.thermal)
    adj_step_kernel<R, true><<<grid, NTHREADS, adj_smem_elems<true>() * sizeof(R), h->stream>>>(a, g, c);
  else
    adj_step_kernel<R, false><<<grid, NTHREADS, adj_smem_elems<false>() * sizeof(R), h->stream>>>(a, g, c);
  CKH(h, cudaGetLastError());
  h->acur = dst;
  h->adj_steps++;
  h->launches++;
  h->adj_path = LKS_PATH_STEP;
  return LKS_OK;
}

// ------------------------------------------------------------------------------------
// Resident (persistent, cooperative) marches
// ------------------------------------------------------------------------------------
struct ResPlan {
  int cfg = -1, ntiles = 0;
};

// Tile shapes of the resident marches: {TXR, TYR, threads}.
// (64 x 14 puts the 512 x 256 channel on 8 x 19 = 152 tiles, one per SM of a GB300.)
constexpr int kNResCfg = 4;
// {tile x, tile y, threads}; the 64 x 14 forward with one step per exchange runs 768.
constexpr int kResCfg[kNResCfg][3] = {{64, 16, 512}, {32, 16, 256}, {32, 8, 256}, {64, 14, 512}};

int device_sms(lks_handle* h) {
  if (h->sms == 0 && cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, h->device) != cudaSuccess)
    h->sms = 0;
  return h->sms > 0 ? h->sms : 1;
}

// Shared memory of a resident march with ks steps per exchange: fields with a halo
// of 2 ks, push values with 2 ks - 1, per-node constants on the first sub-step's
// output region (halo 2 ks - 2).
size_t res_smem_bytes(const lks_problem_desc& d, bool adjoint, int cfg, int ks = 1) {
  const size_t rs = d.real_type == LKS_REAL_F64 ? 8 : 4;
  const int tx = kResCfg[cfg][0], ty = kResCfg[cfg][1], hh = 2 * ks;
  const size_t a2 = (size_t)(tx + 2 * hh) * (ty + 2 * hh), a1 = (size_t)(tx + 2 * hh - 2) * (ty + 2 * hh - 2),
               no = (size_t)(tx + 2 * hh - 4) * (ty + 2 * hh - 4);
  if (adjoint) return rs * (8 * a2 + 9 * a1 + 3 * no);
  return rs * ((d.thermal ? 4 : 3) * a2 + (d.thermal ? 19 : 9) * a1 + no);
}

// Tile shape of a resident march: the most tiles that still leave one CTA per SM
// and fit the shared memory of an SM; none if the lattice needs more CTAs than SMs
// (the one-launch-per-step path runs then).
ResPlan plan_resident(lks_handle* h, bool adjoint) {
  ResPlan best;
  const int sms = device_sms(h);
  int optin = 0;
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device);
  for (int k = 0; k < kNResCfg; ++k) {
    const int nt = ((h->d.nx + kResCfg[k][0] - 1) / kResCfg[k][0]) * ((h->d.ny + kResCfg[k][1] - 1) / kResCfg[k][1]);
    if (res_smem_bytes(h->d, adjoint, k) + 1024 > (size_t)optin) continue;
    if (nt <= sms && nt > best.ntiles) {
      best.cfg = k;
      best.ntiles = nt;
    }
  }
  return best;
}

// Steps per exchange of a resident march on tile shape cfg: res_steps (automatic:
// kResStepsAuto), lowered until the band fits the tile twice and the shared memory
// fits an SM; FP64 keeps one step per exchange.  The automatic choice is one step:
// on a 512 x 256 channel the step is bound by the work inside the CTA, and two
// steps per exchange measured 7.2 / 5.4 us per forward / adjoint step against 4.5 /
// 4.7 us with one.
constexpr int kResStepsAuto = 1;
int res_steps_for(lks_handle* h, bool adjoint, int cfg) {
  if (h->d.real_type != LKS_REAL_F32) return 1;
  int optin = 0;
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device);
  int ks = h->d.res_steps > 0 ? h->d.res_steps : kResStepsAuto;
  while (ks > 1 && (4 * ks > std::min(kResCfg[cfg][0], kResCfg[cfg][1]) ||
                    res_smem_bytes(h->d, adjoint, cfg, ks) + 1024 > (size_t)optin))
    --ks;
  return ks;
}

bool resident_wanted(lks_handle* h, bool adjoint) {
  if (h->d.exec_path == LKS_PATH_STEP || h->d.exec_path == LKS_PATH_COLUMN || !h->d.steady) return false;
  if (lks_host::step_kernels_only(h->d)) return false;  // terms only the per-step kernels carry
  if (adjoint && h->d.thermal) return false;
  int coop = 0;
  cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, h->device);
  return coop && plan_resident(h, adjoint).ntiles > 0;
}

template <typename R, bool TH, int TXR, int TYR, int NT, int KS>
lks_status launch_fwd_resident_cfg(lks_handle* h, int n) {
  const auto& d = h->d;
  const int ntx = (d.nx + TXR - 1) / TXR, nt = ntx * ((d.ny + TYR - 1) / TYR);
  const size_t smem = (size_t)(KS == 1 ? fwd_res_smem_elems<TH, TXR, TYR>() : fwd_tb_smem_elems<TH, TXR, TYR, KS>()) *
                      sizeof(R);
  void (*kern)(ResArgs<R>, Geom, Coef<R>);
  if constexpr (KS == 1) kern = fwd_resident_kernel<R, TH, TXR, TYR, NT>;
  else kern = fwd_resident_tb_kernel<R, TH, TXR, TYR, NT, KS>;
  CKH(h, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  CKH(h, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, smem));
  if (per_sm < 1 || nt > per_sm * device_sms(h)) return fail(h, LKS_ERR_INVALID_ARG, "resident march does not fit");
  ResArgs<R> a{};
  for (int b = 0; b < 2; ++b)
    for (int f = 0; f < h->L.nF; ++f) a.buf[b][f] = state_ptr<R>(h, b, f);
  a.cur = h->cur;
  a.gamma = fld<R>(h, h->L.gamma, 0);
  a.flags = reinterpret_cast<int*>(h->ws + h->L.flags);
  a.status = reinterpret_cast<int*>(h->ws + h->L.status);
  a.n_steps = n;
  a.t0 = h->t;
  a.u_in = (R)inlet_amp(d, h->t + 1);
  a.ntx = ntx;
  Geom g = make_geom(d);
  Coef<R> c = make_coef<R>(d);
  CKH(h, cudaMemsetAsync(a.flags, 0, sizeof(int) * nt, h->stream));
  void* args[] = {&a, &g, &c};
  CKH(h, cudaLaunchCooperativeKernel((const void*)kern, dim3(nt), dim3(NT), args, smem, h->stream));
  h->cur = (h->cur + (KS == 1 ? n : (n + KS - 1) / KS)) & 1;  // buffer of the last exchange
  h->res_steps_fwd = KS;
  h->t += n;
  h->fwd_steps += n;
  h->launches++;
  h->fwd_path = LKS_PATH_RESIDENT;
  return LKS_OK;
}

template <typename R, int TXR, int TYR, int NT, int KS>
lks_status launch_adj_resident_cfg(lks_handle* h, int n) {
  const auto& d = h->d;
  const int ntx = (d.nx + TXR - 1) / TXR, nt = ntx * ((d.ny + TYR - 1) / TYR);
  const size_t smem = (size_t)(KS == 1 ? adj_res_smem_elems<TXR, TYR>() : adj_tb_smem_elems<TXR, TYR, KS>()) * sizeof(R);
  void (*kern)(ResArgs<R>, Geom, Coef<R>);
  if constexpr (KS == 1) kern = adj_resident_kernel<R, TXR, TYR, NT>;
  else kern = adj_resident_tb_kernel<R, TXR, TYR, NT, KS>;
  CKH(h, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  CKH(h, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, smem));
  if (per_sm < 1 || nt > per_sm * device_sms(h)) return fail(h, LKS_ERR_INVALID_ARG, "resident march does not fit");
  ResArgs<R> a{};
  for (int b = 0; b < 2; ++b)
    for (int f = 0; f < 6; ++f) a.buf[b][f] = adj_ptr<R>(h, b, f);
  a.cur = h->acur;
  a.u = state_ptr<R>(h, h->cur, 1);
  a.v = state_ptr<R>(h, h->cur, 2);
  a.gamma = fld<R>(h, h->L.gamma, 0);
  a.emap = reinterpret_cast<const R*>(h->ws + h->L.emap);
  a.flags = reinterpret_cast<int*>(h->ws + h->L.flags);
  a.status = reinterpret_cast<int*>(h->ws + h->L.status);
  a.n_steps = n;
  a.ntx = ntx;
  Geom g = make_geom(d);
  Coef<R> c = make_coef<R>(d);
  CKH(h, cudaMemsetAsync(a.flags, 0, sizeof(int) * nt, h->stream));
  void* args[] = {&a, &g, &c};
  CKH(h, cudaLaunchCooperativeKernel((const void*)kern, dim3(nt), dim3(NT), args, smem, h->stream));
  h->acur = (h->acur + (KS == 1 ? n : (n + KS - 1) / KS)) & 1;  // buffer of the last exchange
  h->res_steps_adj = KS;
  h->adj_steps += n;
  h->launches++;
  h->adj_path = LKS_PATH_RESIDENT;
  return LKS_OK;
}

template <typename R, bool TH>
lks_status launch_fwd_resident_th(lks_handle* h, int n, int k, int ks) {
  if constexpr (std::is_same_v<R, float>) {
    if (k == 0 && ks == 3) return launch_fwd_resident_cfg<R, TH, 64, 16, 512, 3>(h, n);
    if (k == 0 && ks == 2) return launch_fwd_resident_cfg<R, TH, 64, 16, 512, 2>(h, n);
    if (k == 1 && ks == 3) return launch_fwd_resident_cfg<R, TH, 32, 16, 256, 3>(h, n);
    if (k == 1 && ks == 2) return launch_fwd_resident_cfg<R, TH, 32, 16, 256, 2>(h, n);
    if (k == 2 && ks == 2) return launch_fwd_resident_cfg<R, TH, 32, 8, 256, 2>(h, n);
    if (k == 3 && ks == 3) return launch_fwd_resident_cfg<R, TH, 64, 14, 512, 3>(h, n);
    if (k == 3 && ks == 2) return launch_fwd_resident_cfg<R, TH, 64, 14, 512, 2>(h, n);
  }
  if (k == 0) return launch_fwd_resident_cfg<R, TH, 64, 16, 512, 1>(h, n);
  if (k == 1) return launch_fwd_resident_cfg<R, TH, 32, 16, 256, 1>(h, n);
  // 768 threads: the forward's phases on a 64 x 14 tile take fewer, fuller passes
  // (the 62 x 12 coefficient region in one); 6 % faster per step on the 512 x 256
  // channel than 640, 8 % than 512, and 896 was slower again
  if (k == 3) return launch_fwd_resident_cfg<R, TH, 64, 14, 768, 1>(h, n);
  return launch_fwd_resident_cfg<R, TH, 32, 8, 256, 1>(h, n);
}

template <typename R>
lks_status launch_fwd_resident(lks_handle* h, int n) {
  const int k = plan_resident(h, false).cfg;
  const int ks = res_steps_for(h, false, k);
  return h->d.thermal ? launch_fwd_resident_th<R, true>(h, n, k, ks) : launch_fwd_resident_th<R, false>(h, n, k, ks);
}

template <typename R>
lks_status launch_adj_resident(lks_handle* h, int n) {
  const int k = plan_resident(h, true).cfg;
  const int ks = res_steps_for(h, true, k);
  if constexpr (std::is_same_v<R, float>) {
    if (k == 0 && ks == 3) return launch_adj_resident_cfg<R, 64, 16, 512, 3>(h, n);
    if (k == 0 && ks == 2) return launch_adj_resident_cfg<R, 64, 16, 512, 2>(h, n);
    if (k == 1 && ks == 3) return launch_adj_resident_cfg<R, 32, 16, 256, 3>(h, n);
    if (k == 1 && ks == 2) return launch_adj_resident_cfg<R, 32, 16, 256, 2>(h, n);
    if (k == 2 && ks == 2) return launch_adj_resident_cfg<R, 32, 8, 256, 2>(h, n);
    if (k == 3 && ks == 3) return launch_adj_resident_cfg<R, 64, 14, 512, 3>(h, n);
    if (k == 3 && ks == 2) return launch_adj_resident_cfg<R, 64, 14, 512, 2>(h, n);
  }
  if (k == 0) return launch_adj_resident_cfg<R, 64, 16, 512, 1>(h, n);
  if (k == 1) return launch_adj_resident_cfg<R, 32, 16, 256, 1>(h, n);
  if (k == 3) return launch_adj_resident_cfg<R, 64, 14, 512, 1>(h, n);
  return launch_adj_resident_cfg<R, 32, 8, 256, 1>(h, n);
}

// ------------------------------------------------------------------------------------
// TMA-staged per-step kernels (FP32, nx % 4 == 0)
// ------------------------------------------------------------------------------------
// Tiles of 32 x 16 outputs, 640 threads per CTA: the 34 x 18 coefficient region
// takes one pass; the forward fits two CTAs per SM, the adjoint one.  On the
// 1024 x 512 thermal gradient this is 15 % faster than 64 x 8 tiles with 256 / 512
// threads, whose coefficient region took uneven passes (the other threads waiting
// at the barrier), and 7.5 % faster than 64 x 8 with 352 / 704.
constexpr int kFwdNT = 640, kAdjNT = 640;

bool tma_ok(lks_handle* h) {
  // the energy loss is carried by the plain per-step kernels only
  return h->d.real_type == LKS_REAL_F32 && (h->d.nx % 4) == 0 && encode_fn() != nullptr && h->d.kappa_E == 0.0;
}

// Tensor map of one field (nx x ny floats) for boxes of bw x bh, cached per handle.
lks_status field_map(lks_handle* h, const void* ptr, int bw, int bh, CUtensorMap* out) {
  const uint64_t key = reinterpret_cast<uint64_t>(ptr) ^ ((uint64_t)bw << 48) ^ ((uint64_t)bh << 56);
  auto it = h->tmaps.find(key);
  if (it != h->tmaps.end()) {
    *out = it->second;
    return LKS_OK;
  }
  CUtensorMap m;
  const cuuint64_t dims[2] = {(cuuint64_t)h->d.nx, (cuuint64_t)h->d.ny};
  const cuuint64_t strides[1] = {(cuuint64_t)h->d.nx * 4};
  const cuuint32_t box[2] = {(cuuint32_t)bw, (cuuint32_t)bh};
  const cuuint32_t es[2] = {1, 1};
  const CUresult r = encode_fn()(&m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(ptr), dims, strides, box, es,
                                 CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                 CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(h, LKS_ERR_CUDA, "cuTensorMapEncodeTiled failed");
  h->tmaps.emplace(key, m);
  *out = m;
  return LKS_OK;
}

template <typename K>
int persistent_grid(lks_handle* h, K kern, int nt, size_t smem, int ntiles) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, nt, smem) != cudaSuccess || per_sm < 1)
    per_sm = 1;
  return std::max(1, std::min(ntiles, per_sm * device_sms(h)));
}

// Warp-column kernels: asked for, or the lattice has at least four column tiles per
// SM (below that the per-tile TMA kernels, with fewer edge tiles, are faster).
bool use_col(lks_handle* h) {
  if (lks_host::step_kernels_only(h->d)) return false;  // terms only the per-step kernels carry
  if (h->d.exec_path == LKS_PATH_COLUMN) return true;
  if (h->d.exec_path == LKS_PATH_STEP) return false;  // the per-tile kernels, as asked
  const long long tiles = (long long)((h->d.nx + C2_W - 1) / C2_W) * ((h->d.ny + Col2Geo<C2_R>::H - 1) / Col2Geo<C2_R>::H);
  return tiles >= 4ll * device_sms(h);
}

// Warp-column forward (FP32, one lattice): fwd_col2_kernel, one CTA per 60 x 40 tile
// (two columns per lane); thermal problems then run fwd_colT_kernel on the same tiles
// for T.
lks_status launch_fwd_col(lks_handle* h, int t_new, double* Jpartial, float* tu, float* tv, float* tT) {
  const auto& d = h->d;
  const int src = h->cur, dst = 1 - h->cur;
  using G2 = Col2Geo<C2_R>;
  const float* fsrc[4] = {state_ptr<float>(h, src, 0), state_ptr<float>(h, src, 1), state_ptr<float>(h, src, 2),
                          fld<float>(h, h->L.mat, 0)};
  TmaMaps<4> maps;
  lks_status st;
  for (int f = 0; f < 4; ++f)
    if ((st = field_map(h, fsrc[f], C2_BW, G2::BH, &maps.m[f])) != LKS_OK) return st;
  Col2Args a;
  std::memset(&a, 0, sizeof(a));
  for (int f = 0; f < 3; ++f) a.out[f] = state_ptr<float>(h, dst, f);
  a.traj_u = tu;
  a.traj_v = tv;
  a.J_partial = Jpartial;
  a.status = reinterpret_cast<int*>(h->ws + h->L.status);
  a.u_in = (float)inlet_amp(d, t_new);
  a.ntx = (d.nx + C2_W - 1) / C2_W;
  const int grid = a.ntx * ((d.ny + G2::H - 1) / G2::H);
  static bool attr = false;
  if (!attr) {
    CKH(h, cudaFuncSetAttribute(fwd_col2_kernel<C2_R, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)G2::smem));
    attr = true;
  }
  fwd_col2_kernel<C2_R, false><<<grid, COL_NT, G2::smem, h->stream>>>(maps, a, make_geom(d), make_coef<float>(d));
  CKH(h, cudaGetLastError());
  if (d.thermal) {
    const float* tsrc[4] = {state_ptr<float>(h, src, 3), fsrc[1], fsrc[2], fld<float>(h, h->L.mat, 0) + 2 * h->L.N};
    TmaMaps<4> tmaps;
    for (int f = 0; f < 4; ++f)
      if ((st = field_map(h, tsrc[f], C2_BW, G2::BH, &tmaps.m[f])) != LKS_OK) return st;
    ColTArgs b;
    std::memset(&b, 0, sizeof(b));
    b.T_out = state_ptr<float>(h, dst, 3);
    b.traj_T = tT;
    b.u_new = a.out[1];
    b.v_new = a.out[2];
    b.J_partial = Jpartial;
    b.status = a.status;
    b.ntx = a.ntx;
    static bool attrT = false;
    if (!attrT) {
      CKH(h, cudaFuncSetAttribute(fwd_colT_kernel<C2_R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G2::smem));
      attrT = true;
    }
    fwd_colT_kernel<C2_R><<<grid, COL_NT, G2::smem, h->stream>>>(tmaps, b, make_geom(d), make_coef<float>(d));
    CKH(h, cudaGetLastError());
    h->launches++;
  }
  h->cur = dst;
  h->t = t_new;
  h->fwd_steps++;
  h->launches++;
  h->fwd_path = LKS_PATH_COLUMN;
  return LKS_OK;
}

template <bool TH>
lks_status launch_fwd_tma(lks_handle* h, int t_new, double* Jpartial, float* tu, float* tv, float* tT) {
  if (use_col(h)) return launch_fwd_col(h, t_new, Jpartial, tu, tv, TH ? tT : nullptr);
  constexpr int NF = fwd_tma_nf(TH);
  constexpr int BW = kFwdTX + 8, BH = kFwdTY + 4;
  const auto& d = h->d;
  const int src = h->cur, dst = 1 - h->cur;
  TmaMaps<NF> maps;
  lks_status st;
  const float* mat = fld<float>(h, h->L.mat, 0);
  const float* fsrc[6] = {state_ptr<float>(h, src, 0), state_ptr<float>(h, src, 1), state_ptr<float>(h, src, 2), mat,
                          TH ? state_ptr<float>(h, src, 3) : nullptr, mat + 2 * h->L.N};
  for (int f = 0; f < NF; ++f)
    if ((st = field_map(h, fsrc[f], BW, BH, &maps.m[f])) != LKS_OK) return st;
  FwdOutMaps<TH> omaps;
  {
    const float* outs[7] = {state_ptr<float>(h, dst, 0), state_ptr<float>(h, dst, 1), state_ptr<float>(h, dst, 2),
                            TH ? state_ptr<float>(h, dst, 3) : nullptr, tu, tv, tT};
    int nf = 0;
    for (int k = 0; k < 7; ++k) {
      if (!outs[k]) continue;
      if ((st = field_map(h, outs[k], kFwdTX, kFwdTY, &omaps.m[nf++])) != LKS_OK) return st;
    }
  }
  FwdTmaArgs<TH> a;
  a.drho_n = state_ptr<float>(h, dst, 0);
  a.u_n = state_ptr<float>(h, dst, 1);
  a.v_n = state_ptr<float>(h, dst, 2);
  a.T_n = TH ? state_ptr<float>(h, dst, 3) : nullptr;
  a.gamma = fld<float>(h, h->L.gamma, 0);
  a.u_in = (float)inlet_amp(d, t_new);
  a.J_partial = Jpartial;
  a.status = reinterpret_cast<int*>(h->ws + h->L.status);
  a.traj_u = tu;
  a.traj_v = tv;
  a.traj_T = tT;
  a.ntx = (d.nx + kFwdTX - 1) / kFwdTX;
  a.ntiles = a.ntx * ((d.ny + kFwdTY - 1) / kFwdTY);
  const size_t smem = fwd_tma_smem_bytes<TH, kFwdTX, kFwdTY>();
  a.work = nullptr;
  a.designs = nullptr;
  a.u_in_d = nullptr;
  auto kern = fwd_tma_kernel<TH, false, kFwdTX, kFwdTY, kFwdNT>;
  if (!h->tma_grid_fwd) {
    CKH(h, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    h->tma_grid_fwd = persistent_grid(h, kern, kFwdNT, smem, a.ntiles);
  }
  if (Jpartial && h->tma_grid_fwd > h->L.fwd_blocks) return fail(h, LKS_ERR_WORKSPACE, "objective partials undersized");
  kern<<<h->tma_grid_fwd, kFwdNT, smem, h->stream>>>(maps, omaps, a, make_geom(d), make_coef<float>(d));
  CKH(h, cudaGetLastError());
  h->cur = dst;
  h->t = t_new;
  h->fwd_steps++;
  h->launches++;
  h->fwd_path = LKS_PATH_STEP;
  return LKS_OK;
}

// Warp-column adjoint (FP32, non-thermal, one lattice): one CTA per 28 x 32 tile.
template <bool SAME>
lks_status launch_adj_col(lks_handle* h, const float* u1, const float* v1, const float* u0, const float* v0,
                          float* sens, int sens_flow) {
  constexpr int NF = acol_nf(SAME);
  const auto& d = h->d;
  const int src = h->acur, dst = 1 - h->acur;
  TmaMaps<NF> maps;
  lks_status st;
  const float* mat = fld<float>(h, h->L.mat, 0);
  const float* fs[12] = {adj_ptr<float>(h, src, 0), adj_ptr<float>(h, src, 1), adj_ptr<float>(h, src, 2),
                         adj_ptr<float>(h, src, 3), adj_ptr<float>(h, src, 4), adj_ptr<float>(h, src, 5),
                         u1, v1, u0, v0, mat + h->L.N, mat};  // ..., alpha, 1/(1+alpha)
  int f = 0;
  for (int q = 0; q < 12; ++q) {
    if (SAME && (q == 8 || q == 9)) continue;
    if ((st = field_map(h, fs[q], COL_BW, ACOL_BH, &maps.m[f++])) != LKS_OK) return st;
  }
  AdjColArgs a;
  std::memset(&a, 0, sizeof(a));
  for (int q = 0; q < 6; ++q) a.m0[q] = adj_ptr<float>(h, dst, q);
  a.gamma = fld<float>(h, h->L.gamma, 0);
  a.emap = reinterpret_cast<const float*>(h->ws + h->L.emap);
  a.sens = sens;
  a.sens_flow = sens_flow;
  a.status = reinterpret_cast<int*>(h->ws + h->L.status);
  a.ntx = (d.nx + COL_W - 1) / COL_W;
  const int grid = a.ntx * ((d.ny + ACOL_H - 1) / ACOL_H);
  static bool attr_set = false;  // per process: the attribute belongs to the kernel
  if (!attr_set) {
    CKH(h, cudaFuncSetAttribute(adj_col_kernel<SAME, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)acol_smem_bytes(SAME)));
    attr_set = true;
  }
  adj_col_kernel<SAME, false>
      <<<grid, COL_NT, acol_smem_bytes(SAME), h->stream>>>(maps, a, make_geom(d), make_coef<float>(d));
  CKH(h, cudaGetLastError());
  h->acur = dst;
  h->adj_steps++;
  h->launches++;
  h->adj_path = LKS_PATH_COLUMN;
  return LKS_OK;
}

template <bool TH, bool SAME>
lks_status launch_adj_tma(lks_handle* h, const float* u1, const float* v1, const float* u0, const float* v0,
                          const float* T0, float* sens, int sens_flow, int sens_thermal) {
  if constexpr (!TH)
    if (use_col(h)) return launch_adj_col<SAME>(h, u1, v1, u0, v0, sens, sens_flow);
  constexpr int NF = adj_tma_nf(TH, SAME);
  constexpr int NA = TH ? 9 : 6;
  constexpr int BW = kAdjTX + 8, BH = kAdjTY + 4;
  const auto& d = h->d;
  const int src = h->acur, dst = 1 - h->acur;
  TmaMaps<NF> maps;
  lks_status st;
  int f = 0;
  for (int q = 0; q < NA; ++q)
    if ((st = field_map(h, adj_ptr<float>(h, src, q), BW, BH, &maps.m[f++])) != LKS_OK) return st;
  const float* mat = fld<float>(h, h->L.mat, 0);
  const float* extra[8] = {u1, v1, u0, v0, mat + h->L.N, mat, T0, mat + 2 * h->L.N};  // ..., alpha, 1/(1+alpha), T0, B
  for (int q = 0; q < 8; ++q) {
    if (SAME && (q == 2 || q == 3)) continue;
    if (!TH && q >= 6) continue;
    if ((st = field_map(h, extra[q], BW, BH, &maps.m[f++])) != LKS_OK) return st;
  }
  if (f != NF) return fail(h, LKS_ERR_INVALID_ARG, "tensor map count");
  AdjOutMaps<TH> omaps;
  for (int q = 0; q < NA; ++q)
    if ((st = field_map(h, adj_ptr<float>(h, dst, q), kAdjTX, kAdjTY, &omaps.m[q])) != LKS_OK) return st;
  AdjTmaArgs<TH> a;
  for (int q = 0; q < 9; ++q) a.m0[q] = adj_ptr<float>(h, dst, q < NA ? q : 0);
  a.gamma = fld<float>(h, h->L.gamma, 0);
  a.emap = reinterpret_cast<const float*>(h->ws + h->L.emap);
  a.sens = sens;
  a.sens_flow = sens_flow;
  a.sens_thermal = sens_thermal;
  a.status = reinterpret_cast<int*>(h->ws + h->L.status);
  a.ntx = (d.nx + kAdjTX - 1) / kAdjTX;
  a.ntiles = a.ntx * ((d.ny + kAdjTY - 1) / kAdjTY);
  const size_t smem = adj_tma_smem_bytes<TH, SAME, kAdjTX, kAdjTY>();
  a.work = nullptr;
  a.designs = nullptr;
  a.pitch = d.nx;
  auto kern = adj_tma_kernel<TH, SAME, false, kAdjTX, kAdjTY, kAdjNT>;
  int& grid = h->tma_grid_adj[TH ? 1 : 0][SAME ? 1 : 0];
  if (!grid) {
    CKH(h, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    grid = persistent_grid(h, kern, kAdjNT, smem, a.ntiles);
  }
  kern<<<grid, kAdjNT, smem, h->stream>>>(maps, omaps, a, make_geom(d), make_coef<float>(d));
  CKH(h, cudaGetLastError());
  h->acur = dst;
  h->adj_steps++;
  h->launches++;
  h->adj_path = LKS_PATH_STEP;
  return LKS_OK;
}

template <typename R>
lks_status launch_objective(lks_handle* h, const R* u, const R* v, const R* T, double* partial) {
  const auto& d = h->d;
  const Geom g = make_geom(d);
  const Coef<R> c = make_coef<R>(d);
  const R* gam = fld<R>(h, h->L.gamma, 0);
  if (d.thermal)
    objective_kernel<R, true><<<h->L.obj_blocks, NTHREADS, 0, h->stream>>>(u, v, T, gam, g, c, partial);
  else
    objective_kernel<R, false><<<h->L.obj_blocks, NTHREADS, 0, h->stream>>>(u, v, T, gam, g, c, partial);
  CKH(h, cudaGetLastError());
  h->launches++;
  return LKS_OK;
}

int elementwise_grid(size_t n) { return lks_host::elementwise_blocks(n); }

// Relative change of one step of two fields (a0 -> a1, b0 -> b1):
// max(|da| + |db|) / max(|a1| + |b1|).  Reads two words back (synchronises the stream).
template <typename R>
lks_status step_change(lks_handle* h, const R* a0, const R* a1, const R* b0, const R* b1, double* rel) {
  unsigned* dv = reinterpret_cast<unsigned*>(h->ws + h->L.chg);
  CKH(h, cudaMemsetAsync(dv, 0, 2 * sizeof(unsigned), h->stream));
  change_kernel<R><<<elementwise_grid(h->L.N), 256, 0, h->stream>>>(a0, a1, b0, b1, h->L.N, dv);
  CKH(h, cudaGetLastError());
  h->launches++;
  unsigned hv[2] = {0u, 0u};
  CKH(h, cudaMemcpyAsync(hv, dv, sizeof(hv), cudaMemcpyDeviceToHost, h->stream));
  CKH(h, cudaStreamSynchronize(h->stream));
  float d = 0.f, m = 0.f;
  std::memcpy(&d, &hv[0], sizeof(float));
  std::memcpy(&m, &hv[1], sizeof(float));
  *rel = m > 0.f ? (double)d / (double)m : (double)d;
  return LKS_OK;
}

// Snapshot encode / decode of one field with a per-field scale (max |x|).
template <typename R, typename S>
__global__ void absmax_kernel(const R* __restrict__ x, size_t n, float* out) {
  float m = 0.f;
  for (size_t o = (size_t)blockIdx.x * blockDim.x + threadIdx.x; o < n; o += (size_t)gridDim.x * blockDim.x)
    m = fmaxf(m, fabsf((float)x[o]));
  for (int s = 16; s > 0; s >>= 1) m = fmaxf(m, __shfl_down_sync(0xffffffffu, m, s));
  if ((threadIdx.x & 31) == 0) atomicMax(reinterpret_cast<int*>(out), __float_as_int(m));
}

template <typename S>
__device__ __forceinline__ S to_snap(float v);
template <>
__device__ __forceinline__ float to_snap<float>(float v) { return v; }
template <>
__device__ __forceinline__ __nv_bfloat16 to_snap<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }
template <>
__device__ __forceinline__ __half to_snap<__half>(float v) { return __float2half_rn(v); }
__device__ __forceinline__ float from_snap(float v) { return v; }
__device__ __forceinline__ float from_snap(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ float from_snap(__half v) { return __half2float(v); }

template <typename R, typename S>
__global__ void encode_kernel(const R* __restrict__ x, S* __restrict__ y, size_t n, const float* scale) {
  const float s = *scale;
  const float inv = s > 0.f ? 1.f / s : 0.f;
  for (size_t o = (size_t)blockIdx.x * blockDim.x + threadIdx.x; o < n; o += (size_t)gridDim.x * blockDim.x)
    y[o] = to_snap<S>((float)x[o] * inv);
}
template <typename R, typename S>
__global__ void decode_kernel(const S* __restrict__ y, R* __restrict__ x, size_t n, const float* scale) {
  const float s = *scale;
  for (size_t o = (size_t)blockIdx.x * blockDim.x + threadIdx.x; o < n; o += (size_t)gridDim.x * blockDim.x)
    x[o] = (R)(from_snap(y[o]) * s);
}

// 16-bit level store (segment_type BF16 / F16): nT fields of N values each.  BF16
// keeps FP32's exponent range; FP16 covers the O(1e-5 .. 1) values of u, v, T here.
template <typename S>
__global__ void pack_level_kernel(const float* __restrict__ a, const float* __restrict__ b,
                                  const float* __restrict__ c, S* __restrict__ dst, size_t n) {
  for (size_t o = (size_t)blockIdx.x * blockDim.x + threadIdx.x; o < n; o += (size_t)gridDim.x * blockDim.x) {
    dst[o] = to_snap<S>(a[o]);
    dst[n + o] = to_snap<S>(b[o]);
    if (c) dst[2 * n + o] = to_snap<S>(c[o]);
  }
}
template <typename S>
__global__ void unpack_level_kernel(const S* __restrict__ src, float* __restrict__ dst, size_t n, int nf) {
  for (size_t o = (size_t)blockIdx.x * blockDim.x + threadIdx.x; o < n; o += (size_t)gridDim.x * blockDim.x)
    for (int f = 0; f < nf; ++f) dst[(size_t)f * n + o] = (float)src[(size_t)f * n + o];
}

// Level store of the unsteady adjoint (the plain trajectory at L.traj, or the segment
// buffer at L.seg): level `lev` holds u, v[, T].  With 16-bit levels a forward step
// writes into stage slot 2 and the level is packed from there; an adjoint step reads
// a level unpacked into stage slot 0 or 1.
template <typename R>
R* level_write_ptr(lks_handle* h, size_t base, int lev) {
  const auto& L = h->L;
  if (L.lvl16) return fld<R>(h, L.lvl_stage, 0) + (size_t)2 * L.nT * L.N;
  return fld<R>(h, base, 0) + (size_t)lev * L.nT * L.N;
}
template <typename R>
lks_status level_pack(lks_handle* h, size_t base, int lev, const R* u, const R* v, const R* T) {
  const auto& L = h->L;
  if constexpr (sizeof(R) == 4) {
    unsigned char* dst = h->ws + base + (size_t)lev * L.nT * L.N * 2;
    const float* c = L.nT == 3 ? T : nullptr;
    if (h->d.segment_type == LKS_SNAP_BF16)
      pack_level_kernel<__nv_bfloat16><<<elementwise_grid(L.N), 256, 0, h->stream>>>(
          u, v, c, reinterpret_cast<__nv_bfloat16*>(dst), L.N);
    else
      pack_level_kernel<__half><<<elementwise_grid(L.N), 256, 0, h->stream>>>(u, v, c, reinterpret_cast<__half*>(dst),
                                                                            L.N);
    CKH(h, cudaGetLastError());
    h->launches++;
  }
  return LKS_OK;
}
// After a forward step wrote level `lev` through level_write_ptr.
template <typename R>
lks_status level_written(lks_handle* h, size_t base, int lev) {
  const auto& L = h->L;
  if (!L.lvl16) return LKS_OK;
  const R* p = level_write_ptr<R>(h, base, lev);
  return level_pack<R>(h, base, lev, p, p + L.N, p + 2 * L.N);
}
// Level `lev` copied from fields u, v[, T] of the state.
template <typename R>
lks_status level_from_state(lks_handle* h, size_t base, int lev, const R* u, const R* v, const R* T) {
  const auto& L = h->L;
  if (L.lvl16) return level_pack<R>(h, base, lev, u, v, T);
  R* dst = fld<R>(h, base, 0) + (size_t)lev * L.nT * L.N;
  const R* src[3] = {u, v, T};
  for (int f = 0; f < L.nT; ++f)
    CKH(h, cudaMemcpyAsync(dst + (size_t)f * L.N, src[f], L.N * sizeof(R), cudaMemcpyDeviceToDevice, h->stream));
  return LKS_OK;
}
// FP32 (or FP64) fields of stored level `lev` for an adjoint step; 16-bit levels are
// unpacked into stage slot `slot` first.
template <typename R>
lks_status level_read(lks_handle* h, size_t base, int lev, int slot, const R** p) {
  const auto& L = h->L;
  if constexpr (sizeof(R) == 4) {
    if (L.lvl16) {
      float* dst = fld<float>(h, L.lvl_stage, 0) + (size_t)slot * L.nT * L.N;
      const unsigned char* src = h->ws + base + (size_t)lev * L.nT * L.N * 2;
      if (h->d.segment_type == LKS_SNAP_BF16)
        unpack_level_kernel<__nv_bfloat16><<<elementwise_grid(L.N), 256, 0, h->stream>>>(
            reinterpret_cast<const __nv_bfloat16*>(src), dst, L.N, L.nT);
      else
        unpack_level_kernel<__half><<<elementwise_grid(L.N), 256, 0, h->stream>>>(
            reinterpret_cast<const __half*>(src), dst, L.N, L.nT);
      CKH(h, cudaGetLastError());
      h->launches++;
      *p = dst;
      return LKS_OK;
    }
  }
  *p = fld<R>(h, base, 0) + (size_t)lev * L.nT * L.N;
  return LKS_OK;
}

template <typename R>
lks_status snapshot_store(lks_handle* h, int idx) {
  const auto& L = h->L;
  const size_t N = L.N;
  float* sc = reinterpret_cast<float*>(h->ws + L.scales) + (size_t)idx * 2 * L.nF;
  unsigned char* base = h->ws + L.snaps + (size_t)idx * L.nF * N * L.snap_elem;
  const int gsz = elementwise_grid(N);
  if (h->d.snapshot_type == LKS_SNAP_F32 && sizeof(R) == 4) {
    CKH(h, cudaMemcpyAsync(base, state_ptr<R>(h, h->cur, 0), N * L.nF * sizeof(R), cudaMemcpyDeviceToDevice,
                           h->stream));
    return LKS_OK;
  }
  CKH(h, cudaMemsetAsync(sc, 0, sizeof(float) * L.nF, h->stream));
  for (int f = 0; f < L.nF; ++f) {
    const R* x = state_ptr<R>(h, h->cur, f);
    absmax_kernel<R, float><<<gsz, 256, 0, h->stream>>>(x, N, sc + f);
    unsigned char* dst = base + (size_t)f * N * L.snap_elem;
    switch (h->d.snapshot_type) {
      case LKS_SNAP_BF16:
        encode_kernel<R, __nv_bfloat16><<<gsz, 256, 0, h->stream>>>(x, reinterpret_cast<__nv_bfloat16*>(dst), N, sc + f);
        break;
      case LKS_SNAP_F16:
        encode_kernel<R, __half><<<gsz, 256, 0, h->stream>>>(x, reinterpret_cast<__half*>(dst), N, sc + f);
        break;
      default:
        encode_kernel<R, float><<<gsz, 256, 0, h->stream>>>(x, reinterpret_cast<float*>(dst), N, sc + f);
    }
    h->launches += 2;
  }
  CKH(h, cudaGetLastError());
  return LKS_OK;
}

template <typename R>
lks_status snapshot_load(lks_handle* h, int idx) {
  const auto& L = h->L;
  const size_t N = L.N;
  const float* sc = reinterpret_cast<const float*>(h->ws + L.scales) + (size_t)idx * 2 * L.nF;
  const unsigned char* base = h->ws + L.snaps + (size_t)idx * L.nF * N * L.snap_elem;
  const int gsz = elementwise_grid(N);
  if (h->d.snapshot_type == LKS_SNAP_F32 && sizeof(R) == 4) {
    CKH(h, cudaMemcpyAsync(state_ptr<R>(h, h->cur, 0), base, N * L.nF * sizeof(R), cudaMemcpyDeviceToDevice,
                           h->stream));
    return LKS_OK;
  }
  for (int f = 0; f < L.nF; ++f) {
    R* x = state_ptr<R>(h, h->cur, f);
    const unsigned char* src = base + (size_t)f * N * L.snap_elem;
    switch (h->d.snapshot_type) {
      case LKS_SNAP_BF16:
        decode_kernel<R, __nv_bfloat16><<<gsz, 256, 0, h->stream>>>(reinterpret_cast<const __nv_bfloat16*>(src), x, N, sc + f);
        break;
      case LKS_SNAP_F16:
        decode_kernel<R, __half><<<gsz, 256, 0, h->stream>>>(reinterpret_cast<const __half*>(src), x, N, sc + f);
        break;
      default:
        decode_kernel<R, float><<<gsz, 256, 0, h->stream>>>(reinterpret_cast<const float*>(src), x, N, sc + f);
    }
    h->launches++;
  }
  CKH(h, cudaGetLastError());
  return LKS_OK;
}

// Material fields 1/(1+alpha), alpha, B of the current design (FP32 staged kernels).
template <typename R>
lks_status update_materials(lks_handle* h) {
  if constexpr (sizeof(R) == 4) {
    if (!tma_ok(h)) return LKS_OK;
    float* m = fld<float>(h, h->L.mat, 0);
    material_kernel<<<elementwise_grid(h->L.N), 256, 0, h->stream>>>(fld<float>(h, h->L.gamma, 0), h->L.N,
                                                                     make_coef<float>(h->d), m, m + h->L.N,
                                                                     h->d.thermal ? m + 2 * h->L.N : nullptr);
    CKH(h, cudaGetLastError());
    h->launches++;
  }
  return LKS_OK;
}

template <typename R>
lks_status forward_impl(lks_handle* h, const void* gamma_dev, double* J_dev) {
  const auto& d = h->d;
  const auto& L = h->L;
  const size_t fb = L.N * sizeof(R);
  if (gamma_dev != h->ws + L.gamma)
    CKH(h, cudaMemcpyAsync(h->ws + L.gamma, gamma_dev, fb, cudaMemcpyDeviceToDevice, h->stream));
  CKH(h, cudaMemsetAsync(h->ws + L.status, 0, sizeof(int), h->stream));
  if (!(d.steady && d.warm_start && h->phase >= 1)) {  // from rest (drho = 0, u = 0, T = 0)
    CKH(h, cudaMemsetAsync(h->ws + L.stA, 0, fb * L.nF, h->stream));
    h->cur = 0;
    h->t = 0;
  }
  if (lks_status ms = update_materials<R>(h); ms != LKS_OK) return ms;
  double* jfwd = reinterpret_cast<double*>(h->ws + L.jfwd);
  double* jobj = reinterpret_cast<double*>(h->ws + L.jobj);
  double* jval = reinterpret_cast<double*>(h->ws + L.jval);
  lks_status st;
  bool converged = true;
  if (d.steady) {
    if (!resident_wanted(h, false) && d.exec_path == LKS_PATH_RESIDENT)
      return fail(h, LKS_ERR_INVALID_ARG, "resident march unavailable");
    // fixed count: one chunk of n_steps; tol > 0: chunks, each followed by a measured step
    h->fwd_change = 0.0;
    converged = !(d.tol > 0.0);
    int done = 0, chunk = d.n_steps;
    for (;;) {
      if (chunk > 0 && resident_wanted(h, false)) {
        if ((st = launch_fwd_resident<R>(h, chunk)) != LKS_OK) return st;
      } else {
        for (int s = 0; s < chunk; ++s)
          if ((st = launch_fwd<R>(h, h->t + 1, nullptr, nullptr, nullptr, nullptr)) != LKS_OK) return st;
      }
      done += chunk;
      if (converged) break;
      const int prev = h->cur, path = h->fwd_path;  // the chunks' path stays the reported one
      if ((st = launch_fwd<R>(h, h->t + 1, nullptr, nullptr, nullptr, nullptr)) != LKS_OK) return st;
      if (chunk > 0) h->fwd_path = path;
      ++done;
      if ((st = step_change<R>(h, state_ptr<R>(h, prev, 1), state_ptr<R>(h, h->cur, 1), state_ptr<R>(h, prev, 2),
                               state_ptr<R>(h, h->cur, 2), &h->fwd_change)) != LKS_OK)
        return st;
      if (h->fwd_change <= d.tol) {
        converged = true;
        break;
      }
      if (done >= d.max_steps) break;
      chunk = std::min(d.n_steps, d.max_steps - done - 1);
    }
  } else {
    CKH(h, cudaMemsetAsync(jfwd, 0, sizeof(double) * L.fwd_blocks, h->stream));
    const bool plain = d.checkpoint_every == 0;
    if (plain)  // level 0 of the trajectory
      if ((st = level_from_state<R>(h, L.traj, 0, state_ptr<R>(h, h->cur, 1), state_ptr<R>(h, h->cur, 2),
                                    d.thermal ? state_ptr<R>(h, h->cur, 3) : nullptr)) != LKS_OK)
        return st;
    for (int t = 0; t < d.n_steps; ++t) {
      if (!plain && t % d.checkpoint_every == 0)
        if ((st = snapshot_store<R>(h, t / d.checkpoint_every)) != LKS_OK) return st;
      R *tu = nullptr, *tv = nullptr, *tT = nullptr;
      if (plain) {
        R* tr = level_write_ptr<R>(h, L.traj, t + 1);
        tu = tr;
        tv = tr + L.N;
        tT = d.thermal ? tr + 2 * L.N : nullptr;
      }
      if ((st = launch_fwd<R>(h, t + 1, t >= 1 ? jfwd : nullptr, tu, tv, tT)) != LKS_OK) return st;
      if (plain && (st = level_written<R>(h, L.traj, t + 1)) != LKS_OK) return st;
    }
  }
  R* u = state_ptr<R>(h, h->cur, 1);
  R* v = state_ptr<R>(h, h->cur, 2);
  R* T = d.thermal ? state_ptr<R>(h, h->cur, 3) : nullptr;
  if ((st = launch_objective<R>(h, u, v, T, jobj)) != LKS_OK) return st;
  int n2 = d.steady ? 0 : L.fwd_blocks;
  if ((d.steady && d.kappa_p != 0.0) || d.kappa_E != 0.0) {
    // + kappa_p J_p + kappa_E J_E of the final level, after the forward partials (the
    // per-step kernels summed the energy loss of levels 1 .. n - 1 into them)
    boundary_objective_kernel<R><<<1, NTHREADS, 0, h->stream>>>(state_ptr<R>(h, h->cur, 0), u, v, make_geom(d),
                                                                make_coef<R>(d), jfwd + n2);
    CKH(h, cudaGetLastError());
    h->launches++;
    n2 += 1;
  }
  reduce_partials_kernel<<<1, NTHREADS, 0, h->stream>>>(jobj, L.obj_blocks, jfwd, n2, jval);
  CKH(h, cudaGetLastError());
  h->launches++;
  if (J_dev) CKH(h, cudaMemcpyAsync(J_dev, jval, sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
  h->phase = 1;
  return converged ? LKS_OK : fail(h, LKS_ERR_NOT_CONVERGED, "forward march did not reach tol in max_steps");
}

template <typename R>
lks_status flush_sens(lks_handle* h) {
  const auto& L = h->L;
  flush_accum_kernel<R><<<elementwise_grid(L.N), 256, 0, h->stream>>>(fld<R>(h, L.sens, 0),
                                                                       reinterpret_cast<double*>(h->ws + L.sens64), L.N);
  CKH(h, cudaGetLastError());
  h->launches++;
  return LKS_OK;
}

template <typename R>
lks_status adjoint_impl(lks_handle* h) {
  const auto& d = h->d;
  const auto& L = h->L;
  const size_t fb = L.N * sizeof(R);
  if (!(d.steady && d.warm_start && h->have_adj)) {  // from zero (Eqs. afinitial, aginitial)
    CKH(h, cudaMemsetAsync(h->ws + L.adA, 0, fb * L.nA, h->stream));
    h->acur = 0;
  }
  h->have_adj = true;
  lks_status st;
  if (d.steady) {
    const R* u = state_ptr<R>(h, h->cur, 1);
    const R* v = state_ptr<R>(h, h->cur, 2);
    const R* T = d.thermal ? state_ptr<R>(h, h->cur, 3) : nullptr;
    h->adj_change = 0.0;
    bool converged = !(d.tol > 0.0);
    int done = 0, chunk = d.n_adj;
    for (;;) {
      if (chunk > 0 && resident_wanted(h, true)) {
        if ((st = launch_adj_resident<R>(h, chunk)) != LKS_OK) return st;
      } else {
        for (int it = 0; it < chunk; ++it)
          if ((st = launch_adj<R>(h, u, v, u, v, T, nullptr, 0, 0)) != LKS_OK) return st;
      }
      done += chunk;
      if (converged) break;
      const int prev = h->acur, path = h->adj_path;  // the chunks' path stays the reported one
      if ((st = launch_adj<R>(h, u, v, u, v, T, nullptr, 0, 0)) != LKS_OK) return st;
      if (chunk > 0) h->adj_path = path;
      ++done;
      if ((st = step_change<R>(h, adj_ptr<R>(h, prev, 1), adj_ptr<R>(h, h->acur, 1), adj_ptr<R>(h, prev, 2),
                               adj_ptr<R>(h, h->acur, 2), &h->adj_change)) != LKS_OK)
        return st;
      if (h->adj_change <= d.tol) {
        converged = true;
        break;
      }
      if (done >= d.max_steps) break;
      chunk = std::min(d.n_adj, d.max_steps - done - 1);
    }
    h->phase = 2;
    return converged ? LKS_OK : fail(h, LKS_ERR_NOT_CONVERGED, "adjoint march did not reach tol in max_steps");
  }
  CKH(h, cudaMemsetAsync(h->ws + L.sens, 0, fb, h->stream));
  CKH(h, cudaMemsetAsync(h->ws + L.sens64, 0, sizeof(double) * L.N, h->stream));
  const int n = d.n_steps;
  const int t_end = d.thermal ? 0 : 1;
  const int flush_every = 256;
  int since_flush = 0;
  // levels t + 1 and t of the level store at `base` (level numbers relative to `lo`);
  // 16-bit stores unpack level t into stage slot t & 1 (level t + 1 is there from the
  // step before, or unpacked first)
  auto levels = [&](size_t base, int lo, int t, bool first, const R** u1, const R** v1, const R** u0,
                    const R** v0, const R** T0) -> lks_status {
    const int t1 = std::min(t + 1, n);
    const R *p1, *p0;
    lks_status ls;
    if (first && t1 != t && (ls = level_read<R>(h, base, t1 - lo, t1 & 1, &p1)) != LKS_OK) return ls;
    if ((ls = level_read<R>(h, base, t - lo, t & 1, &p0)) != LKS_OK) return ls;
    if (t1 == t) p1 = p0;
    else if (!first) p1 = L.lvl16 ? fld<R>(h, L.lvl_stage, 0) + (size_t)(t1 & 1) * L.nT * L.N
                                  : fld<R>(h, base, 0) + (size_t)(t1 - lo) * L.nT * L.N;
    *u1 = p1;
    *v1 = p1 + L.N;
    *u0 = p0;
    *v0 = p0 + L.N;
    *T0 = d.thermal ? p0 + 2 * L.N : nullptr;
    return LKS_OK;
  };
  if (d.checkpoint_every == 0) {
    for (int t = n; t >= t_end; --t) {
      const R *u1, *v1, *u0, *v0, *T0;
      if ((st = levels(L.traj, 0, t, t == n, &u1, &v1, &u0, &v0, &T0)) != LKS_OK) return st;
      if ((st = launch_adj<R>(h, u1, v1, u0, v0, T0, fld<R>(h, L.sens, 0), t >= 1, t < n)) != LKS_OK) return st;
      if (++since_flush == flush_every) {
        if ((st = flush_sens<R>(h)) != LKS_OK) return st;
        since_flush = 0;
      }
    }
  } else {
    const int K = d.checkpoint_every;
    // Segment s recomputed from its snapshot into the store at `base`: level t_lo,
    // then the forward steps t_lo + 1 .. top.
    auto recompute = [&](int s, size_t base) -> lks_status {
      const Range range("segment recompute");
      const int t_lo = s * K, t_hi = std::min((s + 1) * K, n), top = std::min(t_hi + 1, n);
      lks_status rs;
      h->cur = 0;
      if ((rs = snapshot_load<R>(h, s)) != LKS_OK) return rs;
      if ((rs = level_from_state<R>(h, base, 0, state_ptr<R>(h, h->cur, 1), state_ptr<R>(h, h->cur, 2),
                                    d.thermal ? state_ptr<R>(h, h->cur, 3) : nullptr)) != LKS_OK)
        return rs;
      for (int t = t_lo; t < top; ++t) {
        R* p = level_write_ptr<R>(h, base, t + 1 - t_lo);
        if ((rs = launch_fwd<R>(h, t + 1, nullptr, p, p + L.N, d.thermal ? p + 2 * L.N : nullptr)) != LKS_OK)
          return rs;
        if ((rs = level_written<R>(h, base, t + 1 - t_lo)) != LKS_OK) return rs;
      }
      return LKS_OK;
    };
    // The adjoint steps over segment s, reading its levels from the store at `base`.
    auto march = [&](int s, size_t base) -> lks_status {
      const Range range("segment adjoint");
      const int t_lo = s * K, t_hi = std::min((s + 1) * K, n);
      const int t_stop = (s == 0) ? t_end : t_lo + 1;
      lks_status ms;
      for (int t = t_hi; t >= t_stop; --t) {
        const R *u1, *v1, *u0, *v0, *T0;
        if ((ms = levels(base, t_lo, t, t == t_hi, &u1, &v1, &u0, &v0, &T0)) != LKS_OK) return ms;
        if ((ms = launch_adj<R>(h, u1, v1, u0, v0, T0, fld<R>(h, L.sens, 0), t >= 1, t < n)) != LKS_OK) return ms;
        if (++since_flush == flush_every) {
          if ((ms = flush_sens<R>(h)) != LKS_OK) return ms;
          since_flush = 0;
        }
      }
      return LKS_OK;
    };
    const int last = L.n_ckpt - 1;
    if (!h->aux || !L.seg2) {
      for (int s = last; s >= 0; --s)
        if ((st = recompute(s, L.seg)) != LKS_OK || (st = march(s, L.seg)) != LKS_OK) return st;
    } else {
      // Segment s - 1 is recomputed on a second stream while the adjoint marches
      // segment s on the caller's stream, so that the recompute fills what the
      // adjoint's launches leave idle; segment s sits in store s & 1.  The caller's
      // stream waits for each recompute before its adjoint, and a recompute waits for
      // the adjoint that last read its store.  The last recompute (segment 0) is
      // waited for before the last adjoint, so the second stream ends joined.
      auto store = [&](int s) { return (s & 1) ? L.seg2 : L.seg; };
      // On every exit, error paths included, the caller's stream is restored and
      // made to wait for whatever the second stream holds.
      struct Restore {
        lks_handle* h;
        cudaStream_t s;
        ~Restore() {
          h->stream = s;
          if (cudaEventRecord(h->ev_fork, h->aux) == cudaSuccess) cudaStreamWaitEvent(s, h->ev_fork, 0);
        }
      } restore{h, h->stream};
      const cudaStream_t main = h->stream;
      CKH(h, cudaEventRecord(h->ev_fork, main));
      CKH(h, cudaStreamWaitEvent(h->aux, h->ev_fork, 0));
      h->stream = h->aux;
      if ((st = recompute(last, store(last))) != LKS_OK) return st;
      CKH(h, cudaEventRecord(h->ev_seg[last & 1], h->aux));
      for (int s = last; s >= 0; --s) {
        h->stream = main;
        CKH(h, cudaStreamWaitEvent(main, h->ev_seg[s & 1], 0));
        if (s > 0) {
          h->stream = h->aux;
          if (s < last) CKH(h, cudaStreamWaitEvent(h->aux, h->ev_adj[(s + 1) & 1], 0));
          if ((st = recompute(s - 1, store(s - 1))) != LKS_OK) return st;
          CKH(h, cudaEventRecord(h->ev_seg[(s - 1) & 1], h->aux));
          h->stream = main;
        }
        if ((st = march(s, store(s))) != LKS_OK) return st;
        CKH(h, cudaEventRecord(h->ev_adj[s & 1], main));
      }
    }
  }
  if ((st = flush_sens<R>(h)) != LKS_OK) return st;
  h->phase = 2;
  return LKS_OK;
}

template <typename R>
lks_status sensitivity_impl(lks_handle* h, void* out) {
  const auto& d = h->d;
  const auto& L = h->L;
  if (d.steady) {
    const Geom g = make_geom(d);
    const Coef<R> c = make_coef<R>(d);
    const R* u = state_ptr<R>(h, h->cur, 1);
    const R* v = state_ptr<R>(h, h->cur, 2);
    const R* T = d.thermal ? state_ptr<R>(h, h->cur, 3) : nullptr;
    const R* ux = adj_ptr<R>(h, h->acur, 1);
    const R* uy = adj_ptr<R>(h, h->acur, 2);
    const R* Tt = d.thermal ? adj_ptr<R>(h, h->acur, 6) : nullptr;
    const R* qx = d.thermal ? adj_ptr<R>(h, h->acur, 7) : nullptr;
    const R* qy = d.thermal ? adj_ptr<R>(h, h->acur, 8) : nullptr;
    const R* gam = fld<R>(h, L.gamma, 0);
    if (d.thermal)
      sensitivity_kernel<R, true><<<L.obj_blocks, NTHREADS, 0, h->stream>>>(u, v, T, ux, uy, Tt, qx, qy, gam, g, c,
                                                                            reinterpret_cast<R*>(out));
    else
      sensitivity_kernel<R, false><<<L.obj_blocks, NTHREADS, 0, h->stream>>>(u, v, T, ux, uy, Tt, qx, qy, gam, g, c,
                                                                             reinterpret_cast<R*>(out));
  } else {
    copy_shift_kernel<double, R><<<elementwise_grid(L.N), 256, 0, h->stream>>>(
        reinterpret_cast<const double*>(h->ws + L.sens64), reinterpret_cast<R*>(out), L.N, 0.0);
  }
  CKH(h, cudaGetLastError());
  h->launches++;
  return LKS_OK;
}

template <typename R>
lks_status upload_maps(lks_handle* h) {
  const auto& d = h->d;
  const double A = (1.0 / 6.0 - d.nu) * 4.5;
  h->emap_h.assign(lks::kEdgeMapLen, 0.0);
  for (int cls = 0; cls < 9; ++cls) flow_moment_map(A, cls, &h->emap_h[cls * 60], &h->emap_h[540 + cls * 6]);
  if (sizeof(R) == 8) {
    CKH(h, cudaMemcpy(h->ws + h->L.emap, h->emap_h.data(), lks::kEdgeMapLen * 8, cudaMemcpyHostToDevice));
  } else {
    h->emap_f.assign(h->emap_h.begin(), h->emap_h.end());
    CKH(h, cudaMemcpy(h->ws + h->L.emap, h->emap_f.data(), lks::kEdgeMapLen * 4, cudaMemcpyHostToDevice));
  }
  return LKS_OK;
}

lks_status check_handle(lks_handle* h) { return h ? LKS_OK : LKS_ERR_INVALID_ARG; }

lks3::Ctx3 ctx3(lks_handle* h) { return lks3::Ctx3{&h->d, &h->L3, h->ws, h->stream, &h->launches, &h->err}; }
size_t status_off(const lks_handle* h) { return h->is3 ? h->L3.status : h->L.status; }
lks_status reject3(lks_handle* h, const char* what) {
  return fail(h, LKS_ERR_INVALID_ARG, std::string(what) + " is not available for a D3Q19 problem");
}

}  // namespace

// ------------------------------------------------------------------------------------
// C ABI
// ------------------------------------------------------------------------------------
// Self-test of the bounded device waits (lks_selftest_wait): one thread waits on a
// tile flag nothing sets (0) or on an mbarrier no copy completes (1); the wait gives
// up after its iteration limit and records LKS_ERR_TIMEOUT in *status.
static __global__ void selftest_wait_kernel(int which, int* flag, int* status) {
  __shared__ uint64_t bar;
  if (threadIdx.x != 0) return;
  if (which == 0) {
    wait_flag(flag, 1, status);
  } else {
    mbar_init(&bar, 1);
    fence_mbar_init();
    if (!mbar_wait(&bar, 0)) raise_status(status, LKS_ERR_TIMEOUT);
  }
}

extern "C" {

const char* lks_status_string(lks_status s) {
  switch (s) {
    case LKS_OK: return "ok";
    case LKS_ERR_INVALID_ARG: return "invalid argument";
    case LKS_ERR_WORKSPACE: return "workspace too small or misaligned";
    case LKS_ERR_CUDA: return "CUDA error";
    case LKS_ERR_UNSTABLE: return "non-finite or runaway velocity";
    case LKS_ERR_NOT_CONVERGED: return "not converged";
    case LKS_ERR_TIMEOUT: return "device wait timed out";
    case LKS_ERR_STATE: return "calls out of order";
  }
  return "unknown status";
}

const char* lks_last_error(const lks_handle* h) { return h ? h->err.c_str() : "null handle"; }

lks_status lks_workspace_size(const lks_problem_desc* desc, size_t* bytes) {
  if (!bytes) return LKS_ERR_INVALID_ARG;
  lks_status s = check_desc(desc, nullptr);
  if (s != LKS_OK) return s;
  *bytes = desc->lattice == LKS_LATTICE_D3Q19 ? lks3::make_layout3(*desc).total : make_layout(desc).total;
  return LKS_OK;
}

lks_status lks_create(const lks_problem_desc* desc, void* workspace, size_t bytes, void* stream,
                      lks_handle** out) {
  if (!out) return LKS_ERR_INVALID_ARG;
  *out = nullptr;
  std::string why;
  lks_status s = check_desc(desc, &why);
  if (s != LKS_OK) return s;
  if (desc->lattice == LKS_LATTICE_D3Q19) {
    const lks3::Layout3 L3 = lks3::make_layout3(*desc);
    if (!workspace || bytes < L3.total || (reinterpret_cast<uintptr_t>(workspace) % kAlign) != 0)
      return LKS_ERR_WORKSPACE;
    lks_handle* h = new (std::nothrow) lks_handle();
    if (!h) return LKS_ERR_INVALID_ARG;
    h->d = *desc;
    h->is3 = true;
    h->L3 = L3;
    h->ws = reinterpret_cast<unsigned char*>(workspace);
    h->ws_bytes = bytes;
    h->stream = reinterpret_cast<cudaStream_t>(stream);
    cudaGetDevice(&h->device);
    if ((s = lks3::upload_maps3(ctx3(h))) != LKS_OK) {
      delete h;
      return s;
    }
    *out = h;
    return LKS_OK;
  }
  const Layout L = make_layout(desc);
  if (!workspace || bytes < L.total || (reinterpret_cast<uintptr_t>(workspace) % kAlign) != 0)
    return LKS_ERR_WORKSPACE;
  lks_handle* h = new (std::nothrow) lks_handle();
  if (!h) return LKS_ERR_INVALID_ARG;
  h->d = *desc;
  h->L = L;
  h->ws = reinterpret_cast<unsigned char*>(workspace);
  h->ws_bytes = bytes;
  h->stream = reinterpret_cast<cudaStream_t>(stream);
  cudaGetDevice(&h->device);
  if (L.seg2) {
    bool ok = cudaStreamCreateWithFlags(&h->aux, cudaStreamNonBlocking) == cudaSuccess;
    for (cudaEvent_t* e : {&h->ev_fork, &h->ev_seg[0], &h->ev_seg[1], &h->ev_adj[0], &h->ev_adj[1]})
      ok = ok && cudaEventCreateWithFlags(e, cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
      delete h;
      return LKS_ERR_CUDA;
    }
  }
  s = desc->real_type == LKS_REAL_F64 ? set_smem_attrs<double>() : set_smem_attrs<float>();
  if (s == LKS_OK) s = desc->real_type == LKS_REAL_F64 ? upload_maps<double>(h) : upload_maps<float>(h);
  if (s != LKS_OK) {
    delete h;
    return s;
  }
  *out = h;
  return LKS_OK;
}

lks_status lks_destroy(lks_handle* h) {
  if (!h) return LKS_ERR_INVALID_ARG;
  delete h;
  return LKS_OK;
}

lks_status lks_forward(lks_handle* h, const void* gamma_dev, double* J_dev) {
  if (check_handle(h) != LKS_OK || !gamma_dev) return fail(h, LKS_ERR_INVALID_ARG, "null argument");
  const Range range("lks_forward");
  if (h->is3) {
    int path = LKS_PATH_STEP;
    const lks_status s = lks3::forward3(ctx3(h), gamma_dev, J_dev, &h->cur, &path);
    if (s == LKS_OK) {
      h->phase = 1;
      h->fwd_steps += h->d.n_steps;
      h->fwd_path = path;
    }
    return s;
  }
  return h->d.real_type == LKS_REAL_F64 ? forward_impl<double>(h, gamma_dev, J_dev)
                                        : forward_impl<float>(h, gamma_dev, J_dev);
}

lks_status alks_adjoint(lks_handle* h) {
  if (check_handle(h) != LKS_OK) return LKS_ERR_INVALID_ARG;
  if (h->phase < 1) return fail(h, LKS_ERR_STATE, "alks_adjoint before lks_forward");
  const Range range("alks_adjoint");
  if (h->is3) {
    int path = LKS_PATH_STEP;
    const lks_status s = lks3::adjoint3(ctx3(h), h->cur, &h->acur, &path);
    if (s == LKS_OK) {
      h->phase = 2;
      h->adj_steps += h->d.n_adj;
      h->adj_path = path;
    }
    return s;
  }
  return h->d.real_type == LKS_REAL_F64 ? adjoint_impl<double>(h) : adjoint_impl<float>(h);
}

lks_status lks_sensitivity(lks_handle* h, void* out) {
  if (check_handle(h) != LKS_OK || !out) return fail(h, LKS_ERR_INVALID_ARG, "null argument");
  if (h->phase < 2) return fail(h, LKS_ERR_STATE, "lks_sensitivity before alks_adjoint");
  const Range range("lks_sensitivity");
  if (h->is3) return lks3::sensitivity3(ctx3(h), h->cur, h->acur, out);
  return h->d.real_type == LKS_REAL_F64 ? sensitivity_impl<double>(h, out) : sensitivity_impl<float>(h, out);
}

lks_status lks_gradient_host(lks_handle* h, const void* gamma_host, double* J_host, void* grad_host) {
  if (check_handle(h) != LKS_OK || !gamma_host || !J_host || !grad_host)
    return fail(h, LKS_ERR_INVALID_ARG, "null argument");
  const size_t fb = h->is3 ? h->L3.N * h->L3.rsize : h->L.N * h->L.rsize;
  // The gradient is staged in the inactive adjoint buffer's first field, gamma in
  // the workspace copy itself (lks_forward copies device to device onto itself).
  unsigned char* g_dev = h->ws + (h->is3 ? h->L3.gamma : h->L.gamma);
  CKH(h, cudaMemcpyAsync(g_dev, gamma_host, fb, cudaMemcpyHostToDevice, h->stream));
  lks_status s = lks_forward(h, g_dev, nullptr);
  if (s == LKS_OK) s = alks_adjoint(h);
  if (s != LKS_OK) return s;
  const size_t adA = h->is3 ? h->L3.adA : h->L.adA, adB = h->is3 ? h->L3.adB : h->L.adB;
  unsigned char* grad_dev = h->ws + (h->acur == 0 ? adB : adA);
  if ((s = lks_sensitivity(h, grad_dev)) != LKS_OK) return s;
  CKH(h, cudaMemcpyAsync(grad_host, grad_dev, fb, cudaMemcpyDeviceToHost, h->stream));
  CKH(h, cudaMemcpyAsync(J_host, h->ws + (h->is3 ? h->L3.jval : h->L.jval), sizeof(double), cudaMemcpyDeviceToHost,
                         h->stream));
  int status = 0;
  CKH(h, cudaMemcpyAsync(&status, h->ws + status_off(h), sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  CKH(h, cudaStreamSynchronize(h->stream));
  if (status != 0) return fail(h, (lks_status)status, "device status set during the gradient");
  return LKS_OK;
}

lks_status lks_set_state(lks_handle* h, const void* gamma_dev, const void* rho_dev, const void* u_dev,
                         const void* v_dev, const void* T_dev, int32_t t) {
  if (check_handle(h) != LKS_OK || !gamma_dev || !rho_dev || !u_dev || !v_dev || (h->d.thermal && !T_dev))
    return fail(h, LKS_ERR_INVALID_ARG, "null argument");
  if (h->is3) return reject3(h, "lks_set_state");
  const size_t fb = h->L.N * h->L.rsize;
  CKH(h, cudaMemcpyAsync(h->ws + h->L.gamma, gamma_dev, fb, cudaMemcpyDeviceToDevice, h->stream));
  const void* src[4] = {rho_dev, u_dev, v_dev, T_dev};
  h->cur = 0;
  for (int f = 0; f < h->L.nF; ++f)
    CKH(h, cudaMemcpyAsync(h->ws + h->L.stA + (size_t)f * fb, src[f], fb, cudaMemcpyDeviceToDevice, h->stream));
  h->t = t;
  if (h->phase < 1) h->phase = 1;
  return h->d.real_type == LKS_REAL_F64 ? update_materials<double>(h) : update_materials<float>(h);
}

lks_status lks_get_state(lks_handle* h, void* rho_dev, void* u_dev, void* v_dev, void* T_dev) {
  if (check_handle(h) != LKS_OK || !rho_dev || !u_dev || !v_dev || ((h->d.thermal || h->is3) && !T_dev))
    return fail(h, LKS_ERR_INVALID_ARG, "null argument");
  void* dst[4] = {rho_dev, u_dev, v_dev, T_dev};
  if (h->is3) {  // drho, u, v, w
    const size_t fb3 = h->L3.N * h->L3.rsize;
    const size_t base3 = h->cur == 0 ? h->L3.stA : h->L3.stB;
    for (int f = 0; f < 4; ++f)
      CKH(h, cudaMemcpyAsync(dst[f], h->ws + base3 + (size_t)f * fb3, fb3, cudaMemcpyDeviceToDevice, h->stream));
    return LKS_OK;
  }
  const size_t fb = h->L.N * h->L.rsize;
  const size_t base = h->cur == 0 ? h->L.stA : h->L.stB;
  for (int f = 0; f < h->L.nF; ++f)
    CKH(h, cudaMemcpyAsync(dst[f], h->ws + base + (size_t)f * fb, fb, cudaMemcpyDeviceToDevice, h->stream));
  return LKS_OK;
}

lks_status lks_march(lks_handle* h, int32_t n) {
  if (check_handle(h) != LKS_OK || n < 0) return fail(h, LKS_ERR_INVALID_ARG, "bad argument");
  if (h->is3) return reject3(h, "lks_march");
  for (int s = 0; s < n; ++s) {
    lks_status st = h->d.real_type == LKS_REAL_F64
                        ? launch_fwd<double>(h, h->t + 1, nullptr, nullptr, nullptr, nullptr)
                        : launch_fwd<float>(h, h->t + 1, nullptr, nullptr, nullptr, nullptr);
    if (st != LKS_OK) return st;
  }
  return LKS_OK;
}

lks_status alks_set_adjoint(lks_handle* h, void* const* fields) {
  if (check_handle(h) != LKS_OK || !fields) return fail(h, LKS_ERR_INVALID_ARG, "null argument");
  if (h->is3) return reject3(h, "alks_set_adjoint");
  const size_t fb = h->L.N * h->L.rsize;
  h->acur = 0;
  h->have_adj = true;
  for (int f = 0; f < h->L.nA; ++f) {
    if (!fields[f]) return fail(h, LKS_ERR_INVALID_ARG, "null field");
    CKH(h, cudaMemcpyAsync(h->ws + h->L.adA + (size_t)f * fb, fields[f], fb, cudaMemcpyDeviceToDevice, h->stream));
  }
  return LKS_OK;
}

lks_status alks_get_adjoint(lks_handle* h, void* const* fields) {
  if (check_handle(h) != LKS_OK || !fields) return fail(h, LKS_ERR_INVALID_ARG, "null argument");
  if (h->is3) {
    const size_t fb3 = h->L3.N * h->L3.rsize;
    const size_t base3 = h->acur == 0 ? h->L3.adA : h->L3.adB;
    for (int f = 0; f < lks3::kNA3; ++f) {
      if (!fields[f]) return fail(h, LKS_ERR_INVALID_ARG, "null field");
      CKH(h, cudaMemcpyAsync(fields[f], h->ws + base3 + (size_t)f * fb3, fb3, cudaMemcpyDeviceToDevice, h->stream));
    }
    return LKS_OK;
  }
  const size_t fb = h->L.N * h->L.rsize;
  const size_t base = h->acur == 0 ? h->L.adA : h->L.adB;
  for (int f = 0; f < h->L.nA; ++f) {
    if (!fields[f]) return fail(h, LKS_ERR_INVALID_ARG, "null field");
    CKH(h, cudaMemcpyAsync(fields[f], h->ws + base + (size_t)f * fb, fb, cudaMemcpyDeviceToDevice, h->stream));
  }
  return LKS_OK;
}

lks_status alks_march(lks_handle* h, int32_t n) {
  if (check_handle(h) != LKS_OK || n < 0) return fail(h, LKS_ERR_INVALID_ARG, "bad argument");
  if (h->is3) return reject3(h, "alks_march");
  for (int s = 0; s < n; ++s) {
    lks_status st;
    if (h->d.real_type == LKS_REAL_F64) {
      const double* u = state_ptr<double>(h, h->cur, 1);
      const double* v = state_ptr<double>(h, h->cur, 2);
      const double* T = h->d.thermal ? state_ptr<double>(h, h->cur, 3) : nullptr;
      st = launch_adj<double>(h, u, v, u, v, T, nullptr, 0, 0);
    } else {
      const float* u = state_ptr<float>(h, h->cur, 1);
      const float* v = state_ptr<float>(h, h->cur, 2);
      const float* T = h->d.thermal ? state_ptr<float>(h, h->cur, 3) : nullptr;
      st = launch_adj<float>(h, u, v, u, v, T, nullptr, 0, 0);
    }
    if (st != LKS_OK) return st;
  }
  if (h->phase < 2) h->phase = 2;
  return LKS_OK;
}

lks_status lks_query(lks_handle* h, lks_stats* out) {
  if (check_handle(h) != LKS_OK || !out) return LKS_ERR_INVALID_ARG;
  int status = 0;
  CKH(h, cudaMemcpyAsync(&status, h->ws + status_off(h), sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  CKH(h, cudaStreamSynchronize(h->stream));
  out->forward_steps = h->fwd_steps;
  out->adjoint_steps = h->adj_steps;
  out->kernel_launches = h->launches;
  out->workspace_bytes = h->is3 ? h->L3.total : h->L.total;
  out->device_status = status;
  out->phase = h->phase;
  out->fwd_path = h->fwd_path;
  out->adj_path = h->adj_path;
  out->res_steps_fwd = h->res_steps_fwd;
  out->res_steps_adj = h->res_steps_adj;
  out->fwd_change = h->fwd_change;
  out->adj_change = h->adj_change;
  return status ? (lks_status)status : LKS_OK;
}

// ------------------------------------------------------------------------------------
// Allocation-free gradient (lks_gradient_noalloc): workspace in a static device array
// ------------------------------------------------------------------------------------
}  // extern "C"

namespace {
// Scratch of the allocation-free entry point; in host code this name is only a
// stand-in, the device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[LKS_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kMaxDevices] = {};

// Device address of the static scratch on the current device (looked up once per
// device, with that device current).
lks_status noalloc_scratch(void** out, int* dev_out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return LKS_ERR_CUDA;
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return LKS_ERR_CUDA;
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  *dev_out = dev;
  return LKS_OK;
}

// The nine edge-class maps travel as a kernel argument (4752 bytes, within the
// 32 KB parameter limit), so no host buffer is read after the call returns.
struct EdgeMaps {
  double v[lks::kEdgeMapLen];
};

template <typename R>
__global__ void fill_edge_maps_kernel(EdgeMaps m, R* dst) {
  for (int i = threadIdx.x; i < lks::kEdgeMapLen; i += blockDim.x) dst[i] = (R)m.v[i];
}

// Device-detected failures (instability, a bounded wait that gave up) set the status
// word in the scratch; the allocation-free call has no synchronising query, so the
// objective it returns is overwritten with NaN instead.
__global__ void flag_status_kernel(const int* status, double* J) {
  if (*status != 0) *J = __longlong_as_double(0x7ff8000000000000LL);
}

template <typename R>
lks_status upload_maps_async(lks_handle* h) {
  const double A = (1.0 / 6.0 - h->d.nu) * 4.5;
  EdgeMaps m;
  for (int cls = 0; cls < 9; ++cls) flow_moment_map(A, cls, &m.v[cls * 60], &m.v[540 + cls * 6]);
  fill_edge_maps_kernel<R><<<1, 256, 0, h->stream>>>(m, reinterpret_cast<R*>(h->ws + h->L.emap));
  CKH(h, cudaGetLastError());
  ++h->launches;
  return LKS_OK;
}

template <typename R>
lks_status noalloc_run(lks_handle* h, const void* gamma_dev, double* J_dev, void* grad_dev) {
  lks_status s = set_smem_attrs<R>();
  if (s == LKS_OK) s = upload_maps_async<R>(h);
  if (s == LKS_OK) s = forward_impl<R>(h, gamma_dev, J_dev);
  if (s == LKS_OK) s = adjoint_impl<R>(h);
  if (s == LKS_OK) s = sensitivity_impl<R>(h, grad_dev);
  if (s == LKS_OK) {
    flag_status_kernel<<<1, 1, 0, h->stream>>>(reinterpret_cast<const int*>(h->ws + h->L.status), J_dev);
    if (cudaGetLastError() != cudaSuccess) s = LKS_ERR_CUDA;
  }
  return s;
}
}  // namespace

extern "C" {

lks_status lks_gradient_noalloc(const lks_problem_desc* desc, const void* gamma_dev, double* J_dev,
                                void* dJdgamma_dev, void* stream) {
  if (!gamma_dev || !J_dev || !dJdgamma_dev) return LKS_ERR_INVALID_ARG;
  lks_status s = check_desc(desc, nullptr);
  if (s != LKS_OK) return s;
  if (desc->lattice != LKS_LATTICE_D2Q9) return LKS_ERR_INVALID_ARG;
  if (desc->tol > 0.0) return LKS_ERR_INVALID_ARG;  // a tolerance march reads its change back (synchronises)
  const Layout L = make_layout(desc, false);  // one segment store: this entry point has one stream
  if (L.total > LKS_NOALLOC_SCRATCH_BYTES) return LKS_ERR_WORKSPACE;  // problem too large
  void* ws = nullptr;
  int dev = 0;
  if ((s = noalloc_scratch(&ws, &dev)) != LKS_OK) return s;
  lks_handle h;
  h.d = *desc;
  h.L = L;
  h.ws = reinterpret_cast<unsigned char*>(ws);
  h.ws_bytes = LKS_NOALLOC_SCRATCH_BYTES;
  h.stream = reinterpret_cast<cudaStream_t>(stream);
  h.device = dev;
  return desc->real_type == LKS_REAL_F64 ? noalloc_run<double>(&h, gamma_dev, J_dev, dJdgamma_dev)
                                         : noalloc_run<float>(&h, gamma_dev, J_dev, dJdgamma_dev);
}

lks_status lks_selftest_wait(int32_t which, int32_t* scratch, void* stream, int32_t* recorded) {
  if ((which != 0 && which != 1) || !scratch || !recorded) return LKS_ERR_INVALID_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (cudaMemsetAsync(scratch, 0, 2 * sizeof(int32_t), s) != cudaSuccess) return LKS_ERR_CUDA;
  selftest_wait_kernel<<<1, 32, 0, s>>>(which, scratch, scratch + 1);
  if (cudaGetLastError() != cudaSuccess) return LKS_ERR_CUDA;
  int32_t st = 0;
  if (cudaMemcpyAsync(&st, scratch + 1, sizeof(int32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return LKS_ERR_CUDA;
  *recorded = st;
  return LKS_OK;
}

lks_status lks_edge_objective_map(double A, int32_t cls, double* out) {
  if (!out || cls < 0 || cls > 8) return LKS_ERR_INVALID_ARG;
  double full[60];
  flow_moment_map(A, cls, full, out);
  return LKS_OK;
}

lks_status lks_edge_moment_map(double A, int32_t cls, double* out) {
  if (!out || cls < 0 || cls > 8) return LKS_ERR_INVALID_ARG;
  double full[60];
  flow_moment_map(A, cls, full);
  for (int r = 0; r < 6; ++r)
    for (int k = 0; k < 10; ++k) out[r * 10 + k] = full[r * 10 + k];
  return LKS_OK;
}

}  // extern "C"
